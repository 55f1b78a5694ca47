"""GPU parity: the time step around the CCP and the warm start of the next
PDIP (Sec. 2.3 Eqs. force_balance_disc, particle_evolution_disc; Sec. 3.3)."""
import numpy as np
import pytest
import torch

from gpu_common import Problem, assert_close, dev, to_np
from oracle import contacts as oc, pdip, qp, timestep
from paper_1808_02558_gb300 import binding, workload
from synth import box_scene, random_vector, scene_for
from test_gpu_newton import interior_point
from test_oracle_pdip import closed_form
from test_oracle_qp import sphere_on_plane

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return binding.Context()


def soa_to_np(t):
    return to_np(t).reshape(3, -1).T


@pytest.mark.parametrize("slots", [3, 4])
def test_advance_matches_oracle(ctx, slots):
    pb = Problem(ctx, scene_for("pile8", 3), slots=slots)
    g, lam = interior_point(pb, 7)
    gd, ld, st = pb.state(g, lam)
    pb.ctx.advance(st)
    s1 = timestep.advance(pb.scene, pb.oc, g)
    d = pb.dev
    assert_close(soa_to_np(d["vel"]), s1.vel, 1e-12, floor_rel=1e-3, what="velocity")
    assert_close(soa_to_np(d["omega"]), s1.omega, 1e-12, floor_rel=1e-3, what="angular velocity")
    assert_close(soa_to_np(d["pos"]), s1.pos, 1e-15, floor_rel=1e-3, what="position")


def test_advance_sticking_sphere_contact_at_rest(ctx):
    s = sphere_on_plane((0.01, 0.0, -0.5))
    pb = Problem(ctx, s)
    want, kind = closed_form(s.mass[0], s.mu, pb.r[0], pb.r[1:3])
    assert kind == "stick"
    gd, ld, st = pb.state(want, np.ones(2))
    pb.ctx.advance(st)
    v = soa_to_np(pb.dev["vel"])[0]
    w = soa_to_np(pb.dev["omega"])[0]
    vc = v + np.cross(w, [0.0, 0.0, -s.radius[0]])
    assert np.allclose(vc, 0.0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("slots", [3, 4])
def test_warm_start_after_step_matches_oracle(ctx, slots):
    pb = Problem(ctx, scene_for("pile8", 4), slots=slots)
    g, lam = interior_point(pb, 9)
    gd, ld, st = pb.state(g, lam)
    prev_a = workload.view(pb.con, "body_a")
    prev_b = workload.view(pb.con, "body_b")
    prev_g = gd.clone()
    pb.ctx.advance(st)
    # next step: re-assemble on the advanced positions
    s = pb.scene
    con1 = pb.ctx.assemble(pb.dev, s.floor_z, s.gravity, s.dt, s.delta, s.mu, slots)
    s1 = timestep.advance(s, pb.oc, g)
    oc1 = oc.detect(s1)
    assert con1.Nc == oc1.Nc
    assert np.array_equal(to_np(workload.view(con1, "body_a")), oc1.a)
    assert np.array_equal(to_np(workload.view(con1, "body_b")), oc1.b)
    L, P = qp.padded_size(oc1.Nc, slots)
    g1 = torch.zeros(P, dtype=torch.float64, device="cuda")
    l1 = torch.zeros(2 * oc1.Nc, dtype=torch.float64, device="cuda")
    st1 = pb.ctx.state(g1, l1)
    pb.ctx.pdip_init_warm(st1, prev_a, prev_b, prev_g, slots, gn0=1.0, shrink=0.9)
    want_g, want_l = timestep.warm_start(pb.oc.a, pb.oc.b, g, oc1.a, oc1.b, s.mu, gn0=1.0, shrink=0.9)
    got = qp.from_padded(to_np(g1), oc1.Nc, slots)
    assert_close(got, want_g, 1e-15, floor_rel=1e-6, what="warm gamma")
    assert_close(to_np(l1), want_l, 1e-13, floor_rel=1e-9, what="warm lambda")
    assert np.array_equal(to_np(g1), qp.to_padded(got, oc1.Nc, slots, P))  # dummy rows zero
    # most contacts persist over one step of this pile
    persist = len({(a, b) for a, b in zip(pb.oc.a, pb.oc.b)} & {(a, b) for a, b in zip(oc1.a, oc1.b)})
    assert persist >= 0.9 * oc1.Nc


@pytest.mark.parametrize("walled", [False, True])
def test_three_time_steps_match_oracle(ctx, walled):
    """assemble -> (warm) init -> 4 PDIP iterations -> advance, three times; on
    the 8^3 pile, and on a 6 x 6 x 3 walled box (floor and four side walls)."""
    s = box_scene(3, n=6, layers=3) if walled else scene_for("pile8", 5)
    sctx = binding.Context()
    dev_s, con = workload.assemble(sctx, s)
    opts = sctx.pdip_opts(sctx.solve_opts(tol=1e-12, maxit=200000))
    so = s
    prev = None
    for step in range(3):
        if step > 0:
            con = sctx.assemble(dev_s, s.floor_z, s.gravity, s.dt, s.delta, s.mu, 3, s.walls)
        c_o = oc.detect(so)
        if walled:
            assert int((c_o.a == so.M).sum()) > 4 * 6 * 3  # wall and floor contacts in every step
        _, N, r = qp.qp_data(so, c_o)
        assert con.Nc == c_o.Nc
        g_d = torch.zeros(con.P, dtype=torch.float64, device="cuda")
        l_d = torch.zeros(2 * con.Nc, dtype=torch.float64, device="cuda")
        st = sctx.state(g_d, l_d)
        if prev is None:
            sctx.pdip_init(st, 1.0)
            g_o, l_o = qp.initial_point(c_o.Nc, so.mu)
        else:
            # with walls a sphere can have several contacts with body M: the
            # plane index keeps them apart on both sides
            sctx.pdip_init_warm(st, prev[0], prev[1], prev[2], 3, prev_plane=prev[6] if walled else None)
            g_o, l_o = timestep.warm_start(prev[3], prev[4], prev[5], c_o.a, c_o.b, so.mu,
                                           prev_plane=prev[7] if walled else None,
                                           new_plane=c_o.plane if walled else None)
        for _ in range(4):
            sctx.pdip_step(st, opts, allow=())
            g_o, l_o, _ = pdip.pdip_step(N, r, so.mu, g_o, l_o)
        assert_close(qp.from_padded(to_np(g_d), con.Nc, 3), g_o, 1e-6, floor_rel=1e-4, what=f"gamma, step {step}")
        prev = (workload.view(con, "body_a"), workload.view(con, "body_b"), g_d.clone(), c_o.a, c_o.b, g_o,
                workload.view(con, "plane"), c_o.plane)
        sctx.advance(st)
        so = timestep.advance(so, c_o, g_o)
    assert_close(soa_to_np(dev_s["vel"]), so.vel, 1e-6, floor_rel=1e-3, what="velocity after three steps")
    assert_close(soa_to_np(dev_s["pos"]), so.pos, 1e-12, floor_rel=1e-3, what="position after three steps")
