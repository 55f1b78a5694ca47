"""GPU parity: PDIP iterations against the oracle (Sec. 2.4), entry by entry.

Tolerances (stated per quantity; |got - want| <= rtol * max(|want|, floor)):
* one step with FP64 Newton solves to 1e-12: gamma+ 1e-8 (floor 1e-4 max|gamma|),
  lambda+ 1e-8 (floor 1e-6 max|lambda|).  Solving the oracle's own step with
  Jacobi-PCG at 1e-12 instead of Cholesky moves these entries by at most 3e-9.
* final impulses of a converged PDIP: 1e-6 relative per entry, gamma and
  D gamma (the body impulses), as the impulse bar of the method states.
"""
import numpy as np
import pytest
import torch

from gpu_common import Problem, assert_close, dev, to_np
from oracle import pdip, qp
from paper_1808_02558_gb300 import binding
from synth import Scene, lattice_scene, scene_for
from test_oracle_pdip import closed_form
from test_oracle_qp import sphere_on_plane

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return binding.Context()


def gpu_opts(ctx, tol=1e-12):
    return ctx.pdip_opts(ctx.solve_opts(tol=tol, maxit=200000))


def check_step(stats, info, g_got, l_got, g1, l1, rtol=1e-8, s_tol=1e-8):
    assert abs(stats.eta - info.eta) <= 1e-12 * info.eta
    assert abs(stats.t - info.t) <= 1e-12 * info.t
    assert abs(stats.r_t - info.r_t_norm) <= 1e-10 * info.r_t_norm
    assert stats.halvings == info.halvings
    assert abs(stats.s - info.s) <= s_tol * info.s
    assert_close(g_got, g1, rtol, floor_rel=1e-4, what="gamma+")
    assert_close(l_got, l1, rtol, floor_rel=1e-6, what="lambda+")


def test_single_step_matches_oracle(ctx):
    pb = Problem(ctx, scene_for("pile8", 2))
    g, lam = pb.oracle_iterates(2)
    g1, l1, info = pdip.pdip_step(pb.N, pb.r, pb.scene.mu, g, lam)
    gd, ld, st = pb.state(g, lam)
    stats = pb.ctx.pdip_step(st, gpu_opts(pb.ctx), allow=())
    check_step(stats, info, pb.unpad(to_np(gd)), to_np(ld), g1, l1)


def run_gpu_pdip(ctx, pb, iters, tol_gap=None, opts=None):
    ctx = pb.ctx
    g0, l0 = qp.initial_point(pb.Nc, pb.scene.mu)
    gd, ld, st = pb.state(g0, l0)
    ctx.pdip_init(st, 1.0)
    assert np.array_equal(pb.unpad(to_np(gd)), g0)
    assert_close(to_np(ld), l0, 1e-15, what="cold-start lambda")
    opts = opts or gpu_opts(ctx)
    for _ in range(iters):
        if tol_gap is not None:
            eta, _ = ctx.pdip_measure(st)
            if eta <= tol_gap:
                break
        ctx.pdip_step(st, opts, allow=())
    return pb.unpad(to_np(gd)), to_np(ld)


def test_trajectory_pile8(ctx):
    """Six PDIP iterations from the cold start; per-step deviations of about 1e-9
    compound along the trajectory, hence 1e-6 per entry."""
    pb = Problem(ctx, scene_for("pile8", 1))
    K = 6
    g, lam = pb.oracle_iterates(K)
    gg, ll = run_gpu_pdip(ctx, pb, K)
    assert_close(gg, g, 1e-6, floor_rel=1e-4, what="gamma after 6 iterations")
    assert_close(ll, lam, 1e-6, floor_rel=1e-6, what="lambda after 6 iterations")


@pytest.mark.parametrize("vel,kind", [((0.01, 0.0, -0.5), "stick"), ((2.0, 0.5, -0.1), "slip")])
def test_sphere_on_plane_final_impulses(ctx, vel, kind):
    s = sphere_on_plane(vel)
    pb = Problem(ctx, s)
    want, k = closed_form(s.mass[0], s.mu, pb.r[0], pb.r[1:3])
    assert k == kind
    gg, _ = run_gpu_pdip(ctx, pb, 200, tol_gap=1e-12)
    assert np.allclose(gg, want, rtol=0, atol=1e-6 * max(1.0, np.abs(want).max()) * s.mass[0])


def test_small_lattice_final_impulses(ctx):
    s = lattice_scene(2, 1)
    pb = Problem(ctx, s)
    res = pdip.pdip_solve(pb.N, pb.r, s.mu, tol_gap=1e-8, tol_dual=1e-6, maxit=200)
    gg, _ = run_gpu_pdip(ctx, pb, res.iters)
    assert_close(gg, res.gamma, 1e-6, floor_rel=1e-3, what="final gamma, 2^3 lattice")
    assert_close(pb.D @ gg, pb.D @ res.gamma, 1e-6, floor_rel=1e-3, what="final D gamma, 2^3 lattice")


@pytest.mark.parametrize("mixed", [0, 1])
def test_stack_final_impulses(ctx, mixed):
    """16 x 16 columns of 10 spheres (2560 contacts, 2^13 padded unknowns), the
    benchmark's dt, mu and velocity recipe: every contact carries load, so the
    PDIP of Sec. 2.4 converges to gap 1e-8 and dual residual 1e-8.  pdip_solve
    on the GPU (FP64 Newton solves, or FP32 inner PCG with FP64 refinement)
    against the oracle's loop with direct solves: final impulses and body
    impulses D gamma to 1e-6 per entry, purely relative (the oracle's result
    moves by 1e-13 when its solver changes)."""
    s = scene_for("stack16", 1)
    pb = Problem(ctx, s)
    assert pb.P == 1 << 13
    res = pdip.pdip_solve(pb.N, pb.r, s.mu, tol_gap=1e-8, tol_dual=1e-8, maxit=200)
    assert res.converged
    g0, l0 = qp.initial_point(pb.Nc, s.mu)
    gd, ld, st = pb.state(g0, l0)
    pb.ctx.pdip_init(st, 1.0)
    so = pb.ctx.solve_opts(tol=1e-12, maxit=200000, mixed=mixed, inner_tol=1e-3 if mixed else 0.0, max_outer=60)
    stats, n = pb.ctx.pdip_solve(st, pb.ctx.pdip_opts(so), gap_tol=1e-8, dual_tol=1e-8, max_iter=200, allow=())
    assert stats.status == binding.QP_OK and stats.eta <= 1e-8 and stats.r_dual <= 1e-8
    assert abs(n - res.iters) <= 1
    gg = pb.unpad(to_np(gd))
    assert_close(gg, res.gamma, 1e-6, what="final gamma, columns")
    assert_close(pb.D @ gg, pb.D @ res.gamma, 1e-6, floor_rel=1e-9, what="final D gamma, columns")
    assert_close(to_np(ld), res.lam, 1e-6, what="final lambda, columns")


def test_single_step_with_qtt_refresh_matches_oracle(ctx):
    """pdip_step with the QTT refresh (compress + invert + QTT-PCG) takes the oracle's step."""
    pb = Problem(ctx, scene_for("pile8", 3))
    g, lam = pb.oracle_iterates(2)
    g1, l1, info = pdip.pdip_step(pb.N, pb.r, pb.scene.mu, g, lam)
    gd, ld, st = pb.state(g, lam)
    so = pb.ctx.solve_opts(binding.QP_QTT_PCG, None, tol=1e-12, maxit=100000)
    opts = pb.ctx.pdip_opts(so, qtt_refresh=1, qtt_eps=1e-2, qtt_rmax=10)
    stats = pb.ctx.pdip_step(st, opts, allow=())
    assert stats.ms_refresh > 0
    check_step(stats, info, pb.unpad(to_np(gd)), to_np(ld), g1, l1)
    # second step warm-starts the inverse from the context's previous one
    g2, l2, _ = pdip.pdip_step(pb.N, pb.r, pb.scene.mu, g1, l1)
    pb.ctx.pdip_step(st, opts, allow=())
    assert_close(pb.unpad(to_np(gd)), g2, 1e-7, floor_rel=1e-4, what="gamma after two QTT steps")
    assert_close(to_np(ld), l2, 1e-7, floor_rel=1e-6, what="lambda after two QTT steps")


def test_pdip_solve_loop_matches_oracle(ctx):
    """pdip_solve runs the loop of Sec. 2.4 to the tolerances: same iterate and
    iteration count as the oracle's loop."""
    s = lattice_scene(2, 1)
    pb = Problem(ctx, s)
    res = pdip.pdip_solve(pb.N, pb.r, s.mu, tol_gap=1e-8, tol_dual=1e-6, maxit=200)
    assert res.converged
    g0, l0 = qp.initial_point(pb.Nc, s.mu)
    gd, ld, st = pb.state(g0, l0)
    pb.ctx.pdip_init(st, 1.0)
    stats, n = pb.ctx.pdip_solve(st, gpu_opts(pb.ctx), gap_tol=1e-8, dual_tol=1e-6, max_iter=200, allow=())
    assert stats.status == binding.QP_OK
    assert abs(n - res.iters) <= 1
    assert stats.eta <= 1e-8 and stats.r_dual <= 1e-6
    assert_close(pb.unpad(to_np(gd)), res.gamma, 1e-6, floor_rel=1e-3, what="pdip_solve gamma")


def test_pdip_solve_sphere_on_plane_and_cap(ctx):
    s = sphere_on_plane((2.0, 0.5, -0.1))
    pb = Problem(ctx, s)
    want, k = closed_form(s.mass[0], s.mu, pb.r[0], pb.r[1:3])
    g0, l0 = qp.initial_point(pb.Nc, s.mu)
    gd, ld, st = pb.state(g0, l0)
    pb.ctx.pdip_init(st, 1.0)
    stats, n = pb.ctx.pdip_solve(st, gpu_opts(pb.ctx), gap_tol=1e-12, dual_tol=1e-9, max_iter=200, allow=())
    assert 0 < n < 200
    gg = pb.unpad(to_np(gd))
    assert np.allclose(gg, want, rtol=0, atol=1e-6 * max(1.0, np.abs(want).max()) * s.mass[0])
    # a cap below the iterations needed returns QP_NOT_CONVERGED after exactly that many steps
    gd2, ld2, st2 = pb.state(g0, l0)
    pb.ctx.pdip_init(st2, 1.0)
    stats2, n2 = pb.ctx.pdip_solve(st2, gpu_opts(pb.ctx), gap_tol=1e-12, dual_tol=1e-9, max_iter=2)
    assert stats2.status == binding.QP_NOT_CONVERGED and n2 == 2


def test_qtt_inverse_reuse_across_newton_iterations(ctx):
    """qtt_refresh = 0 without X reuses the context's last refreshed inverse
    (Sec. 3.3 re-use); with nothing refreshed yet it is an invalid argument."""
    pb = Problem(ctx, scene_for("pile8", 2))
    g, lam = pb.oracle_iterates(2)
    gd, ld, st = pb.state(g, lam)
    so = pb.ctx.solve_opts(binding.QP_QTT_PCG, None, tol=1e-10, maxit=20000)
    with pytest.raises(binding.QPError) as e:
        pb.ctx.pdip_step(st, pb.ctx.pdip_opts(so, qtt_refresh=0), allow=())
    assert e.value.code == binding.QP_INVALID_ARG
    s1 = pb.ctx.pdip_step(st, pb.ctx.pdip_opts(so, qtt_refresh=1, qtt_eps=1e-2, qtt_rmax=10), allow=())
    assert s1.ms_refresh > 0
    g2, l2, _ = pdip.pdip_step(pb.N, pb.r, pb.scene.mu, *pb.oracle_iterates(3))
    s2 = pb.ctx.pdip_step(st, pb.ctx.pdip_opts(so, qtt_refresh=0), allow=())
    assert s2.ms_refresh == 0 and s2.solve.rel_res <= 1e-10
    assert_close(pb.unpad(to_np(gd)), g2, 1e-7, floor_rel=1e-4, what="gamma after reuse")
