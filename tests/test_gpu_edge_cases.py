"""GPU edge cases of the whole path: a scene without contacts, one contact,
invalid arguments (status codes, no fault)."""
import numpy as np
import pytest
import torch

from gpu_common import Problem, assert_close, to_np
from oracle import contacts as oc, qp, timestep
from paper_1808_02558_gb300 import binding
from synth import Scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return binding.Context()


def free_sphere():
    z = np.zeros((1, 3))
    return Scene(name="free", pos=[[0.0, 0.0, 3.0]], vel=[[0.2, 0.0, -0.1]], omega=z, radius=[0.5])


def test_no_contacts_whole_path(ctx):
    pb = Problem(ctx, free_sphere())
    assert pb.con.Nc == 0 and pb.con.P == 2
    g = torch.zeros(pb.con.P, dtype=torch.float64, device="cuda")
    lam = torch.zeros(1, dtype=torch.float64, device="cuda")  # no multipliers; a non-null buffer
    st = pb.ctx.state(g, lam)
    pb.ctx.pdip_init(st, 1.0)
    assert torch.count_nonzero(g).item() == 0
    rhs = torch.full((pb.con.P,), 5.0, dtype=torch.float64, device="cuda")
    pb.ctx.newton_rhs(st, rhs)
    assert torch.count_nonzero(rhs).item() == 0
    x = torch.randn(pb.con.P, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    pb.ctx.newton_apply(st, x, y)
    assert torch.equal(x, y)  # identity (dummy) rows only
    dx = torch.full_like(rhs, 3.0)
    stats = pb.ctx.newton_solve(st, rhs, dx, pb.ctx.solve_opts(tol=1e-10), allow=())
    assert stats.iters == 0 and torch.count_nonzero(dx).item() == 0
    eta, rd = pb.ctx.pdip_measure(st)
    assert eta == 0.0 and rd == 0.0
    ps, n = pb.ctx.pdip_solve(st, pb.ctx.pdip_opts(pb.ctx.solve_opts(tol=1e-10)), allow=())
    assert ps.status == binding.QP_OK and n == 0
    # the time step is free fall
    pb.ctx.advance(st)
    s1 = timestep.advance(pb.scene, pb.oc, np.zeros(0))
    assert_close(to_np(pb.dev["vel"]).reshape(3, -1).T, s1.vel, 1e-15, floor_rel=1e-3, what="free fall")
    # a warm start from an empty previous set
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    pb.ctx.pdip_init_warm(st, e, e, torch.zeros(0, dtype=torch.float64, device="cuda"), 3)


def test_invalid_arguments_return_status(ctx):
    pb = Problem(ctx, Scene(name="sop", pos=[[0.2, 0.1, 0.49]], vel=[[0.1, 0, 0]], omega=np.zeros((1, 3)),
                            radius=[0.5]))
    g = torch.zeros(pb.con.P, dtype=torch.float64, device="cuda")
    lam = torch.ones(2, dtype=torch.float64, device="cuda")
    st = pb.ctx.state(g, lam)
    rhs = torch.zeros(pb.con.P, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.QPError) as e:
        pb.ctx.newton_solve(st, rhs, rhs, pb.ctx.solve_opts(tol=-1.0), allow=())
    assert e.value.code == binding.QP_INVALID_ARG
    with pytest.raises(binding.QPError) as e:
        pb.ctx.newton_solve(st, rhs, rhs, pb.ctx.solve_opts(binding.QP_QTT_PCG, None, tol=1e-8), allow=())
    assert e.value.code == binding.QP_INVALID_ARG
    with pytest.raises(binding.QPError) as e:
        pb.ctx.pdip_init(st, -1.0)
    assert e.value.code == binding.QP_INVALID_ARG
    with pytest.raises(binding.QPError) as e:
        pb.ctx.pdip_init_warm(st, torch.zeros(1, dtype=torch.int32, device="cuda"),
                              torch.zeros(1, dtype=torch.int32, device="cuda"),
                              torch.zeros(3, dtype=torch.float64, device="cuda"), 5)
    assert e.value.code == binding.QP_INVALID_ARG
    x = torch.zeros(pb.con.P, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.QPError) as e:
        pb.ctx.newton_apply(st, x, x)  # aliased
    assert e.value.code == binding.QP_INVALID_ARG
    # the context stays usable after the errors
    pb.ctx.pdip_init(st, 1.0)
    eta, rd = pb.ctx.pdip_measure(st)
    assert np.isfinite(eta) and eta > 0


def test_context_without_contacts_is_not_ready():
    c = binding.Context()
    g = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = c.state(g, g)
    with pytest.raises(binding.QPError) as e:
        c.pdip_init(st, 1.0)
    assert e.value.code == binding.QP_NOT_READY
    c.close()
