"""GPU parity on the 40^3 polydisperse pile (2^20 padded unknowns) at the PDIP
iterates the benchmark times, entry by entry.

The oracle runs PDIP iterations 0..7 from the cold start (Sec. 2.4; Newton
systems by its Jacobi-PCG to 1e-10) and keeps the iterates (gamma_k, lambda_k)
for k = 0, 3, 7: the late ones are the ill-conditioned systems (88 and 150 CG
iterations against 40 at k = 0).  At each, the library starts from the same
(gamma_k, lambda_k):

* Newton rhs (Sec. 3.3): 1e-12 of the per-entry magnitude sum |N||gamma| + |r| +
  |barrier term| (FP64 rounding of the sum);
* Newton solution (Eq. qp_Newton_system through the Schur complement): the
  library's mixed-precision solve (FP32 inner PCG, FP64 refinement, the
  benchmark's kernel) to relative residual 1e-12 against the oracle's solve to
  1e-14: 1e-8 per entry with a floor of 1e-3 max|dgamma| (the oracle's own
  1e-12 solve differs from its 1e-14 solve by <= 2.1e-10 on that scale);
* one PDIP iteration: surrogate gap, t, ||r_t||, halvings and step length, and
  gamma+ (floor 1e-4 max), lambda+ (floor 1e-6 max) to 1e-8; at the benchmark's
  own tolerance (1e-8 residual) to 1e-6 with floors 1e-3 / 1e-6.
"""
import numpy as np
import pytest
import torch

from gpu_common import Problem, assert_close, to_np
from oracle import krylov, pdip, qp
from paper_1808_02558_gb300 import binding
from synth import scene_for

pytestmark = pytest.mark.gpu

KEEP = (0, 3, 7)


def pcg(tol):
    def solve(S, b):
        x, info = krylov.jacobi_pcg(S, b, tol=tol, maxit=100000)
        return x, info["iters"]
    return solve


@pytest.fixture(scope="module")
def pile():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pb = Problem(None, scene_for("pile40p", 1))
    assert pb.P == 1 << 20
    mu = pb.scene.mu
    g, lam = qp.initial_point(pb.Nc, mu)
    pb.iter = {}
    for k in range(max(KEEP) + 1):
        if k in KEEP:
            pb.iter[k] = (g.copy(), lam.copy())
        if k < max(KEEP):
            g, lam, _ = pdip.pdip_step(pb.N, pb.r, mu, g, lam, newton_solver=pcg(1e-10))
    pb.step = {k: pdip.pdip_step(pb.N, pb.r, mu, *pb.iter[k], newton_solver=pcg(1e-14)) for k in KEEP}
    return pb


def mixed_opts(ctx, tol):
    return ctx.solve_opts(tol=tol, maxit=200000, mixed=1, inner_tol=1e-3, max_outer=80)


@pytest.mark.parametrize("k", [3, 7])
def test_newton_rhs_and_solution(pile, k):
    g, lam = pile.iter[k]
    mu = pile.scene.mu
    gd, ld, st = pile.state(g, lam)
    rhs = torch.empty(pile.P, dtype=torch.float64, device="cuda")
    pile.ctx.newton_rhs(st, rhs)
    f = qp.constraints(g, mu)
    t = pdip.NU * 2 * pile.Nc / float(-(f @ lam))
    want = qp.newton_rhs(pile.N, pile.r, g, lam, t, mu)
    bar = np.abs(qp.newton_rhs(pile.N, pile.r, g, lam, t, mu) + pile.N @ g + pile.r)
    scale = abs(pile.N) @ np.abs(g) + np.abs(pile.r) + bar
    assert_close(pile.unpad(to_np(rhs)), want, 1e-12, scale=scale, what=f"rhs at iterate {k}")
    dx = torch.empty_like(rhs)
    stats = pile.ctx.newton_solve(st, rhs, dx, mixed_opts(pile.ctx, 1e-12), allow=())
    assert stats.rel_res <= 1e-12
    info = pile.step[k][2]
    assert_close(pile.unpad(to_np(dx)), info.dgamma, 1e-8, floor_rel=1e-3, what=f"dgamma at iterate {k}")
    assert np.all(to_np(dx)[3 * pile.Nc:] == 0.0)


@pytest.mark.parametrize("k", KEEP)
def test_pdip_step(pile, k):
    g1, l1, info = pile.step[k]
    gd, ld, st = pile.state(*pile.iter[k])
    stats = pile.ctx.pdip_step(st, pile.ctx.pdip_opts(mixed_opts(pile.ctx, 1e-12)), allow=())
    assert stats.solve.rel_res <= 1e-12
    assert abs(stats.eta - info.eta) <= 1e-12 * info.eta
    assert abs(stats.t - info.t) <= 1e-12 * info.t
    assert abs(stats.r_t - info.r_t_norm) <= 1e-10 * info.r_t_norm
    assert stats.halvings == info.halvings
    assert abs(stats.s - info.s) <= 1e-8 * info.s
    assert_close(pile.unpad(to_np(gd)), g1, 1e-8, floor_rel=1e-4, what=f"gamma+ at iterate {k}")
    assert_close(to_np(ld), l1, 1e-8, floor_rel=1e-6, what=f"lambda+ at iterate {k}")


def test_pdip_step_at_benchmark_tolerance(pile):
    """The benchmark's launch configuration (residual 1e-8) at the latest iterate."""
    k = max(KEEP)
    g1, l1, info = pile.step[k]
    gd, ld, st = pile.state(*pile.iter[k])
    stats = pile.ctx.pdip_step(st, pile.ctx.pdip_opts(mixed_opts(pile.ctx, 1e-8)), allow=())
    assert stats.solve.rel_res <= 1e-8
    assert stats.halvings == info.halvings
    assert abs(stats.s - info.s) <= 1e-6 * info.s
    assert_close(pile.unpad(to_np(gd)), g1, 1e-6, floor_rel=1e-3, what="gamma+ at tol 1e-8")
    assert_close(to_np(ld), l1, 1e-6, floor_rel=1e-6, what="lambda+ at tol 1e-8")
