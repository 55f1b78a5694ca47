"""GPU parity: fused Schur apply, Newton rhs and the persistent PCG solve (Sec. 2.4, 3.3).

Entry-by-entry checks: an operator apply y = S x to rtol times the per-entry
magnitude sum (|S| |x|)_i (1e-12 in FP64, 1e-5 in FP32, whose data are rounded
to float32), a Newton solution to 1e-8 of max(|x_i|, 1e-3 max|x|) against
Cholesky.  Residual norms are checked as norms."""
import numpy as np
import pytest
import scipy.linalg as sla
import torch

from gpu_common import Problem, assert_close, dev, to_np
from oracle import pdip, qp
from paper_1808_02558_gb300 import binding
from synth import lattice_scene, random_vector, scene_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return binding.Context()


@pytest.fixture(scope="module")
def pile8(ctx):
    pb = Problem(ctx, scene_for("pile8", 1))
    pb.iters = {k: pb.oracle_iterates(k) for k in (0, 3)}
    return pb


def interior_point(pb, seed=0):
    """A strictly feasible (gamma, lambda) with spread values (no PDIP run)."""
    rng = np.random.default_rng(seed)
    g = np.zeros(3 * pb.Nc)
    g[0::3] = rng.uniform(0.5, 20.0, pb.Nc)
    ang = rng.uniform(0, 2 * np.pi, pb.Nc)
    rad = rng.uniform(0, 0.9, pb.Nc) * pb.scene.mu * g[0::3]
    g[1::3], g[2::3] = rad * np.cos(ang), rad * np.sin(ang)
    lam = rng.uniform(0.01, 5.0, 2 * pb.Nc)
    return g, lam


def check_apply(pb, g, lam, tol64=1e-12, tol32=1e-5):
    x = random_vector(7, 1, pb.P)
    xd = dev(x)
    y = torch.empty_like(xd)
    # plain N
    pb.ctx.newton_apply(None, xd, y)
    want = pb.pad(pb.N @ pb.unpad(x))
    dummy = np.ones(pb.P, bool)
    dummy[(pb.slots * np.arange(pb.Nc)[:, None] + np.arange(3)).reshape(-1)] = False
    want[dummy] = x[dummy]
    scale = pb.pad(abs(pb.N) @ np.abs(pb.unpad(x)))
    scale[dummy] = np.abs(x[dummy])
    assert_close(to_np(y), want, tol64, scale=scale, what="N x")
    # Schur S at (g, lam)
    gd, ld, st = pb.state(g, lam)
    pb.ctx.newton_apply(st, xd, y)
    S = qp.schur_matrix(pb.N, g, lam, pb.scene.mu)
    want = pb.pad(S @ pb.unpad(x))
    want[dummy] = x[dummy]
    scale = pb.pad(abs(S) @ np.abs(pb.unpad(x)))
    scale[dummy] = np.abs(x[dummy])
    assert_close(to_np(y), want, tol64, scale=scale, what="S x")
    x32 = xd.float()
    y32 = torch.empty_like(x32)
    pb.ctx.newton_apply(st, x32, y32, binding.QP_F32)
    assert_close(to_np(y32).astype(np.float64), want, tol32, scale=scale, what="S x in FP32")


def test_apply_pile8_iterate(pile8):
    g, lam = pile8.iters[3]
    check_apply(pile8, g, lam)


@pytest.mark.parametrize("slots", [3, 4])
def test_apply_polydisperse_slots(ctx, slots):
    pb = Problem(ctx, lattice_scene(6, 3, polydisperse=True), slots)
    check_apply(pb, *interior_point(pb, 1))


def test_apply_full_size_pile40p(ctx):
    pb = Problem(ctx, scene_for("pile40p", 1))
    assert pb.P == 1 << 20
    check_apply(pb, *interior_point(pb, 2))


def test_rhs_and_t(pile8):
    g, lam = pile8.iters[3]
    gd, ld, st = pile8.state(g, lam)
    rhs = torch.empty(pile8.P, dtype=torch.float64, device="cuda")
    pile8.ctx.newton_rhs(st, rhs)
    f = qp.constraints(g, pile8.scene.mu)
    t = pdip.NU * 2 * pile8.Nc / float(-(f @ lam))
    assert abs(st.t - t) <= 1e-12 * t
    want = qp.newton_rhs(pile8.N, pile8.r, g, lam, t, pile8.scene.mu)
    bar = np.abs(want + pile8.N @ g + pile8.r)
    scale = abs(pile8.N) @ np.abs(g) + np.abs(pile8.r) + bar
    assert_close(pile8.unpad(to_np(rhs)), want, 1e-12, scale=scale, what="Newton rhs")
    assert np.all(to_np(rhs)[3 * pile8.Nc:] == 0.0)


@pytest.mark.parametrize("k", [0, 3])
def test_solve_jacobi_fp64_matches_cholesky(pile8, k):
    g, lam = pile8.iters[k]
    gd, ld, st = pile8.state(g, lam)
    rhs = torch.empty(pile8.P, dtype=torch.float64, device="cuda")
    pile8.ctx.newton_rhs(st, rhs)
    dx = torch.empty_like(rhs)
    stats = pile8.ctx.newton_solve(st, rhs, dx, pile8.ctx.solve_opts(tol=1e-12, maxit=50000), allow=())
    S = qp.schur_matrix(pile8.N, g, lam, pile8.scene.mu)
    b = pile8.unpad(to_np(rhs))
    exact = sla.cho_solve(sla.cho_factor(S.toarray()), b)
    x = pile8.unpad(to_np(dx))
    assert np.linalg.norm(b - S @ x) <= 1e-11 * np.linalg.norm(b)
    assert stats.rel_res <= 1e-12 * 1.0001
    assert_close(x, exact, 1e-8, floor_rel=1e-3, what="dgamma vs Cholesky")
    assert np.all(to_np(dx)[3 * pile8.Nc:] == 0.0)


def test_solve_mixed_precision_full_size(ctx):
    pb = Problem(ctx, scene_for("pile40p", 1))
    g, lam = interior_point(pb, 3)
    gd, ld, st = pb.state(g, lam)
    rhs = torch.empty(pb.P, dtype=torch.float64, device="cuda")
    pb.ctx.newton_rhs(st, rhs)
    dx = torch.empty_like(rhs)
    opts = pb.ctx.solve_opts(tol=1e-8, maxit=100000, mixed=1, inner_tol=1e-3, max_outer=60)
    stats = pb.ctx.newton_solve(st, rhs, dx, opts, allow=())
    S = qp.schur_matrix(pb.N, g, lam, pb.scene.mu)
    b = pb.unpad(to_np(rhs))
    res = np.linalg.norm(b - S @ pb.unpad(to_np(dx))) / np.linalg.norm(b)
    assert res <= 1.05e-8 and stats.rel_res <= 1e-8
    assert abs(res - stats.rel_res) <= 1e-9


@pytest.mark.parametrize("mixed", [0, 1])
def test_failed_pipelined_solve_falls_back_on_fresh_context(ctx, mixed):
    """The first solve of a fresh context runs the pipelined kernel (small
    system), fails on an unattainable tolerance and is redone by the classic
    kernel, whose work vectors must survive the pipelined solver's allocations."""
    pb = Problem(ctx, scene_for("pile8", 2))
    g, lam = interior_point(pb, 1)
    gd, ld, st = pb.state(g, lam)
    rhs = torch.empty(pb.P, dtype=torch.float64, device="cuda")
    pb.ctx.newton_rhs(st, rhs)
    dx = torch.empty_like(rhs)
    opts = pb.ctx.solve_opts(tol=1e-30, maxit=40, mixed=mixed, inner_tol=1e-3 if mixed else 0.0, max_outer=2)
    stats = pb.ctx.newton_solve(st, rhs, dx, opts)
    assert stats.status in (binding.QP_NOT_CONVERGED, binding.QP_BREAKDOWN)
    assert torch.isfinite(dx).all().item()
    opts = pb.ctx.solve_opts(tol=1e-10, maxit=50000, mixed=mixed, inner_tol=1e-3 if mixed else 0.0, max_outer=60)
    stats = pb.ctx.newton_solve(st, rhs, dx, opts, allow=())
    S = qp.schur_matrix(pb.N, g, lam, pb.scene.mu)
    b = pb.unpad(to_np(rhs))
    assert np.linalg.norm(b - S @ pb.unpad(to_np(dx))) <= 1.05e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("eps", [1e-12, 0.02, 0.1])
def test_qtt_direct_mode_refines_to_tolerance(ctx, eps):
    """QTT direct mode (Sec. 3.3): dx += X (rhs - S dx) with X the TT-SVD of the
    exact inverse at eps.  On this 16-contact system an exact X needs one or two
    steps; eps = 0.02 truncates the middle rank (spectral radius of I - S X
    about 0.25, so many steps); eps = 0.1 makes it exceed 1 (1.27), the
    refinement diverges and the solve falls back to Jacobi-PCG."""
    from oracle import tt
    pb = Problem(ctx, lattice_scene(2, 1))
    g, lam = interior_point(pb, 4)
    gd, ld, st = pb.state(g, lam)
    rhs = torch.empty(pb.P, dtype=torch.float64, device="cuda")
    pb.ctx.newton_rhs(st, rhs)
    S = qp.schur_matrix(pb.N, g, lam, pb.scene.mu)
    Sp = qp.padded_matrix(S, pb.Nc, 3, pb.P).toarray()
    X = pb.ctx.qtt_from_cores(tt.qtt_inverse_dense(Sp, eps))
    dx = torch.empty_like(rhs)
    opts = pb.ctx.solve_opts(binding.QP_QTT_DIRECT, X, tol=1e-11, maxit=1000, max_outer=200)
    stats = pb.ctx.newton_solve(st, rhs, dx, opts, allow=())
    b = pb.unpad(to_np(rhs))
    res = np.linalg.norm(b - S @ pb.unpad(to_np(dx))) / np.linalg.norm(b)
    assert res <= 1.05e-11 and stats.rel_res <= 1e-11
    if eps == 0.1:
        assert stats.fallback == 1
        return
    assert stats.fallback == 0 and stats.iters == stats.outer
    if eps < 1e-10:
        assert stats.outer <= 2
    else:
        assert 5 <= stats.outer <= 40


def test_solve_zero_rhs(pile8):
    g, lam = pile8.iters[0]
    gd, ld, st = pile8.state(g, lam)
    rhs = torch.zeros(pile8.P, dtype=torch.float64, device="cuda")
    dx = torch.full_like(rhs, 7.0)
    stats = pile8.ctx.newton_solve(st, rhs, dx, pile8.ctx.solve_opts(tol=1e-10), allow=())
    assert stats.iters == 0 and torch.count_nonzero(dx).item() == 0


@pytest.mark.parametrize("mixed", [0, 1])
def test_solve_qtt_preconditioned(pile8, mixed):
    """QTT-PCG (Sec. 3.3): S compressed and inverted in QTT, applied inside the PCG."""
    g, lam = pile8.iters[3]
    gd, ld, st = pile8.state(g, lam)
    rhs = torch.empty(pile8.P, dtype=torch.float64, device="cuda")
    pile8.ctx.newton_rhs(st, rhs)
    S_tt = pile8.ctx.qtt_compress(st, 1e-2, 10)
    X = pile8.ctx.qtt_inverse(S_tt, 1e-2, 10, sweeps=3)
    dx = torch.empty_like(rhs)
    opts = pile8.ctx.solve_opts(binding.QP_QTT_PCG, X, tol=1e-10, maxit=20000, mixed=mixed,
                                inner_tol=1e-3 if mixed else 0.0, max_outer=60,
                                core_dtype=binding.QP_BF16 if mixed else binding.QP_F32)
    stats = pile8.ctx.newton_solve(st, rhs, dx, opts, allow=())
    S = qp.schur_matrix(pile8.N, g, lam, pile8.scene.mu)
    b = pile8.unpad(to_np(rhs))
    res = np.linalg.norm(b - S @ pile8.unpad(to_np(dx))) / np.linalg.norm(b)
    assert res <= 1.05e-10 and stats.rel_res <= 1e-10
    jac = pile8.ctx.newton_solve(st, rhs, torch.empty_like(rhs),
                                 pile8.ctx.solve_opts(tol=1e-10, maxit=20000, mixed=mixed,
                                                      inner_tol=1e-3 if mixed else 0.0, max_outer=60), allow=())
    print(f"QTT-PCG iters {stats.iters} vs Jacobi-PCG {jac.iters} (mixed={mixed})")


@pytest.mark.parametrize("mixed", [0, 1])
def test_solve_bicgstab_jacobi_and_qtt(pile8, mixed):
    """BiCGSTAB (the paper's Sec. 4.2 Krylov method), Jacobi and QTT preconditioned."""
    g, lam = pile8.iters[3]
    gd, ld, st = pile8.state(g, lam)
    rhs = torch.empty(pile8.P, dtype=torch.float64, device="cuda")
    pile8.ctx.newton_rhs(st, rhs)
    S = qp.schur_matrix(pile8.N, g, lam, pile8.scene.mu)
    b = pile8.unpad(to_np(rhs))
    X = pile8.ctx.qtt_inverse(pile8.ctx.qtt_compress(st, 1e-2, 10), 1e-2, 10, sweeps=3)
    tol = 1e-10 if mixed else 1e-12
    for precond, Xh in ((binding.QP_JACOBI_PCG, None), (binding.QP_QTT_PCG, X)):
        dx = torch.empty_like(rhs)
        opts = pile8.ctx.solve_opts(precond, Xh, tol=tol, maxit=50000, mixed=mixed,
                                    inner_tol=1e-3 if mixed else 0.0, max_outer=80,
                                    core_dtype=binding.QP_BF16 if mixed else binding.QP_F32,
                                    krylov=binding.QP_BICGSTAB)
        stats = pile8.ctx.newton_solve(st, rhs, dx, opts, allow=())
        res = np.linalg.norm(b - S @ pile8.unpad(to_np(dx))) / np.linalg.norm(b)
        assert res <= 1.05 * tol and stats.rel_res <= tol
        if not mixed:
            # residual 1e-12: the solution to 1e-8 per entry (floor 1e-3 max), as for PCG
            exact = sla.cho_solve(sla.cho_factor(S.toarray()), b)
            assert_close(pile8.unpad(to_np(dx)), exact, 1e-8, floor_rel=1e-3, what="BiCGSTAB dgamma")


def test_qtt_breakdown_falls_back_to_jacobi(pile8):
    """An indefinite QTT preconditioner (X = -I) breaks CG down; the solve is redone with Jacobi."""
    g, lam = pile8.iters[3]
    gd, ld, st = pile8.state(g, lam)
    rhs = torch.empty(pile8.P, dtype=torch.float64, device="cuda")
    pile8.ctx.newton_rhs(st, rhs)
    d = pile8.L
    eye = [np.array([1.0, 0.0, 0.0, 1.0]).reshape(1, 4, 1) for _ in range(d)]
    eye[0] = -eye[0]
    Xneg = pile8.ctx.qtt_from_cores(eye)
    dx = torch.empty_like(rhs)
    stats = pile8.ctx.newton_solve(st, rhs, dx, pile8.ctx.solve_opts(binding.QP_QTT_PCG, Xneg, tol=1e-10,
                                                                      maxit=50000), allow=())
    assert stats.fallback == 1 and stats.status == binding.QP_OK and stats.rel_res <= 1e-10
