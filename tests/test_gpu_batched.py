"""GPU parity: many independent Newton systems in one launch (two-block
clusters: a scene on both blocks or one scene per block) against the oracle's
Schur matrices and the single-scene solver."""
import numpy as np
import pytest
import torch

from gpu_common import Problem, assert_close, to_np
from oracle import qp
from paper_1808_02558_gb300 import binding
from synth import Scene, lattice_scene
from test_gpu_newton import interior_point
from test_oracle_qp import sphere_on_plane

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return binding.Context()


def scenes():
    out = [lattice_scene(n, 10 + n, polydisperse=(n % 2 == 1), mu=0.2 + 0.1 * n) for n in (2, 3, 4, 5, 6)]
    out += [lattice_scene(3, 40, mu=0.8), sphere_on_plane((0.3, 0.1, -0.2)),
            Scene(name="free", pos=[[0.0, 0.0, 3.0]], vel=[[0.0, 0.0, 0.0]], omega=[[0.0, 0.0, 0.0]], radius=[0.5])]
    return out


@pytest.mark.parametrize("block,slots,split", [(256, 3, 0), (0, 3, 0), (512, 4, 0), (1024, 3, 1), (256, 4, 2),
                                               (128, 3, 1)])
def test_batched_solves_match_oracle_and_single(ctx, block, slots, split):
    """split 0: the scenes above an even share of the SMs run on two blocks;
    1: one block per scene (scenes paired in clusters); 2: every scene on two
    blocks."""
    pbs, states, rhs, dx, keep = [], [], [], [], []
    sc = scenes()
    if block == 128:  # an odd count leaves the second block of the last cluster idle
        sc = sc[:3]
    for i, s in enumerate(sc):
        pb = Problem(ctx, s, slots=slots)
        g, lam = interior_point(pb, i) if pb.Nc > 0 else (np.zeros(0), np.zeros(0))
        gd, ld, st = pb.state(g, lam) if pb.Nc > 0 else (None, None, None)
        r = torch.empty(pb.P, dtype=torch.float64, device="cuda")
        if st is not None:
            pb.ctx.newton_rhs(st, r)
        else:
            r.zero_()
        pbs.append((pb, g, lam))
        states.append(st)
        rhs.append(r)
        dx.append(torch.full_like(r, 9.0))
        keep.append((gd, ld))
    stats, used = binding.newton_solve_batched([p[0].ctx for p in pbs], states, rhs, dx, tol=1e-10,
                                               block_threads=block, split=split, allow=())
    assert used == block if block else used in (256, 512, 1024)
    for (pb, g, lam), st, r, x, s in zip(pbs, states, rhs, dx, stats):
        assert s.status == binding.QP_OK
        if pb.Nc == 0:
            assert torch.count_nonzero(x).item() == 0 and s.iters == 0
            continue
        S = qp.schur_matrix(pb.N, g, lam, pb.scene.mu)
        b = pb.unpad(to_np(r))
        xs = pb.unpad(to_np(x))
        assert np.linalg.norm(b - S @ xs) <= 1.05e-10 * np.linalg.norm(b)
        assert s.rel_res <= 1e-10
        assert np.array_equal(to_np(x), pb.pad(xs))  # dummy rows stay zero
        one = torch.empty_like(r)
        pb.ctx.newton_solve(st, r, one, pb.ctx.solve_opts(tol=1e-10, maxit=100000, mixed=1, inner_tol=1e-3,
                                                          max_outer=60), allow=())
        # two solves to residual 1e-10 of the same system (different kernels)
        assert_close(xs, pb.unpad(to_np(one)), 1e-6, floor_rel=1e-2, what="batched vs single solve")


def test_batched_without_state_is_plain_N(ctx):
    s = sphere_on_plane((0.3, 0.1, -0.2))
    pb = Problem(ctx, s)
    b = torch.tensor([1.0, -2.0, 0.5, 0.0], dtype=torch.float64, device="cuda")
    x = torch.empty_like(b)
    stats, _ = binding.newton_solve_batched([pb.ctx], [None], [b], [x], tol=1e-12, block_threads=128, allow=())
    m = s.mass[0]
    want = np.array([1.0 * m, -2.0 * m / 3.5, 0.5 * m / 3.5])  # N = diag(1/m, 3.5/m, 3.5/m)
    assert np.allclose(to_np(x)[:3], want, rtol=1e-10, atol=0)
    assert to_np(x)[3] == 0.0


def test_batched_rejects_bad_arguments(ctx):
    pb = Problem(ctx, sphere_on_plane((0.3, 0.1, -0.2)))
    b = torch.ones(pb.P, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.QPError) as e:
        binding.newton_solve_batched([pb.ctx], [None], [b], [b], tol=1e-8, allow=())
    assert e.value.code == binding.QP_INVALID_ARG
    x = torch.empty_like(b)
    with pytest.raises(binding.QPError) as e:
        binding.newton_solve_batched([pb.ctx], [None], [b], [x], tol=1e-8, block_threads=100, allow=())
    assert e.value.code == binding.QP_INVALID_ARG
    with pytest.raises(binding.QPError) as e:
        binding.newton_solve_batched([pb.ctx], [None], [b], [x], tol=1e-8, split=3, allow=())
    assert e.value.code == binding.QP_INVALID_ARG


def test_split_and_unsplit_solves_agree(ctx):
    """The same 20^3 Newton system on one block and on a two-block cluster: both
    reach the tolerance and agree to it (the sums are taken in a different
    order, so not bitwise)."""
    s = lattice_scene(20, 5)
    pb = Problem(ctx, s)
    g, lam = interior_point(pb, 3)
    gd, ld, st = pb.state(g, lam)
    r = torch.empty(pb.P, dtype=torch.float64, device="cuda")
    pb.ctx.newton_rhs(st, r)
    out = {}
    for split in (1, 2):
        x = torch.full_like(r, 9.0)
        stats, _ = binding.newton_solve_batched([pb.ctx], [st], [r], [x], tol=1e-10, block_threads=512,
                                                split=split, allow=())
        assert stats[0].status == binding.QP_OK and stats[0].rel_res <= 1e-10
        out[split] = pb.unpad(to_np(x))
    S = qp.schur_matrix(pb.N, g, lam, pb.scene.mu)
    b = pb.unpad(to_np(r))
    for x in out.values():
        assert np.linalg.norm(b - S @ x) <= 1.05e-10 * np.linalg.norm(b)
    assert_close(out[2], out[1], 1e-6, floor_rel=1e-2, what="split vs unsplit solve")


@pytest.mark.parametrize("tile,cdt,split", [(0, binding.QP_F32, 0), (1, binding.QP_F32, 0), (2, binding.QP_BF16, 0),
                                            (0, binding.QP_BF16, 1)])
def test_batched_qtt_preconditioner(ctx, tile, cdt, split):
    """Scenes with their own QTT inverse of their Jacobi-scaled Schur matrix
    (compressed with the state) next to scenes on Jacobi, in one launch.  The
    scenes of up to 2^6 unknowns get exact inverses (ranks up to 64: every rank
    class of the tile table occurs) and take the iteration count of the
    single-scene QTT-PCG with the same inverse; a 2^9 scene gets a truncated one
    (rank 10), which may break down and then finish with Jacobi, as the
    single-scene solver does.  All: residual 1e-10 against the oracle S.  split
    0 puts these few scenes on two-block clusters, split 1 on one block each."""
    sc = [lattice_scene(2, 12, mu=0.4), sphere_on_plane((0.3, 0.1, -0.2)), lattice_scene(2, 21, mu=0.7),
          lattice_scene(4, 14, mu=0.6), lattice_scene(3, 40, mu=0.8)]
    rank = [64, 64, 64, 10, None]
    pbs, states, rhs, dx, keep, X = [], [], [], [], [], []
    for i, (s, rk) in enumerate(zip(sc, rank)):
        pb = Problem(ctx, s)
        g, lam = interior_point(pb, i)
        gd, ld, st = pb.state(g, lam)
        r = torch.empty(pb.P, dtype=torch.float64, device="cuda")
        pb.ctx.newton_rhs(st, r)
        pbs.append((pb, g, lam))
        states.append(st)
        rhs.append(r)
        dx.append(torch.full_like(r, 9.0))
        keep.append((gd, ld))
        if rk is None:
            X.append(None)
            continue
        eps = 1e-7 if rk == 64 else 1e-2
        S_tt = pb.ctx.qtt_compress(st, eps, rk)
        X.append(pb.ctx.qtt_inverse(S_tt, eps, rk, sweeps=4))
        S_tt.free()
    assert X[0].d == 6 and X[1].d == 2
    stats, used = binding.newton_solve_batched([p[0].ctx for p in pbs], states, rhs, dx, tol=1e-10, maxit=20000,
                                               block_threads=256, split=split, allow=(), precond=X,
                                               core_dtype=cdt, qtt_tile=tile)
    for (pb, g, lam), st, r, x, s, Xi, rk in zip(pbs, states, rhs, dx, stats, X, rank):
        assert s.status == binding.QP_OK
        S = qp.schur_matrix(pb.N, g, lam, pb.scene.mu)
        b = pb.unpad(to_np(r))
        xs = pb.unpad(to_np(x))
        assert np.linalg.norm(b - S @ xs) <= 1.05e-10 * np.linalg.norm(b)
        if rk != 64:
            continue
        assert s.fallback == 0
        one = torch.empty_like(r)
        so = pb.ctx.solve_opts(binding.QP_QTT_PCG, Xi, tol=1e-10, maxit=20000, mixed=1, inner_tol=1e-3,
                               max_outer=60, core_dtype=cdt)
        s1 = pb.ctx.newton_solve(st, r, one, so, allow=())
        assert s1.fallback == 0
        assert abs(s.iters - s1.iters) <= max(3, 0.2 * s1.iters), (s.iters, s1.iters)
        assert_close(xs, pb.unpad(to_np(one)), 1e-6, floor_rel=1e-2, what="batched vs single QTT solve")
    for Xi in X:
        if Xi is not None:
            Xi.free()


def test_batched_qtt_tile_table(ctx):
    for nt in (256, 1024):
        t = ctx.batch_qtt_tiles(nt)
        assert len(t) == 4 and all(v in (1, 2) for v in t[:3]) and t[3] == 1
        assert ctx.batch_qtt_tiles(nt) == t  # measured once, then cached
    with pytest.raises(binding.QPError) as e:
        ctx.batch_qtt_tiles(300)
    assert e.value.code == binding.QP_INVALID_ARG
