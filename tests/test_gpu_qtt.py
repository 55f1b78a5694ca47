"""GPU parity: QTT mat-vec against the oracle's core-by-core contraction (Sec. 3.2)."""
import numpy as np
import pytest
import torch

from gpu_common import dev, relerr, to_np
from oracle import contacts as oc, qp, tt
from paper_1808_02558_gb300 import binding
from synth import lattice_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return binding.Context()


def random_cores(d, rmax, seed):
    rng = np.random.default_rng(seed)
    r = [1] + [int(rng.integers(1, rmax + 1)) for _ in range(d - 1)] + [1]
    return [rng.standard_normal((r[k], 4, r[k + 1])) / np.sqrt(2 * r[k + 1]) for k in range(d)]


@pytest.mark.parametrize("d,rmax", [(1, 1), (2, 3), (10, 8), (13, 17)])
def test_apply_random_cores(ctx, d, rmax):
    cores = random_cores(d, rmax, d)
    A = ctx.qtt_from_cores(cores)
    assert A.ranks() == tt.tt_ranks(cores)
    x = np.random.default_rng(1).standard_normal(1 << d)
    want = tt.qtt_matvec(cores, x)
    y = torch.empty(1 << d, dtype=torch.float64, device="cuda")
    ctx.qtt_apply(A, dev(x), y, binding.QP_F64, binding.QP_F64)
    assert relerr(to_np(y), want) <= 1e-13
    x32 = dev(x).float()
    y32 = torch.empty_like(x32)
    ctx.qtt_apply(A, x32, y32, binding.QP_F32, binding.QP_F32)
    assert relerr(to_np(y32).astype(np.float64), want) <= 1e-5 * d
    ctx.qtt_apply(A, x32, y32, binding.QP_BF16, binding.QP_F32)
    assert relerr(to_np(y32).astype(np.float64), want) <= 1e-2 * d
    # cores round trip
    back = A.cores()
    assert all(np.array_equal(a, b) for a, b in zip(back, cores))


def test_apply_compressed_schur_matrix(ctx):
    s = lattice_scene(3, 4)
    con = oc.detect(s)
    _, N, r = qp.qp_data(s, con)
    g, lam = qp.initial_point(con.Nc, s.mu)
    L, P = qp.padded_size(con.Nc, 3)
    S = qp.padded_matrix(qp.schur_matrix(N, g, lam, s.mu), con.Nc, 3, P).toarray()
    cores = tt.qtt_compress_dense(S, 1e-12)
    A = ctx.qtt_from_cores(cores)
    x = np.random.default_rng(2).standard_normal(P)
    y = torch.empty(P, dtype=torch.float64, device="cuda")
    ctx.qtt_apply(A, dev(x), y)
    assert relerr(to_np(y), S @ x) <= 1e-11


def test_apply_full_size_d20(ctx):
    cores = random_cores(20, 10, 20)
    A = ctx.qtt_from_cores(cores)
    x = np.random.default_rng(3).standard_normal(1 << 20)
    want = tt.qtt_matvec(cores, x)
    y = torch.empty(1 << 20, dtype=torch.float64, device="cuda")
    ctx.qtt_apply(A, dev(x), y)
    assert relerr(to_np(y), want) <= 1e-13
