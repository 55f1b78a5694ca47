"""GPU parity: QTT mat-vec, rounding, compression and inverse against the oracle (Sec. 3.1-3.3).

Mat-vecs and reconstructions are compared entry by entry, |got - want| <=
rtol max(|want|, floor), with floors stated per check (a fraction of the
largest entry).  Inverse quality is a Frobenius-norm approximation error, the
quantity the TT format controls, and is compared as such."""
import numpy as np
import pytest
import torch

from gpu_common import assert_close, dev, relerr, to_np
from oracle import contacts as oc, qp, tt
from paper_1808_02558_gb300 import binding
from synth import lattice_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return binding.Context()


def bf16_round(x):
    """Round to bfloat16 (nearest, ties to even) through float32, as float64."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(x))


def random_cores(d, rmax, seed):
    rng = np.random.default_rng(seed)
    r = [1] + [int(rng.integers(1, rmax + 1)) for _ in range(d - 1)] + [1]
    return [rng.standard_normal((r[k], 4, r[k + 1])) / np.sqrt(2 * r[k + 1]) for k in range(d)]


# ranks <= 12 take the two-cores-per-pass kernel in FP32/BF16, larger ranks (and
# FP64) the one-core kernel; (13, 17) and (15, 14) mix both within one apply
@pytest.mark.parametrize("d,rmax", [(1, 1), (2, 3), (3, 12), (10, 8), (13, 17), (15, 14)])
def test_apply_random_cores(ctx, d, rmax):
    cores = random_cores(d, rmax, d)
    A = ctx.qtt_from_cores(cores)
    assert A.ranks() == tt.tt_ranks(cores)
    x = np.random.default_rng(1).standard_normal(1 << d)
    want = tt.qtt_matvec(cores, x)
    y = torch.empty(1 << d, dtype=torch.float64, device="cuda")
    ctx.qtt_apply(A, dev(x), y, binding.QP_F64, binding.QP_F64)
    assert_close(to_np(y), want, 1e-11, floor_rel=1e-3, what="FP64 apply")
    x32 = dev(x).float()
    y32 = torch.empty_like(x32)
    ctx.qtt_apply(A, x32, y32, binding.QP_F32, binding.QP_F32)
    # the oracle contracts the same float32 input; FP32 chain error ~1e-5..3e-5 on this scale
    want32 = tt.qtt_matvec(cores, to_np(x32).astype(np.float64))
    assert_close(to_np(y32), want32, 2e-4, floor_rel=1e-2, what="FP32 apply")
    ctx.qtt_apply(A, x32, y32, binding.QP_BF16, binding.QP_F32)
    # BF16 cores: the oracle contracts the same bf16-rounded cores in FP64
    wantb = tt.qtt_matvec([bf16_round(c) for c in cores], to_np(x32).astype(np.float64))
    assert_close(to_np(y32), wantb, 2e-4, floor_rel=1e-2, what="BF16-core apply")
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
    # ||S - S_TT||_F <= 1e-12 ||S||_F, so each entry of (S - S_TT) x is below 1e-12 ||S||_F ||x||
    assert_close(to_np(y), S @ x, 1e-9, floor=1e-3 * np.linalg.norm(S) * np.linalg.norm(x), what="S_TT x")


def test_apply_full_size_d20(ctx):
    cores = random_cores(20, 10, 20)
    A = ctx.qtt_from_cores(cores)
    x = np.random.default_rng(3).standard_normal(1 << 20)
    want = tt.qtt_matvec(cores, x)
    y = torch.empty(1 << 20, dtype=torch.float64, device="cuda")
    ctx.qtt_apply(A, dev(x), y)
    assert_close(to_np(y), want, 1e-11, floor_rel=1e-3, what="FP64 apply, d = 20")
    x32 = dev(x).float()
    y32 = torch.empty_like(x32)
    ctx.qtt_apply(A, x32, y32, binding.QP_F32, binding.QP_F32)
    want32 = tt.qtt_matvec(cores, to_np(x32).astype(np.float64))
    assert_close(to_np(y32), want32, 5e-4, floor_rel=1e-2, what="FP32 apply, d = 20")


# ---------------------------------------------------------------- tensor-core steps
def capped_cores(d, r, seed):
    """Ranks min(r, 4^k, 4^(d-k)): the profile of a compressed Schur matrix's
    inverse at rank cap r."""
    rng = np.random.default_rng(seed)
    ranks = [min(r, 4 ** min(k, d - k)) for k in range(d + 1)]
    return [rng.standard_normal((ranks[k], 4, ranks[k + 1])) / np.sqrt(2 * ranks[k + 1]) for k in range(d)]


# rank caps that pad K (2 r_k not a multiple of 32) and M (2 r_{k-1} < 128);
# d = 8 has cores whose column items span several J' per tile (2^(d-k) < 32)
@pytest.mark.parametrize("d,r", [(8, 64), (10, 33), (12, 64), (14, 40)])
def test_apply_tensor_core_steps(d, r):
    c = binding.Context()
    cores = capped_cores(d, r, 100 + d)
    A = c.qtt_from_cores(cores)
    x32 = dev(np.random.default_rng(d).standard_normal(1 << d)).float()
    xin = to_np(x32).astype(np.float64)
    want = {binding.QP_F32: tt.qtt_matvec(cores, xin),
            binding.QP_BF16: tt.qtt_matvec([bf16_round(g) for g in cores], xin)}
    for cdt, name in ((binding.QP_BF16, "BF16"), (binding.QP_F32, "F32")):
        got = {}
        for mode in (0, 1, 2):
            c.qtt_set_tensor_cores(mode)
            y = torch.full_like(x32, float("nan"))
            c.qtt_apply(A, x32, y, cdt, binding.QP_F32)
            got[mode] = to_np(y).astype(np.float64)
            assert_close(got[mode], want[cdt], 2e-4, floor_rel=1e-2, what=f"{name} cores, tensor-core mode {mode}")
        # the split-TF32 products stay near FP32 accuracy: the largest error
        # relative to the largest entry is ~3e-6 (BF16 cores) to ~1.2e-5 (F32
        # cores) on the tensor cores, whose accumulator rounds more coarsely
        # than an FMA chain, against ~4e-7 on the CUDA cores: far below TF32's
        # 2^-11 ~ 5e-4 and the BF16 cores' 2^-9
        scale = np.abs(want[cdt]).max()
        e = {m: np.abs(got[m] - want[cdt]).max() / scale for m in got}
        assert e[0] <= 2e-6 and max(e.values()) <= 4e-5, (name, e)
    with pytest.raises(binding.QPError) as e:
        c.qtt_set_tensor_cores(3)
    assert e.value.code == binding.QP_INVALID_ARG
    A.free()
    c.close()


def test_apply_tensor_core_full_size_d20():
    """d = 20 (2^20 unknowns) at rank cap 64, BF16 cores, a Kronecker-product x:
    4096 sampled entries against the oracle's per-entry product."""
    c = binding.Context()
    d = 20
    cores = [bf16_round(g) for g in capped_cores(d, 64, 7)]
    A = c.qtt_from_cores(cores)
    rng = np.random.default_rng(8)
    v = rng.standard_normal((d, 2))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    x = v[0]
    for k in range(1, d):
        x = np.kron(x, v[k])
    x32 = dev(x).float()
    rows = np.sort(rng.choice(1 << d, 4096, replace=False))
    want = tt.qtt_matvec_kron_entries(cores, v, rows)
    for mode in (1, 0):
        c.qtt_set_tensor_cores(mode)
        y = torch.full_like(x32, float("nan"))
        c.qtt_apply(A, x32, y, binding.QP_BF16, binding.QP_F32)
        yn = to_np(y)
        assert np.isfinite(yn).all()
        assert_close(yn[rows].astype(np.float64), want, 5e-4, floor_rel=1e-2, what=f"d = 20, rank 64, mode {mode}")
    A.free()
    c.close()


# ---------------------------------------------------------------- rounding (Sec. 3.1)
def test_round_sum_recovers_ranks(ctx):
    rng = np.random.default_rng(7)
    d = 9
    A = rng.standard_normal((1 << d, 1 << d))
    A = A @ A.T
    cores = tt.qtt_compress_dense(A, 1e-3)
    dbl = tt.tt_add(cores, cores)
    G = ctx.qtt_from_cores(dbl)
    # below eps = 1e-7 the SVDs are one-sided Jacobi on the cores (no Gram
    # matrix): the redundant half of the doubled ranks sits at FP64 rounding and
    # is removed even at eps = 1e-12; at eps = 1e-6 the Gram route does it
    want = 2 * tt.qtt_matrix(cores)
    for eps in (1e-12, 1e-6):
        R = ctx.qtt_round(G, eps)
        assert R.ranks() == tt.tt_ranks(cores), (eps, R.ranks(), tt.tt_ranks(cores))
        assert_close(tt.qtt_matrix(R.cores()), want, 1e-9 if eps < 1e-7 else 1e-5, floor_rel=1e-2,
                     what=f"round(A + A), eps {eps}")


@pytest.mark.parametrize("eps,rmax", [(1e-1, 1000), (1e-2, 1000), (1e-2, 6), (1e-6, 1000), (1e-10, 1000),
                                      (1e-12, 7)])
def test_round_matches_oracle(ctx, eps, rmax):
    rng = np.random.default_rng(11)
    d = 8
    cores = random_cores(d, 9, 3)
    # a sum with redundant directions exercises rank-deficient orthogonalisation
    big = tt.tt_add(cores, tt.tt_scale(random_cores(d, 5, 4), 0.3))
    want = tt.tt_round(big, eps, rmax)
    R = ctx.qtt_round(ctx.qtt_from_cores(big), eps, rmax)
    assert R.ranks() == tt.tt_ranks(want)
    full = tt.qtt_matrix(big)
    got = tt.qtt_matrix(R.cores())
    assert_close(got, tt.qtt_matrix(want), 1e-7, floor_rel=1e-2, what="rounded reconstruction")
    if rmax >= 1000:
        assert np.linalg.norm(got - full) <= eps * np.linalg.norm(full) * (1 + 1e-9)


# ---------------------------------------------------------------- compression (Alg. 1)
def schur_dense(s, slots=3, k_iter=0):
    con = oc.detect(s)
    _, N, r = qp.qp_data(s, con)
    g, lam = qp.initial_point(con.Nc, s.mu)
    L, P = qp.padded_size(con.Nc, slots)
    S = qp.padded_matrix(qp.schur_matrix(N, g, lam, s.mu), con.Nc, slots, P).toarray()
    Nd = qp.padded_matrix(N, con.Nc, slots, P).toarray()
    return con, g, lam, S, Nd, P


@pytest.mark.parametrize("slots", [3, 4])
@pytest.mark.parametrize("eps", [1e-2, 1e-4, 1e-6])
def test_compress_matches_oracle_ttsvd(eps, slots):
    s = lattice_scene(3, 4, polydisperse=True)
    con, g, lam, S, Nd, P = schur_dense(s, slots)
    ctx = binding.Context()
    from paper_1808_02558_gb300 import workload

    workload.assemble(ctx, s, slots)
    gd = dev(qp.to_padded(g, con.Nc, slots, P))
    ld = dev(lam)
    st = ctx.state(gd, ld)
    for A_dense, state in ((S, st), (Nd, None)):
        want = tt.qtt_compress_dense(A_dense, eps, 100, reverse=True)
        X = ctx.qtt_compress(state, eps, 100)
        got = tt.qtt_matrix(X.cores())
        assert X.ranks() == tt.tt_ranks(want)
        assert_close(got, tt.qtt_matrix(want), 1e-7, floor_rel=1e-2, what="compressed reconstruction")
        if max(X.ranks()) < 100:
            assert np.linalg.norm(got - A_dense) <= eps * np.linalg.norm(A_dense) * (1 + 1e-9)


def test_compress_rank_cap_and_probe_full_size():
    from paper_1808_02558_gb300 import workload
    from synth import random_vector, scene_for

    s = scene_for("pile20", 1)
    ctx = binding.Context()
    _, con = workload.assemble(ctx, s)
    o = oc.detect(s)
    _, N, _ = qp.qp_data(s, o)
    g, lam = qp.initial_point(o.Nc, s.mu)
    L, P = qp.padded_size(o.Nc, 3)
    st = ctx.state(dev(qp.to_padded(g, o.Nc, 3, P)), dev(lam))
    X = ctx.qtt_compress(st, 1e-2, 10)
    assert max(X.ranks()) <= 10 and X.d == 17
    # probe ||(S - S_TT) z|| / ||S z|| with the oracle's S and the library's QTT apply
    S = qp.padded_matrix(qp.schur_matrix(N, g, lam, s.mu), o.Nc, 3, P)
    z = random_vector(3, 2, P)
    y = torch.empty(P, dtype=torch.float64, device="cuda")
    ctx.qtt_apply(X, dev(z), y)
    err = np.linalg.norm(to_np(y) - S @ z) / np.linalg.norm(S @ z)
    assert err < 0.5, err


# ---------------------------------------------------------------- inverse (Sec. 3.2, 3.3)
def test_inverse_tridiagonal_toeplitz(ctx):
    d = 8
    n = 1 << d
    T = 2.5 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    S = ctx.qtt_from_cores(tt.qtt_compress_dense(T, 1e-14))
    X = ctx.qtt_inverse(S, 1e-6, 40, sweeps=4)
    Xd = tt.qtt_matrix(X.cores())
    Tinv = np.linalg.inv(T)
    assert relerr(Xd, Tinv) <= 1e-4
    # symmetrised then rounded: symmetric up to the rounding accuracy
    assert np.linalg.norm(Xd - Xd.T) <= 1e-5 * np.linalg.norm(Xd)
    # warm start from the previous inverse of a perturbed matrix (Sec. 3.3 inverse update)
    T2 = T + 0.05 * np.diag(np.cos(np.arange(n)))
    S2 = ctx.qtt_from_cores(tt.qtt_compress_dense(T2, 1e-14))
    X2 = ctx.qtt_inverse(S2, 1e-6, 40, sweeps=2, warm=X)
    assert relerr(tt.qtt_matrix(X2.cores()), np.linalg.inv(T2)) <= 1e-3


@pytest.mark.parametrize("eps", [1e-2, 1e-3])
def test_inverse_of_compressed_schur_matrix(eps):
    from paper_1808_02558_gb300 import workload

    s = lattice_scene(3, 4, polydisperse=True)
    con, g, lam, Sd, Nd, P = schur_dense(s, 3)
    ctx = binding.Context()
    workload.assemble(ctx, s, 3)
    st = ctx.state(dev(qp.to_padded(g, con.Nc, 3, P)), dev(lam))
    STT = ctx.qtt_compress(st, 1e-10, 128)
    X = ctx.qtt_inverse(STT, eps, 64, sweeps=4)
    Xd = tt.qtt_matrix(X.cores())
    Sinv = np.linalg.inv(Sd)
    # this 2^8 matrix is barely compressible: compare with the TT-SVD of the exact
    # inverse under the same rank cap (the best the format allows)
    ref = tt.qtt_matrix(tt.qtt_inverse_dense(Sd, eps, 64))
    err = relerr(Xd, Sinv)
    best = relerr(ref, Sinv)
    # two-site sweeps truncate every split at eps locally; at eps = 1e-2 the sweep
    # result sits within a small factor of the best approximation
    assert err <= 4 * max(best, eps), (err, best)


# ---------------------------------------------------------------- d = 12 (4096 x 4096)
@pytest.fixture(scope="module")
def d12():
    """Schur matrix of a 7^3 polydisperse lattice (937 contacts, 2^12 padded) at
    the cold start, with the library context holding the same scene."""
    from paper_1808_02558_gb300 import workload

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = lattice_scene(7, 4, polydisperse=True)
    con, g, lam, S, Nd, P = schur_dense(s, 3)
    assert P == 1 << 12
    ctx = binding.Context()
    workload.assemble(ctx, s, 3)
    st = ctx.state(dev(qp.to_padded(g, con.Nc, 3, P)), dev(lam))
    return ctx, st, S


@pytest.mark.parametrize("eps,rmax", [(1e-2, 64), (1e-4, 128)])
def test_compress_d12_matches_oracle_ttsvd(d12, eps, rmax):
    """Alg. 1 (right-to-left) at d = 12: ranks equal to the oracle's TT-SVD of the
    dense matrix, reconstruction error equal to the oracle's, and the two
    reconstructions equal entry by entry (floor 1e-2 max|S|).  128 is the
    largest rank qtt_compress keeps."""
    ctx, st, S = d12
    want = tt.qtt_compress_dense(S, eps, rmax, reverse=True)
    X = ctx.qtt_compress(st, eps, rmax)
    assert X.ranks() == tt.tt_ranks(want)
    got = tt.qtt_matrix(X.cores())
    ref = tt.qtt_matrix(want)
    e_got = np.linalg.norm(got - S) / np.linalg.norm(S)
    e_ref = np.linalg.norm(ref - S) / np.linalg.norm(S)
    assert abs(e_got - e_ref) <= 1e-6 * max(e_ref, 1e-12) + 1e-12, (e_got, e_ref)
    assert_close(got, ref, 1e-6, floor_rel=1e-2, what=f"d = 12 reconstruction at eps {eps}")
    X.free()


def test_inverse_d12_against_dense_inverse(d12):
    """Two-site inverse (Sec. 3.2) of S_TT at d = 12 against the exact inverse:
    within a small factor of the best rank-64 approximation (TT-SVD of the dense
    inverse at the same eps and cap), and a working preconditioner: the spectrum
    of X S is clustered enough that ||I - X S||_2 < 1 on random probes."""
    ctx, st, S = d12
    STT = ctx.qtt_compress(st, 1e-4, 128)
    X = ctx.qtt_inverse(STT, 1e-2, 64, sweeps=4)
    Xd = tt.qtt_matrix(X.cores())
    Sinv = np.linalg.inv(S)
    best = relerr(tt.qtt_matrix(tt.qtt_inverse_dense(S, 1e-2, 64)), Sinv)
    err = relerr(Xd, Sinv)
    assert err <= 4 * max(best, 1e-2), (err, best)
    z = np.random.default_rng(5).standard_normal((S.shape[0], 4))
    assert np.linalg.norm(z - Xd @ (S @ z)) < np.linalg.norm(z)
    X.free()
    STT.free()
