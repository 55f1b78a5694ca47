"""Oracle pins for TT-SVD, rounding and QTT arithmetic (Sec. 3.1-3.2).

Exact ranks of matrices whose QTT structure is known in closed form, the
worked sin(x+y+z) example of Sec. 3.1, the TT-SVD error bound, and dense
reconstruction of the mat-vec.
"""
import os

import numpy as np
import pytest

from oracle import tt


def qtt_ranks(A, eps=1e-12, reverse=False):
    return tt.tt_ranks(tt.qtt_compress_dense(A, eps, reverse=reverse))


@pytest.mark.parametrize("reverse", [False, True])
def test_exact_ranks_of_structured_matrices(reverse):
    d = 7
    n = 1 << d
    assert qtt_ranks(np.eye(n), reverse=reverse) == [1] * (d + 1)
    assert max(qtt_ranks(np.eye(n, k=1), reverse=reverse)) == 2
    T = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    assert max(qtt_ranks(T, reverse=reverse)) <= 3
    # I_{2^(d-m)} (x) B: the first d-m cores are rank 1
    m = 3
    B = np.random.default_rng(0).standard_normal((1 << m, 1 << m))
    r = qtt_ranks(np.kron(np.eye(1 << (d - m)), B), reverse=reverse)
    assert r[: d - m + 1] == [1] * (d - m + 1)


def test_identity_padding_adds_at_most_one_rank():
    d = 6
    n = 1 << d
    T = 2 * np.eye(n // 2) - np.eye(n // 2, k=1) - np.eye(n // 2, k=-1)
    A = np.zeros((n, n))
    A[: n // 2, : n // 2] = T
    A[n // 2:, n // 2:] = np.eye(n // 2)
    Tfull = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    base = qtt_ranks(Tfull)
    padded = qtt_ranks(A)
    assert all(p <= b + 1 for p, b in zip(padded, base))


def golden(name):
    """key -> list of ints from a fixture under tests/golden (comments start with #)."""
    out = {}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)) as f:
        for line in f:
            line = line.split("#")[0].split()
            if line:
                out[line[0]] = [int(v) for v in line[1:]]
    return out


@pytest.mark.parametrize("n", [5, 17])
def test_sine_cube_example(n):
    # Sec. 3.1 worked example: ranks and storage as the paper prints them
    g = golden("sine_cube_sec3_1.txt")
    x = np.linspace(0, 1, n)
    A = np.sin(x[:, None, None] + x[None, :, None] + x[None, None, :])
    cores = tt.tt_svd(A, 1e-12)
    assert tt.tt_ranks(cores) == g["tt_ranks"]
    assert sum(G.size for G in cores) == g["storage_per_n"][0] * n
    assert np.abs(tt.tt_full(cores) - A).max() < 1e-13


def test_sine_vector_qtt_rank_two():
    d = 10
    i = np.arange(1 << d)
    v = np.sin(0.37 * i + 0.2).reshape((2,) * d)
    assert max(tt.tt_ranks(tt.tt_svd(v, 1e-12))) == 2


@pytest.mark.parametrize("eps", [1e-1, 1e-2, 1e-3])
@pytest.mark.parametrize("reverse", [False, True])
def test_ttsvd_error_bound(eps, reverse):
    rng = np.random.default_rng(11)
    d = 8
    n = 1 << d
    U = rng.standard_normal((n, 5))
    A = U @ rng.standard_normal((5, n)) + 0.05 * rng.standard_normal((n, n))
    cores = tt.qtt_compress_dense(A, eps, reverse=reverse)
    err = np.linalg.norm(tt.qtt_matrix(cores) - A) / np.linalg.norm(A)
    assert err <= eps * (1 + 1e-10)


def test_qtt_roundtrip_and_matvec():
    rng = np.random.default_rng(2)
    d = 7
    A = rng.standard_normal((1 << d, 1 << d))
    cores = tt.qtt_compress_dense(A, 1e-14)
    assert np.allclose(tt.qtt_matrix(cores), A, atol=1e-12)
    x = rng.standard_normal(1 << d)
    assert np.allclose(tt.qtt_matvec(cores, x), A @ x, rtol=0, atol=1e-12 * np.abs(A @ x).max())
    At = tt.qtt_transpose(cores)
    assert np.allclose(tt.qtt_matrix(At), A.T, atol=1e-12)


def test_qtt_index_map_msb_first():
    # entry (i, j) lands at b_k = 2 i_k + j_k with i_1 the most significant bit
    d = 3
    A = np.zeros((8, 8))
    A[5, 3] = 1.0                      # i = 101, j = 011
    T = tt.qtt_tensorize(A)
    assert T[2 * 1 + 0, 2 * 0 + 1, 2 * 1 + 1] == 1.0 and T.sum() == 1.0


def test_rounding_recovers_ranks_and_bound():
    rng = np.random.default_rng(5)
    d = 8
    A = rng.standard_normal((1 << d, 1 << d))
    A = A @ A.T
    cores = tt.qtt_compress_dense(A, 1e-3)
    dbl = tt.tt_add(cores, cores)
    assert tt.tt_ranks(dbl)[1:-1] == [2 * r for r in tt.tt_ranks(cores)[1:-1]]
    rnd = tt.tt_round(dbl, 1e-12)
    assert tt.tt_ranks(rnd) == tt.tt_ranks(cores)
    assert np.allclose(tt.qtt_matrix(rnd), 2 * tt.qtt_matrix(cores), atol=1e-9 * np.abs(A).max())
    for eps in (1e-2, 1e-1):
        r2 = tt.tt_round(dbl, eps)
        full = 2 * tt.qtt_matrix(cores)
        assert np.linalg.norm(tt.qtt_matrix(r2) - full) <= eps * np.linalg.norm(full) * (1 + 1e-10)


def test_inverse_reference_on_spd_matrix():
    d = 6
    n = 1 << d
    T = 2.5 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    X = tt.qtt_inverse_dense(T, 1e-10)
    assert np.allclose(tt.qtt_matrix(X) @ T, np.eye(n), atol=1e-8)


def test_kron_entries_match_the_matvec():
    """Entries of A_TT (v_1 x ... x v_d) from the per-mode factorisation equal
    the full one-core-at-a-time contraction (itself pinned against A @ x)."""
    rng = np.random.default_rng(7)
    d = 7
    ranks = [1, 3, 5, 6, 4, 5, 2, 1]
    cores = [rng.standard_normal((ranks[k], 4, ranks[k + 1])) for k in range(d)]
    v = rng.standard_normal((d, 2))
    x = v[0]
    for k in range(1, d):
        x = np.kron(x, v[k])
    want = tt.qtt_matvec(cores, x)
    rows = np.arange(1 << d)
    got = tt.qtt_matvec_kron_entries(cores, v, rows)
    assert np.allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())
    # a transposed core (i and j swapped) changes the result
    bad = [c.reshape(c.shape[0], 2, 2, c.shape[2]).transpose(0, 2, 1, 3).reshape(c.shape) for c in cores]
    assert not np.allclose(tt.qtt_matvec_kron_entries(bad, v, rows), want, rtol=0, atol=1e-6 * np.abs(want).max())
