"""Oracle: tensor-train decomposition, rounding and QTT matrix arithmetic.

Test infrastructure (see the package docstring); plain numpy, float64.

* TT format (Sec. 3.1, Eq. TTdeccores): cores G_k of shape (r_{k-1}, n_k, r_k),
  r_0 = r_d = 1.
* TT-SVD (Sec. 3.1, Alg. 1): successive truncated SVDs of the unfolding
  matrices.  Reading of the truncation rule: each step keeps the smallest rank
  r with sqrt(sum_{l>r} sigma_l^2) <= delta, delta = eps ||A||_F / sqrt(d-1)
  (the accuracy target is read relative to ||A||_F), capped at r_max.  The
  `reverse` option runs the same algorithm on the tensor with its modes in
  reverse order (right-to-left sweep) and returns the cores in natural order.
* QTT of a matrix (Sec. 3.2): a 2^d x 2^d matrix A becomes the d-dimensional
  tensor T(b_1, ..., b_d) = A(i, j) with b_k = 2 i_k + j_k and i = sum_k i_k
  2^(d-k) (most significant bit first).  Each core, viewed as G_k(a, i_k, j_k, b),
  is a 2x2 matrix for every pair of rank indices.
* Mat-vec (Sec. 3.2): contract one core at a time; here the plain einsum chain.
* Rounding: right-to-left QR orthogonalisation, then left-to-right truncated
  SVD with the same delta (Oseledets, "Tensor-train decomposition", SIAM J. Sci.
  Comput. 33 (2011), Alg. 2).
* QTT inverse reference: dense inverse followed by TT-SVD (small d only).

Pins: exact ranks of identity (1), shift (2), tridiagonal Toeplitz (<= 3),
sin(x+y+z) on an n^3 grid (2, 2) with storage 8n (Sec. 3.1 example), Kronecker
products; the TT-SVD error bound ||A - A_TT||_F <= eps ||A||_F; mat-vec against
the dense matrix.
"""
from __future__ import annotations

import math

import numpy as np


def trunc_rank(s: np.ndarray, delta: float, rmax: int) -> int:
    """Smallest r with tail norm of s beyond r at most delta; 1 <= r <= rmax."""
    tail2 = np.concatenate([np.cumsum((s[::-1] ** 2))[::-1][1:], [0.0]])
    ok = np.nonzero(np.sqrt(tail2) <= delta)[0]
    r = int(ok[0]) + 1 if ok.size else s.size
    return max(1, min(r, rmax, s.size))


def tt_svd(T: np.ndarray, eps: float, rmax: int = 1 << 30, reverse: bool = False) -> list:
    """Alg. 1 of the paper on a d-dimensional array T."""
    if reverse:
        d = T.ndim
        cores = tt_svd(np.transpose(T, tuple(range(d - 1, -1, -1))), eps, rmax)
        return [np.transpose(G, (2, 1, 0)) for G in cores[::-1]]
    dims = T.shape
    d = len(dims)
    nrm = float(np.linalg.norm(T))
    delta = eps * nrm / math.sqrt(max(d - 1, 1))
    cores = []
    r_prev = 1
    Mk = T.reshape(dims[0], -1)
    for k in range(d - 1):
        U, s, Vt = np.linalg.svd(Mk, full_matrices=False)
        rk = trunc_rank(s, delta, rmax)
        cores.append(U[:, :rk].reshape(r_prev, dims[k], rk))
        V = s[:rk, None] * Vt[:rk]
        r_prev = rk
        Mk = V.reshape(rk * dims[k + 1], -1)
    cores.append(Mk.reshape(r_prev, dims[-1], 1))
    return cores


def tt_full(cores: list) -> np.ndarray:
    """Contract a TT back into the full tensor."""
    out = cores[0]
    for G in cores[1:]:
        out = np.tensordot(out, G, axes=([out.ndim - 1], [0]))
    return out.reshape(out.shape[1:-1])


def tt_ranks(cores: list) -> list:
    return [1] + [G.shape[2] for G in cores]


def qtt_tensorize(A: np.ndarray) -> np.ndarray:
    """2^d x 2^d matrix -> (4,)*d tensor with b_k = 2 i_k + j_k, MSB first."""
    n = A.shape[0]
    d = int(round(math.log2(n)))
    assert (1 << d) == n and A.shape == (n, n)
    T = A.reshape((2,) * (2 * d))
    perm = [x for k in range(d) for x in (k, d + k)]
    return np.transpose(T, perm).reshape((4,) * d)


def qtt_matrix(cores: list) -> np.ndarray:
    """Dense 2^d x 2^d matrix of a QTT (inverse of qtt_tensorize)."""
    d = len(cores)
    T = tt_full(cores).reshape((2,) * (2 * d))
    perm = [2 * k for k in range(d)] + [2 * k + 1 for k in range(d)]
    return np.transpose(T, perm).reshape(1 << d, 1 << d)


def qtt_compress_dense(A: np.ndarray, eps: float, rmax: int = 1 << 30, reverse: bool = False) -> list:
    return tt_svd(qtt_tensorize(A), eps, rmax, reverse)


def qtt_matvec(cores: list, x: np.ndarray) -> np.ndarray:
    """y = A_TT x, contracting one core (a 2x2 matrix per rank pair) at a time."""
    d = len(cores)
    # Z holds indices (a, i_1..i_{k}, j_{k+1}..j_d) as (r, 2^k, 2^(d-k)).
    Z = x.reshape(1, 1, 1 << d)
    for k, G in enumerate(cores):
        r0, _, r1 = G.shape
        G4 = G.reshape(r0, 2, 2, r1)                          # (a, i, j, b)
        rest = Z.shape[2] // 2
        Zk = Z.reshape(r0, Z.shape[1], 2, rest)               # (a, I, j, J)
        Z = np.einsum("aijb,aIjJ->bIiJ", G4, Zk).reshape(r1, Z.shape[1] * 2, rest)
    return Z.reshape(-1)


def qtt_matvec_kron_entries(cores: list, v: np.ndarray, rows) -> np.ndarray:
    """Entries y[rows] of y = A_TT x for the Kronecker-product vector
    x = v_1 (x) v_2 (x) ... (x) v_d (v of shape (d, 2), v_1 on the most
    significant bit).  The QTT matrix acts mode by mode (Sec. 3.2), so for such
    an x the column bits separate and y(i) = prod_k M_k(i_k), a product of the
    r_{k-1} x r_k matrices M_k(i_k)[a, b] = sum_j G_k(a, i_k, j, b) v_k[j]:
    O(d r^2) work per entry, at any d."""
    d = len(cores)
    Ms = [np.einsum("aijb,j->iab", G.reshape(G.shape[0], 2, 2, G.shape[2]), np.asarray(v[k], dtype=np.float64))
          for k, G in enumerate(cores)]
    out = np.empty(len(rows))
    for n, i in enumerate(rows):
        acc = np.ones((1, 1))
        for k in range(d):
            acc = acc @ Ms[k][(int(i) >> (d - 1 - k)) & 1]
        out[n] = acc[0, 0]
    return out


def tt_add(A: list, B: list) -> list:
    """A + B as a TT of ranks r_A + r_B (block cores)."""
    d = len(A)
    out = []
    for k in range(d):
        Ga, Gb = A[k], B[k]
        if d == 1:
            out.append(Ga + Gb)
        elif k == 0:
            out.append(np.concatenate([Ga, Gb], axis=2))
        elif k == d - 1:
            out.append(np.concatenate([Ga, Gb], axis=0))
        else:
            G = np.zeros((Ga.shape[0] + Gb.shape[0], Ga.shape[1], Ga.shape[2] + Gb.shape[2]))
            G[:Ga.shape[0], :, :Ga.shape[2]] = Ga
            G[Ga.shape[0]:, :, Ga.shape[2]:] = Gb
            out.append(G)
    return out


def tt_scale(A: list, alpha: float) -> list:
    out = [G.copy() for G in A]
    out[0] = out[0] * alpha
    return out


def qtt_transpose(A: list) -> list:
    """Transpose of a QTT matrix: swap i_k and j_k in every core."""
    return [G.reshape(G.shape[0], 2, 2, G.shape[2]).transpose(0, 2, 1, 3).reshape(G.shape) for G in A]


def tt_norm(A: list) -> float:
    return float(np.linalg.norm(tt_full(A)))


def tt_round(A: list, eps: float, rmax: int = 1 << 30) -> list:
    """QR right-to-left, then truncated SVD left-to-right (Oseledets 2011)."""
    cores = [G.copy() for G in A]
    d = len(cores)
    for k in range(d - 1, 0, -1):
        r0, n, r1 = cores[k].shape
        Q, R = np.linalg.qr(cores[k].reshape(r0, n * r1).T)
        cores[k] = Q.T.reshape(-1, n, r1)
        cores[k - 1] = np.tensordot(cores[k - 1], R.T, axes=([2], [0]))
    nrm = float(np.linalg.norm(cores[0]))
    delta = eps * nrm / math.sqrt(max(d - 1, 1))
    for k in range(d - 1):
        r0, n, r1 = cores[k].shape
        U, s, Vt = np.linalg.svd(cores[k].reshape(r0 * n, r1), full_matrices=False)
        rk = trunc_rank(s, delta, rmax)
        cores[k] = U[:, :rk].reshape(r0, n, rk)
        cores[k + 1] = np.tensordot(s[:rk, None] * Vt[:rk], cores[k + 1], axes=([1], [0]))
    return cores


def qtt_inverse_dense(A: np.ndarray, eps: float, rmax: int = 1 << 30) -> list:
    """Reference approximate inverse: exact inverse, then TT-SVD at eps."""
    return qtt_compress_dense(np.linalg.inv(A), eps, rmax)
