"""Oracle: QP data of the relaxed cone complementarity problem and Newton blocks.

Test infrastructure (see the package docstring); plain numpy/scipy, float64.

* Contact Jacobian D in R^{6M x 3Nc} (Sec. 2.2-2.3, Eq. force_balance_disc):
  column u in {n, t1, t2} of contact c is (+u, rho_b x u) on body b and
  (-u, -rho_a x u) on body a; the static floor has no columns.  With this sign
  D_n^T v is the normal separation velocity of Eq. complementarity_disc.
* N = D^T M^-1 D (Eq. Ndef) and r = b + D^T M^-1 k, k = M v + dt f, b_c =
  (Phi_c/dt, 0, 0) (Eq. rdef); the body force is gravity only, so
  M^-1 k = (v + dt g, omega).
* PDIP constraints (Sec. 2.4, "Application to the CCP"):
  f_c = (g1^2 + g2^2 - mu^2 gn^2)/2 and f_{Nc+c} = -gn.
* Schur complement of the Newton system Eq. qp_Newton_system (Sec. 3.3):
  S = N + M_hat - B E^-1 C = N + blockdiag(H_c) with
  H_c = l_c diag(-mu^2, 1, 1) + (l_c/(-f_c)) g g^T + (l'_c/gn) e1 e1^T,
  g = grad f_c = (-mu^2 gn, g1, g2), l'_c the multiplier of -gn <= 0.
  The paper prints the M_hat entry as +mu^2 lambda and asks lambda < 0; with
  lambda = -1/(t f) > 0 and Hess f_c = diag(-mu^2, 1, 1) the consistent entry is
  -mu^2 lambda (the reading used here); S is then symmetric positive definite.
* Padded layout (Sec. 3.3, uniform tree of 2^L leaves with dummy identity rows):
  unknown (c, u) sits at row slots*c + u, slots in {3, 4}; every other row of
  the 2^L x 2^L matrix is an identity row.

Pins: sphere-on-plane closed form N = diag(1/m, 7/(2m), 7/(2m)); symmetry and
block pattern of N equal to the contact edge-adjacency graph (Sec. 3.3); S SPD.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


def padded_size(Nc: int, slots: int = 3) -> tuple[int, int]:
    """(L, P = 2^L): smallest power of two holding slots*Nc rows, at least 2."""
    rows = max(1, slots * Nc)
    L = max(1, int(math.ceil(math.log2(rows))))
    return L, 1 << L


def jacobian(scene, con) -> sp.csr_matrix:
    """D as a sparse 6M x 3Nc matrix (rows: body v(3), omega(3))."""
    M, Nc = scene.M, con.Nc
    rows, cols, vals = [], [], []
    U = np.stack([con.n, con.t1, con.t2], axis=2)  # (Nc, 3, 3): U[c, :, u]
    for side, body, arm, sgn in ((0, con.a, con.ra, -1.0), (1, con.b, con.rb, 1.0)):
        real = body < M
        cs = np.nonzero(real)[0]
        for u in range(3):
            vec = U[cs, :, u]
            tor = np.cross(arm[cs], vec)
            for k in range(3):
                rows.append(6 * body[cs] + k)
                cols.append(3 * cs + u)
                vals.append(sgn * vec[:, k])
                rows.append(6 * body[cs] + 3 + k)
                cols.append(3 * cs + u)
                vals.append(sgn * tor[:, k])
    r = np.concatenate(rows) if rows else np.zeros(0, dtype=np.int64)
    c = np.concatenate(cols) if cols else np.zeros(0, dtype=np.int64)
    v = np.concatenate(vals) if vals else np.zeros(0)
    return sp.csr_matrix((v, (r, c)), shape=(6 * M, 3 * Nc))


def inv_mass_diag(scene) -> np.ndarray:
    return np.repeat(np.stack([scene.inv_mass, scene.inv_inertia], axis=1), 3, axis=1).reshape(-1)


def qp_data(scene, con):
    """(D, N, r) of Eqs. Ndef and rdef, compact 3Nc layout."""
    D = jacobian(scene, con)
    Minv = sp.diags(inv_mass_diag(scene))
    N = (D.T @ Minv @ D).tocsr()
    g = np.asarray(scene.gravity, dtype=np.float64)
    vk = np.concatenate([scene.vel + scene.dt * g, scene.omega], axis=1).reshape(-1)
    b = np.zeros(3 * con.Nc)
    b[0::3] = con.phi / scene.dt
    r = b + D.T @ vk
    return D, N, r


def constraints(gamma: np.ndarray, mu) -> np.ndarray:
    """f(gamma) in R^{2Nc}: cone constraints then non-negativity of gn."""
    gn, g1, g2 = gamma[0::3], gamma[1::3], gamma[2::3]
    mu = np.broadcast_to(np.asarray(mu, dtype=np.float64), gn.shape)
    fc = 0.5 * (g1 * g1 + g2 * g2 - mu * mu * gn * gn)
    return np.concatenate([fc, -gn])


def constraint_grads(gamma: np.ndarray, mu) -> np.ndarray:
    """grad f_c per contact as (Nc, 3); grad f_{Nc+c} = -e1 is implicit."""
    gn, g1, g2 = gamma[0::3], gamma[1::3], gamma[2::3]
    mu = np.broadcast_to(np.asarray(mu, dtype=np.float64), gn.shape)
    return np.stack([-mu * mu * gn, g1, g2], axis=1)


def lagrangian_grad(gamma, lam, mu) -> np.ndarray:
    """sum_i lambda_i grad f_i, compact layout."""
    Nc = gamma.size // 3
    g = constraint_grads(gamma, mu) * lam[:Nc, None]
    g[:, 0] -= lam[Nc:]
    return g.reshape(-1)


def schur_blocks(gamma, lam, mu) -> np.ndarray:
    """Per-contact 3x3 blocks H_c of S - N (Sec. 3.3 Schur complement)."""
    Nc = gamma.size // 3
    f = constraints(gamma, mu)
    g = constraint_grads(gamma, mu)
    mu = np.broadcast_to(np.asarray(mu, dtype=np.float64), (Nc,))
    lc, ln = lam[:Nc], lam[Nc:]
    H = np.zeros((Nc, 3, 3))
    H[:, 0, 0] = -mu * mu * lc
    H[:, 1, 1] = lc
    H[:, 2, 2] = lc
    H += (lc / (-f[:Nc]))[:, None, None] * g[:, :, None] * g[:, None, :]
    H[:, 0, 0] += ln / gamma[0::3]
    return H


def blockdiag(H: np.ndarray) -> sp.csr_matrix:
    return sp.block_diag([sp.coo_matrix(h) for h in H], format="csr") if H.shape[0] else sp.csr_matrix((0, 0))


def schur_matrix(N, gamma, lam, mu) -> sp.csr_matrix:
    """S = N + blockdiag(H) in the compact layout."""
    return (N + blockdiag(schur_blocks(gamma, lam, mu))).tocsr()


def newton_rhs(N, r, gamma, lam, t, mu) -> np.ndarray:
    """rhs of S dgamma = rhs: -(N gamma + r) + (1/t) sum_i grad f_i / f_i."""
    Nc = gamma.size // 3
    f = constraints(gamma, mu)
    g = constraint_grads(gamma, mu)
    rhs = -(N @ gamma + r)
    add = g / f[:Nc, None]
    add[:, 0] += (-1.0) / f[Nc:]
    return rhs + add.reshape(-1) / t


def to_padded(x: np.ndarray, Nc: int, slots: int, P: int) -> np.ndarray:
    """Compact (3Nc,) -> padded (P,) with zeros on dummy rows."""
    out = np.zeros(P, dtype=x.dtype)
    idx = (slots * np.arange(Nc)[:, None] + np.arange(3)[None, :]).reshape(-1)
    out[idx] = x
    return out


def from_padded(y: np.ndarray, Nc: int, slots: int) -> np.ndarray:
    idx = (slots * np.arange(Nc)[:, None] + np.arange(3)[None, :]).reshape(-1)
    return y[idx]


def padded_matrix(A: sp.spmatrix, Nc: int, slots: int, P: int) -> sp.csr_matrix:
    """Embed a compact 3Nc x 3Nc matrix into the 2^L layout; dummy rows = identity."""
    A = sp.coo_matrix(A)
    idx = (slots * np.arange(Nc)[:, None] + np.arange(3)[None, :]).reshape(-1)
    real = np.zeros(P, dtype=bool)
    real[idx] = True
    dummy = np.nonzero(~real)[0]
    rows = np.concatenate([idx[A.row], dummy])
    cols = np.concatenate([idx[A.col], dummy])
    vals = np.concatenate([A.data, np.ones(dummy.size)])
    return sp.csr_matrix((vals, (rows, cols)), shape=(P, P))


def initial_point(Nc: int, mu) -> tuple[np.ndarray, np.ndarray]:
    """Sec. 3.3 cold start: gn = 1, gt = 0; lambda_i = -1/f_i (centred at t = 1)."""
    gamma = np.zeros(3 * Nc)
    gamma[0::3] = 1.0
    f = constraints(gamma, mu)
    return gamma, -1.0 / f
