"""Oracle: primal-dual interior point iteration for the CCP quadratic program.

Test infrastructure (see the package docstring); plain numpy/scipy, float64.

The paper (Sec. 2.4) gives the perturbed KKT residual r_t, the Newton system and
"a backtracking line search, and a strategy to increase t".  The steps below are
the standard primal-dual interior point method for inequality-constrained convex
problems (Boyd and Vandenberghe, Convex Optimization, Sec. 11.7), in the paper's
notation, with these readings:

  * surrogate gap eta = -f^T lambda, t = nu * m / eta, m = 2Nc, nu = 10;
  * Newton step from the Schur complement S dgamma = rhs (Sec. 3.3), then
    dlambda_i = -lambda_i - 1/(t f_i) - (lambda_i/f_i) grad f_i^T dgamma;
  * step s = 0.99 min(1, min_{dlambda_i<0} -lambda_i/dlambda_i), halved
    (beta = 0.5) until f(gamma + s dgamma) < 0, then halved until
    ||r_t(gamma+, lambda+)|| <= (1 - alpha s) ||r_t(gamma, lambda)||, alpha = 0.01;
  * stop when eta <= tol_gap and ||r_dual||_2 <= tol_dual (both 1e-8);
  * cold start gamma_n = 1, gamma_t = 0, lambda = -1/f (Sec. 3.3).

Pins: closed-form stick/slip/separation of one sphere on a frictional plane;
KKT conditions (cone, dual cone, complementarity) against a brute-force
projected-gradient solve on 2-4 contacts.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import qp
from .krylov import jacobi_pcg

NU = 10.0
ALPHA = 0.01
BETA = 0.5
STEP_FRACTION = 0.99
MAX_HALVINGS = 60


@dataclass
class PDIPState:
    gamma: np.ndarray
    lam: np.ndarray


@dataclass
class StepInfo:
    eta: float
    t: float
    r_dual_norm: float
    r_t_norm: float
    s: float
    dgamma: np.ndarray
    dlam: np.ndarray
    krylov_iters: int = 0
    halvings: int = 0


def residuals(N, r, gamma, lam, t, mu):
    """(r_dual, r_cent) of Sec. 2.4 at (gamma, lambda) for barrier parameter t."""
    f = qp.constraints(gamma, mu)
    r_dual = N @ gamma + r + qp.lagrangian_grad(gamma, lam, mu)
    r_cent = -lam * f - 1.0 / t
    return r_dual, r_cent


def solve_newton(S: sp.spmatrix, rhs: np.ndarray, method: str = "auto", tol: float = 1e-14):
    """Solve S x = rhs: dense Cholesky when small, else sparse LU / Jacobi-PCG."""
    n = rhs.size
    if n == 0:
        return rhs.copy(), 0
    if method == "auto":
        method = "cholesky" if n <= 6000 else "splu"
    if method == "cholesky":
        c = sla.cho_factor(S.toarray(), lower=True)
        return sla.cho_solve(c, rhs), 0
    if method == "splu":
        import scipy.sparse.linalg as spla
        return spla.splu(sp.csc_matrix(S)).solve(rhs), 0
    x, info = jacobi_pcg(S, rhs, tol=tol, maxit=100000)
    return x, info["iters"]


def pdip_step(N, r, mu, gamma, lam, method="auto", newton_solver=None) -> tuple[np.ndarray, np.ndarray, StepInfo]:
    """One PDIP iteration from (gamma, lambda); returns the new iterate and info."""
    Nc = gamma.size // 3
    m = 2 * Nc
    f = qp.constraints(gamma, mu)
    eta = float(-(f @ lam))
    t = NU * m / eta
    r_dual, r_cent = residuals(N, r, gamma, lam, t, mu)
    rt_norm = float(np.sqrt(r_dual @ r_dual + r_cent @ r_cent))
    S = qp.schur_matrix(N, gamma, lam, mu)
    rhs = qp.newton_rhs(N, r, gamma, lam, t, mu)
    if newton_solver is None:
        dgamma, its = solve_newton(S, rhs, method)
    else:
        dgamma, its = newton_solver(S, rhs)
    g = qp.constraint_grads(gamma, mu)
    gradf_dg = np.concatenate([(g * dgamma.reshape(-1, 3)).sum(axis=1), -dgamma[0::3]])
    dlam = -lam - 1.0 / (t * f) - (lam / f) * gradf_dg
    neg = dlam < 0
    s_max = 1.0
    if np.any(neg):
        s_max = min(1.0, float(np.min(-lam[neg] / dlam[neg])))
    s = STEP_FRACTION * s_max
    halv = 0
    while np.any(qp.constraints(gamma + s * dgamma, mu) >= 0.0):
        s *= BETA
        halv += 1
        if halv > MAX_HALVINGS:
            raise RuntimeError("PDIP line search: no feasible step")
    while True:
        rd, rc = residuals(N, r, gamma + s * dgamma, lam + s * dlam, t, mu)
        if np.sqrt(rd @ rd + rc @ rc) <= (1.0 - ALPHA * s) * rt_norm:
            break
        s *= BETA
        halv += 1
        if halv > MAX_HALVINGS:
            raise RuntimeError("PDIP line search: no sufficient decrease")
    info = StepInfo(eta=eta, t=t, r_dual_norm=float(np.linalg.norm(r_dual)), r_t_norm=rt_norm, s=s,
                    dgamma=dgamma, dlam=dlam, krylov_iters=its, halvings=halv)
    return gamma + s * dgamma, lam + s * dlam, info


@dataclass
class PDIPResult:
    gamma: np.ndarray
    lam: np.ndarray
    iters: int
    eta: float
    r_dual_norm: float
    converged: bool
    history: list = field(default_factory=list)


def pdip_solve(N, r, mu, tol_gap=1e-8, tol_dual=1e-8, maxit=200, method="auto", gamma0=None, lam0=None,
               keep_iterates=False, newton_solver=None) -> PDIPResult:
    """PDIP to eta <= tol_gap and ||r_dual|| <= tol_dual from the cold start.

    Returns after `maxit` iterations with converged=False when the tolerances
    are not met (no exception), so that callers can inspect the iterate.
    """
    Nc = r.size // 3
    if gamma0 is None:
        gamma, lam = qp.initial_point(Nc, mu)
    else:
        gamma, lam = gamma0.copy(), lam0.copy()
    hist = []
    for it in range(maxit + 1):
        f = qp.constraints(gamma, mu)
        eta = float(-(f @ lam))
        r_dual = N @ gamma + r + qp.lagrangian_grad(gamma, lam, mu)
        rdn = float(np.linalg.norm(r_dual))
        if (eta <= tol_gap and rdn <= tol_dual) or it == maxit:
            return PDIPResult(gamma, lam, it, eta, rdn, eta <= tol_gap and rdn <= tol_dual, hist)
        if keep_iterates:
            hist.append((gamma.copy(), lam.copy()))
        gamma, lam, info = pdip_step(N, r, mu, gamma, lam, method, newton_solver)
        if not keep_iterates:
            hist.append(info.s)
    raise AssertionError("unreachable")
