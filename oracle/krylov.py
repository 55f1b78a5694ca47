"""Oracle: Jacobi-preconditioned conjugate gradients (the plain Newton solver).

Test infrastructure (see the package docstring); plain numpy/scipy, float64.

Textbook preconditioned CG (Saad, Iterative Methods for Sparse Linear Systems,
Alg. 9.1) with the diagonal of S as preconditioner, started from x0 = 0 and
stopped when ||b - S x||_2 <= tol ||b||_2 (the recurrence residual; the true
residual is reported too).  The paper solves the Schur system with Krylov
methods (Sec. 3.3, 4.2); its timed baseline here is this Jacobi-PCG.

Pin: exact solution of SPD systems (dense Cholesky) on small cases.
"""
from __future__ import annotations

import numpy as np


def jacobi_pcg(S, b, tol=1e-10, maxit=10000, x0=None, precond=None):
    """Solve S x = b; precond(r) -> z overrides the Jacobi preconditioner."""
    n = b.size
    x = np.zeros(n) if x0 is None else x0.copy()
    dinv = 1.0 / S.diagonal()
    apply_m = precond if precond is not None else (lambda v: dinv * v)
    r = b - S @ x
    bn = float(np.linalg.norm(b))
    if bn == 0.0:
        return x, {"iters": 0, "rel_res": 0.0, "true_rel_res": 0.0, "converged": True}
    z = apply_m(r)
    p = z.copy()
    rz = float(r @ z)
    it = 0
    converged = float(np.linalg.norm(r)) <= tol * bn
    while not converged and it < maxit:
        q = S @ p
        alpha = rz / float(p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        if float(np.linalg.norm(r)) <= tol * bn:
            converged = True
            break
        z = apply_m(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    true = float(np.linalg.norm(b - S @ x)) / bn
    return x, {"iters": it, "rel_res": float(np.linalg.norm(r)) / bn, "true_rel_res": true,
               "converged": converged}
