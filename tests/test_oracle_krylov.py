"""Oracle pin for the Jacobi-PCG Newton solver: exact solution by dense Cholesky."""
import numpy as np
import scipy.linalg as sla

from oracle import contacts as oc, krylov, pdip, qp
from synth import lattice_scene


def test_jacobi_pcg_matches_cholesky_on_schur_system():
    s = lattice_scene(3, 2)
    c = oc.detect(s)
    _, N, r = qp.qp_data(s, c)
    g, lam = qp.initial_point(c.Nc, s.mu)
    for _ in range(4):
        g, lam, _ = pdip.pdip_step(N, r, s.mu, g, lam)
    S = qp.schur_matrix(N, g, lam, s.mu)
    f = qp.constraints(g, s.mu)
    rhs = qp.newton_rhs(N, r, g, lam, pdip.NU * 2 * c.Nc / float(-(f @ lam)), s.mu)
    x, info = krylov.jacobi_pcg(S, rhs, tol=1e-12, maxit=20000)
    exact = sla.cho_solve(sla.cho_factor(S.toarray()), rhs)
    assert info["converged"] and info["true_rel_res"] < 1e-11
    assert np.linalg.norm(x - exact) <= 1e-8 * np.linalg.norm(exact)
