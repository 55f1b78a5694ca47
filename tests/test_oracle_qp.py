"""Oracle pins for D, N, r, the Schur blocks and the padded layout (Sec. 2.3, 2.4, 3.3)."""
import numpy as np
import scipy.linalg as sla

from oracle import contacts as oc, pdip, qp
from synth import Scene, lattice_scene


def sphere_on_plane(vel, omega=(0, 0, 0), R=0.5, phi=0.0, dt=1e-3, mu=0.5):
    return Scene(name="sop", pos=[[0.3, -0.2, R + phi]], vel=[vel], omega=[omega], radius=[R], dt=dt, mu=mu,
                 delta=max(0.0, phi) + 1e-12)


def test_sphere_on_plane_N_closed_form():
    s = sphere_on_plane([0.1, 0.0, 0.0])
    c = oc.detect(s)
    _, N, _ = qp.qp_data(s, c)
    m = s.mass[0]
    assert np.allclose(N.toarray(), np.diag([1 / m, 3.5 / m, 3.5 / m]), rtol=1e-14, atol=1e-14)


def test_sphere_on_plane_r_closed_form():
    v = np.array([0.3, -0.2, 0.05])
    w = np.array([1.0, 2.0, -3.0])
    s = sphere_on_plane(v, w, phi=0.01)
    c = oc.detect(s)
    _, _, r = qp.qp_data(s, c)
    rho = c.rb[0]
    vel = v + s.dt * np.array(s.gravity) + np.cross(w, rho)
    want = np.array([0.01 / s.dt + vel[2], vel @ c.t1[0], vel @ c.t2[0]])
    assert np.allclose(r, want, rtol=1e-13, atol=1e-13)


def test_N_symmetric_and_pattern_is_edge_adjacency():
    s = lattice_scene(4, 5)
    c = oc.detect(s)
    _, N, _ = qp.qp_data(s, c)
    A = N.toarray()
    assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()
    share = np.zeros((c.Nc, c.Nc), dtype=bool)
    for i in range(c.Nc):
        bi = {c.a[i], c.b[i]} - {s.M}
        for j in range(c.Nc):
            share[i, j] = bool(bi & ({c.a[j], c.b[j]} - {s.M}))
    blk = np.abs(A).reshape(c.Nc, 3, c.Nc, 3).max(axis=(1, 3)) > 0
    assert np.array_equal(blk, share)


def test_schur_spd_and_newton_direction():
    s = lattice_scene(3, 1)
    c = oc.detect(s)
    _, N, r = qp.qp_data(s, c)
    g, lam = qp.initial_point(c.Nc, s.mu)
    for _ in range(3):
        g, lam, _ = pdip.pdip_step(N, r, s.mu, g, lam)
    S = qp.schur_matrix(N, g, lam, s.mu).toarray()
    assert np.allclose(S, S.T, rtol=0, atol=1e-12 * np.abs(S).max())
    sla.cholesky(S)  # SPD
    # the Schur step is a Newton step: d/ds ||r_t(gamma + s dg, lam + s dl)|| = -||r_t||
    f = qp.constraints(g, s.mu)
    t = pdip.NU * 2 * c.Nc / float(-(f @ lam))
    rhs = qp.newton_rhs(N, r, g, lam, t, s.mu)
    dg = np.linalg.solve(S, rhs)
    gg = qp.constraint_grads(g, s.mu)
    gdg = np.concatenate([(gg * dg.reshape(-1, 3)).sum(1), -dg[0::3]])
    dl = -lam - 1.0 / (t * f) - (lam / f) * gdg
    rd, rc = pdip.residuals(N, r, g, lam, t, s.mu)
    r0 = np.sqrt(rd @ rd + rc @ rc)
    h = 1e-7
    rd2, rc2 = pdip.residuals(N, r, g + h * dg, lam + h * dl, t, s.mu)
    slope = (np.sqrt(rd2 @ rd2 + rc2 @ rc2) - r0) / (h * r0)
    assert abs(slope + 1.0) < 1e-4


def test_schur_block_is_barrier_hessian():
    # lambda_c (-f_c) Hess[-log(-f_c)] + (lambda'/gn) e1 e1^T, checked by finite differences
    rng = np.random.default_rng(0)
    mu = 0.4
    g = np.array([2.0, 0.3, -0.2])
    lam = rng.uniform(0.5, 2.0, size=2)
    H = qp.schur_blocks(g, lam, mu)[0]

    def barrier(x):
        fc = 0.5 * (x[1] ** 2 + x[2] ** 2 - mu * mu * x[0] ** 2)
        return -np.log(-fc)

    fc = qp.constraints(g, mu)[0]
    h = 1e-4
    Hb = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            e_i, e_j = np.eye(3)[i] * h, np.eye(3)[j] * h
            Hb[i, j] = (barrier(g + e_i + e_j) - barrier(g + e_i - e_j) - barrier(g - e_i + e_j)
                        + barrier(g - e_i - e_j)) / (4 * h * h)
    want = lam[0] * (-fc) * Hb
    want[0, 0] += lam[1] / g[0]
    assert np.allclose(H, want, rtol=1e-6, atol=1e-8)


def test_padded_layout_identity_rows():
    s = lattice_scene(3, 2)
    c = oc.detect(s)
    _, N, _ = qp.qp_data(s, c)
    for slots in (3, 4):
        L, P = qp.padded_size(c.Nc, slots)
        assert P >= slots * c.Nc and P // 2 < max(slots * c.Nc, 2)
        A = qp.padded_matrix(N, c.Nc, slots, P).toarray()
        x = np.random.default_rng(1).standard_normal(P)
        y = A @ x
        idx = (slots * np.arange(c.Nc)[:, None] + np.arange(3)).reshape(-1)
        dummy = np.setdiff1d(np.arange(P), idx)
        assert np.array_equal(y[dummy], x[dummy])
        assert np.allclose(y[idx], N @ x[idx], rtol=1e-14, atol=1e-14)
