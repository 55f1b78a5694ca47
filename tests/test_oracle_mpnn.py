"""Pins of the learned warm start's oracle (message-passing network)."""
import numpy as np

from oracle import contacts as oc, mpnn, qp
from synth import lattice_scene


def small_problem(seed=3):
    s = lattice_scene(3, seed, polydisperse=True)
    con = oc.detect(s)
    _, _, r = qp.qp_data(s, con)
    scale = np.array([1, 1, 1, 0.05, 0.05, 0.5, 0.5, 2.0])
    x = mpnn.features(s, con, r, scale)
    rng = np.random.default_rng(seed)
    y = rng.standard_normal((con.Nc, 3))
    return s, con, x, y


def test_parameter_count():
    assert mpnn.NPARAM == 64 * 8 + 64 + 3 * (64 * 128 + 64) + 3 * 64 + 3


def test_backward_matches_finite_differences():
    s, con, x, y = small_problem()
    rng = np.random.default_rng(2)
    theta = 0.5 * mpnn.init_params(1) + 0.01 * rng.standard_normal(mpnn.NPARAM)
    L, g = mpnn.grad(theta, x, con.a, con.b, s.M, y)
    assert 0.1 < L < 100.0
    idx = np.concatenate([rng.choice(mpnn.NPARAM, 60, replace=False), [0, 512, 600, mpnn.NPARAM - 1]])
    h = 1e-5
    for i in idx:
        e = np.zeros(mpnn.NPARAM)
        e[i] = h
        fd = (mpnn.loss(theta + e, x, con.a, con.b, s.M, y) - mpnn.loss(theta - e, x, con.a, con.b, s.M, y)) / (2 * h)
        # central differences: O(h^2) truncation plus roundoff of order eps L / h
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9 * L, (i, fd, g[i])


def test_permutation_equivariance():
    s, con, x, y = small_problem(4)
    theta = mpnn.init_params(5)
    o, _ = mpnn.forward(theta, x, con.a, con.b, s.M)
    perm = np.random.default_rng(6).permutation(con.Nc)
    o2, _ = mpnn.forward(theta, x[perm], con.a[perm], con.b[perm], s.M)
    assert np.allclose(o2, o[perm], rtol=1e-12, atol=1e-12)


def test_message_is_a_body_sum():
    """Two contacts sharing body 1 exchange their features; the floor (body M) sends nothing."""
    M = 3
    a, b = np.array([0, 1, M]), np.array([1, 2, 2])
    h = np.array([[1.0], [10.0], [100.0]])
    s = mpnn.message(h, a, b, M)
    # m0 = 1, m1 = 1 + 10, m2 = 10 + 100, m_floor = 0
    assert np.array_equal(s[:, 0], [1 + 11, 11 + 110, 0 + 110])


def test_warm_start_inside_cones():
    rng = np.random.default_rng(9)
    o = rng.standard_normal((50, 3)) * 3
    g, lam = mpnn.warm_start(o, 2.0, 0.4, 1e-3)
    f = qp.constraints(g, 0.4)
    assert np.all(f < 0) and np.all(g[0::3] >= 1e-3) and np.all(lam > 0)


def test_features_of_a_sphere_on_a_plane():
    """Closed form: the floor contact's normal is +z; its frame is t1 = +y, t2 = -x
    (n x e_x normalised, then n x t1); the relative velocity in that frame is the
    sphere's velocity after gravity's step plus w x rho, projected; Phi/dt and mu
    follow; each feature is multiplied by its scale."""
    import sys
    import os

    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from test_oracle_qp import sphere_on_plane

    v = np.array([0.3, -0.2, 0.05])
    w = np.array([1.0, 2.0, -3.0])
    s = sphere_on_plane(v, w, phi=0.01, mu=0.7)
    con = oc.detect(s)
    _, _, r = qp.qp_data(s, con)
    scale = np.array([1.0, 2.0, 3.0, 0.5, 0.25, 4.0, 5.0, 6.0])
    x = mpnn.features(s, con, r, scale)
    rho = np.array([0.0, 0.0, -0.5 - 0.005])  # contact point (x, y, Phi/2) minus the centre
    vel = v + s.dt * np.array(s.gravity) + np.cross(w, rho)
    want = np.array([0.0, 0.0, 1.0, 0.01 / s.dt, vel[2], vel[1], -vel[0], 0.7]) * scale
    assert x.shape == (1, 8)
    assert np.allclose(x[0], want, rtol=1e-12, atol=1e-12)
