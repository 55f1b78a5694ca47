"""Pins of the time-stepping oracle (Sec. 2.3 Eqs. force_balance_disc and
particle_evolution_disc; warm start of persisting contacts, Sec. 3.3)."""
import numpy as np
import pytest

from oracle import contacts as oc, pdip, qp, timestep
from synth import Scene, lattice_scene, random_vector, scene_for
from test_oracle_pdip import closed_form
from test_oracle_qp import sphere_on_plane


def test_free_fall_closed_form():
    s = Scene(name="ff", pos=[[0.0, 0.0, 5.0]], vel=[[0.3, -0.1, 0.2]], omega=[[1.0, 2.0, 3.0]], radius=[0.5])
    con = oc.detect(s)
    assert con.Nc == 0
    s1 = timestep.advance(s, con, np.zeros(0))
    v = np.array([0.3, -0.1, 0.2 - 9.81e-3])
    assert np.allclose(s1.vel[0], v, rtol=0, atol=1e-16)
    assert np.array_equal(s1.omega[0], [1.0, 2.0, 3.0])
    assert np.allclose(s1.pos[0], [0.0, 0.0, 5.0] + 1e-3 * v, rtol=0, atol=1e-15)


def test_post_step_velocity_identity():
    """D^T v^{k+1} + b = N gamma + r for any gamma (Eqs. Ndef, rdef)."""
    s = scene_for("pile8", 2)
    con = oc.detect(s)
    D, N, r = qp.qp_data(s, con)
    gamma = random_vector(3, 5, 3 * con.Nc)
    s1 = timestep.advance(s, con, gamma)
    v6 = np.concatenate([s1.vel, s1.omega], axis=1).reshape(-1)
    b = np.zeros(3 * con.Nc)
    b[0::3] = con.phi / s.dt
    lhs = D.T @ v6 + b
    rhs = N @ gamma + r
    assert np.allclose(lhs, rhs, rtol=0, atol=1e-10 * np.abs(rhs).max())


@pytest.mark.parametrize("vel,kind", [((0.01, 0.0, -0.5), "stick"), ((2.0, 0.5, -0.1), "slip")])
def test_sphere_on_plane_contact_velocity_after_step(vel, kind):
    """Stick: the contact point is at rest after the step.  Slip: it slides
    against the friction impulse, with the normal velocity mu |u_t| that the
    cone relaxation of the complementarity condition (Eq. complementarity_relax)
    prescribes for an active contact."""
    s = sphere_on_plane(vel)
    con = oc.detect(s)
    _, N, r = qp.qp_data(s, con)
    gamma, k = closed_form(s.mass[0], s.mu, r[0], r[1:3])
    assert k == kind
    s1 = timestep.advance(s, con, gamma)
    rho = np.array([0.0, 0.0, -s.radius[0]])  # centre to contact point
    vc = s1.vel[0] + np.cross(s1.omega[0], rho)
    scale = np.abs(vel).max()
    if kind == "stick":
        assert np.allclose(vc, 0.0, rtol=0, atol=1e-12 * scale)
    else:
        ft = gamma[1] * con.t1[0] + gamma[2] * con.t2[0]
        vt = vc - vc[2] * np.array([0.0, 0.0, 1.0])
        assert abs(vc[2] - s.mu * np.linalg.norm(vt)) <= 1e-12 * scale
        cosang = vt @ ft / (np.linalg.norm(vt) * np.linalg.norm(ft))
        assert cosang <= -1 + 1e-12


def test_two_spheres_momentum_balance():
    """Contact impulses are internal: linear momentum changes by the gravity
    impulse only, angular momentum about the origin by its moment."""
    s = Scene(name="two", pos=[[0.0, 0.0, 5.0], [0.99, 0.02, 5.01]], vel=[[0.5, 0.0, 0.0], [-0.4, 0.1, 0.0]],
              omega=[[0.0, 0.0, 0.0], [0.1, 0.0, 0.0]], radius=[0.5, 0.5])
    con = oc.detect(s)
    assert con.Nc == 1
    gamma = np.array([3.0, 0.4, -0.7])
    s1 = timestep.advance(s, con, gamma)
    g = np.asarray(s.gravity)
    m = s.mass[:, None]
    dP = (m * s1.vel).sum(0) - (m * s.vel).sum(0)
    assert np.allclose(dP, s.dt * g * s.mass.sum(), rtol=0, atol=1e-13)
    I = (1.0 / s.inv_inertia)[:, None]

    def L(sc):
        return (I * sc.omega).sum(0) + np.cross(s.pos, m * sc.vel).sum(0)

    dL = L(s1) - L(s)
    assert np.allclose(dL, np.cross(s.pos, m * s.dt * g).sum(0), rtol=0, atol=1e-12)


def test_warm_start_hand_case():
    M = 3
    prev_a, prev_b = [0, 1, M], [1, 2, 0]
    prev_gamma = np.array([5.0, 1.0, 1.0,      # |gt| = 1.41 <= 0.9*0.5*5 = 2.25: kept
                           0.2, 0.1, 0.0,      # gn below gn0 = 1: raised to 1, gt kept (0.1 <= 0.45)
                           4.0, 3.0, 4.0])     # |gt| = 5 > 1.8: scaled to 1.8
    new_a, new_b = [1, 0, 0, M], [2, 1, 2, 0]
    gamma, lam = timestep.warm_start(prev_a, prev_b, prev_gamma, new_a, new_b, 0.5, gn0=1.0, shrink=0.9)
    want = np.array([1.0, 0.1, 0.0,
                     5.0, 1.0, 1.0,
                     1.0, 0.0, 0.0,
                     4.0, 3.0 * 1.8 / 5.0, 4.0 * 1.8 / 5.0])
    assert np.allclose(gamma, want, rtol=0, atol=1e-15)
    f = qp.constraints(gamma, 0.5)
    assert np.all(f < 0) and np.allclose(lam * f, -1.0, rtol=1e-15)


def test_warm_start_identity_on_same_contacts():
    """Same contact set: every contact takes its own impulse (moved inside the cone)."""
    s = scene_for("pile8", 1)
    con = oc.detect(s)
    _, N, r = qp.qp_data(s, con)
    g, lam = qp.initial_point(con.Nc, s.mu)
    for _ in range(3):
        g, lam, _ = pdip.pdip_step(N, r, s.mu, g, lam)
    g2, _ = timestep.warm_start(con.a, con.b, g, con.a, con.b, s.mu, gn0=1e-6, shrink=1.0)
    assert np.array_equal(g2, g)


def test_warm_start_keeps_floor_and_wall_apart():
    """A sphere in contact with the floor and a wall has two contacts (M, b):
    with plane indices each takes its own previous impulse; without them the
    two previous impulses cannot both be matched."""
    prev_a, prev_b = np.array([2, 2]), np.array([0, 0])
    prev_plane = np.array([0, 1])  # floor, then wall 0
    prev_gamma = np.array([5.0, 0.1, 0.0, 3.0, 0.0, 0.2])
    new_a, new_b, new_plane = np.array([2, 2]), np.array([0, 0]), np.array([1, 0])  # order swapped
    g, lam = timestep.warm_start(prev_a, prev_b, prev_gamma, new_a, new_b, 0.5, gn0=1.0, shrink=0.9,
                                 prev_plane=prev_plane, new_plane=new_plane)
    assert np.allclose(g, [3.0, 0.0, 0.2, 5.0, 0.1, 0.0])
    assert np.all(lam > 0)
    g2, _ = timestep.warm_start(prev_a, prev_b, prev_gamma, new_a, new_b, 0.5, gn0=1.0, shrink=0.9)
    assert g2[0] == g2[3]  # one previous contact serves both
