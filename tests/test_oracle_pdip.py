"""Oracle pins for the PDIP solution of the CCP (Sec. 2.3-2.4).

(i)  one sphere on a frictional plane: closed-form separation / stick / slip;
(ii) 2-4 contacts: KKT conditions of Eq. qp (cone feasibility, dual cone,
     complementarity) and the optimum value against a brute-force accelerated
     projected-gradient solve with exact projection onto each friction cone.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import contacts as oc, pdip, qp
from synth import Scene
from test_oracle_qp import sphere_on_plane


def closed_form(m, mu, rn, rt, ratio=3.5):
    """Exact CCP solution for N = diag(1/m, ratio/m, ratio/m)."""
    nt = np.linalg.norm(rt)
    if rn >= mu * nt:
        return np.zeros(3), "separate"
    if nt <= ratio * mu * (-rn):
        return np.concatenate([[-m * rn], -(m / ratio) * rt]), "stick"
    gn = m * (mu * nt - rn) / (1.0 + ratio * mu * mu)
    return np.concatenate([[gn], -mu * gn * rt / nt]), "slip"


@pytest.mark.parametrize("vel,kind", [((0.01, 0.0, -0.5), "stick"), ((2.0, 0.5, -0.1), "slip"),
                                      ((0.05, 0.0, 0.3), "separate"), ((1.5, 0.0, 0.05), "slip")])
def test_sphere_on_plane_closed_form(vel, kind):
    s = sphere_on_plane(vel)
    c = oc.detect(s)
    _, N, r = qp.qp_data(s, c)
    want, got_kind = closed_form(s.mass[0], s.mu, r[0], r[1:3])
    assert got_kind == kind
    res = pdip.pdip_solve(N, r, s.mu, tol_gap=1e-12, tol_dual=1e-8, maxit=200)
    scale = max(1.0, np.abs(want).max()) * s.mass[0]
    assert res.eta <= (1e-12 if kind != "separate" else 1e-8)
    # at the cone apex (separation) grad f_c vanishes and the dual residual of
    # the quadratic cone constraint converges sublinearly; the gap still closes
    assert res.converged or kind == "separate"
    assert np.allclose(res.gamma, want, rtol=0, atol=1e-6 * scale)


def project_cones(g, mu):
    g = g.reshape(-1, 3).copy()
    gn = g[:, 0]
    st = np.hypot(g[:, 1], g[:, 2])
    inside = st <= mu * gn
    polar = mu * st <= -gn
    mid = ~inside & ~polar
    gp = (gn[mid] + mu * st[mid]) / (1 + mu * mu)
    g[mid, 0] = gp
    sc = mu * gp / st[mid]
    g[mid, 1] *= sc
    g[mid, 2] *= sc
    g[polar] = 0.0
    return g.reshape(-1)


def brute_force(N, r, mu, iters=200000):
    """Accelerated projected gradient (FISTA) on Eq. qp, run to stagnation."""
    L = spla.eigsh(N, k=1, return_eigenvectors=False)[0] if N.shape[0] > 3 else np.linalg.eigvalsh(N.toarray()).max()
    g = np.zeros(r.size)
    y = g.copy()
    tk = 1.0
    for _ in range(iters):
        gn = project_cones(y - (N @ y + r) / L, mu)
        tk1 = 0.5 * (1 + np.sqrt(1 + 4 * tk * tk))
        y = gn + ((tk - 1) / tk1) * (gn - g)
        if np.abs(gn - g).max() <= 1e-15 * max(1.0, np.abs(gn).max()):
            g = gn
            break
        g, tk = gn, tk1
    return g


def small_scene(kind):
    z = 0.5
    if kind == "pair_on_floor":      # 2 spheres touching each other and the floor: 3 contacts
        pos = [[0.0, 0.0, z - 0.004], [0.995, 0.02, z - 0.002]]
        vel = [[0.4, 0.1, -0.3], [-0.2, 0.05, -0.1]]
    elif kind == "row_of_three":     # 3 spheres in a row on the floor: 5 contacts... (2 pairs + 3 floor)
        pos = [[0.0, 0.0, z - 0.003], [0.99, 0.01, z - 0.001], [1.985, -0.01, z - 0.002]]
        vel = [[0.3, 0.0, -0.2], [0.0, 0.1, -0.05], [-0.3, 0.0, 0.0]]
    else:                            # sphere resting on two others: 4 contacts
        pos = [[0.0, 0.0, z - 0.002], [0.995, 0.0, z - 0.001], [0.5, 0.01, z + 0.86]]
        vel = [[0.0, 0.0, 0.0], [0.1, 0.0, 0.0], [0.0, 0.05, -0.4]]
    M = len(pos)
    return Scene(name=kind, pos=pos, vel=vel, omega=np.zeros((M, 3)), radius=np.full(M, 0.5), mu=0.3)


@pytest.mark.parametrize("kind", ["pair_on_floor", "row_of_three", "stack"])
def test_kkt_against_brute_force(kind):
    s = small_scene(kind)
    c = oc.detect(s)
    assert 2 <= c.Nc <= 5
    D, N, r = qp.qp_data(s, c)
    res = pdip.pdip_solve(N, r, s.mu, tol_gap=1e-10, tol_dual=1e-7, maxit=400)
    assert res.eta <= 1e-8
    g = res.gamma
    mu = s.mu
    scale = np.abs(g).max()
    u = N @ g + r
    G, U = g.reshape(-1, 3), u.reshape(-1, 3)
    # primal cone, dual cone, per-contact complementarity
    assert np.all(np.hypot(G[:, 1], G[:, 2]) <= mu * G[:, 0] + 1e-9 * scale)
    assert np.all(U[:, 0] >= mu * np.hypot(U[:, 1], U[:, 2]) - 1e-6 * max(1.0, np.abs(U).max()))
    assert np.all(np.abs((G * U).sum(axis=1)) <= 1e-6 * max(1.0, scale * np.abs(U).max()))
    # optimum value and body impulses against brute force
    gb = brute_force(N, r, mu)
    q = lambda x: 0.5 * x @ (N @ x) + r @ x
    assert abs(q(g) - q(gb)) <= 1e-7 * max(1.0, abs(q(gb)))
    assert np.allclose(D @ g, D @ gb, rtol=0, atol=1e-5 * max(1.0, np.abs(D @ gb).max()))


def test_column_at_rest_matches_linear_solve():
    """A vertical column of spheres with no jitter and no velocity: every contact
    is loaded along z, so the CCP solution has gamma_t = 0 and normal impulses
    that make every post-step relative normal velocity exactly -Phi/dt (Eq.
    complementarity_disc with gamma_n > 0).  For the chain that is a small
    linear system in the impulses, written here from the momentum balance of
    each sphere (Eq. force_balance_disc), independently of N and r."""
    from synth import column_scene

    h = 6
    s = column_scene(1, h, 3, jitter=0.0, vel_sigma=0.0)
    c = oc.detect(s)
    assert c.Nc == h
    _, N, r = qp.qp_data(s, c)
    res = pdip.pdip_solve(N, r, s.mu, tol_gap=1e-12, tol_dual=1e-9, maxit=100)
    assert res.converged
    m, dt, g = s.mass[0], s.dt, s.gravity[2]
    below = {int(b): k for k, b in enumerate(c.b)}      # contact under sphere j
    A = np.zeros((h, h))
    rhs = np.zeros(h)
    # w_j = dt g + (gamma_below(j) - gamma_below(j+1)) / m;  u_c = w_j - w_{j-1} + Phi_c / dt = 0
    for j in range(h):
        k = below[j]
        for sgn, jj in ((1.0, j), (-1.0, j - 1)):
            if jj < 0:
                continue
            A[k, below[jj]] += sgn / m
            if jj + 1 < h:
                A[k, below[jj + 1]] -= sgn / m
            rhs[k] -= sgn * dt * g
        rhs[k] -= c.phi[k] / dt
    want_n = np.linalg.solve(A, rhs)
    assert np.all(want_n > 0)
    assert np.allclose(res.gamma[0::3], want_n, rtol=1e-8, atol=0)
    assert np.abs(res.gamma[1::3]).max() <= 1e-8 * want_n.max()
    assert np.abs(res.gamma[2::3]).max() <= 1e-8 * want_n.max()


def test_column_scene_converges_to_kkt():
    """The 16 x 16 x 10 column scene (every contact loaded, no cone apex): the
    PDIP reaches gap 1e-8 and dual residual 1e-8, and the KKT conditions hold."""
    from synth import scene_for

    s = scene_for("stack16", 1)
    c = oc.detect(s)
    _, N, r = qp.qp_data(s, c)
    res = pdip.pdip_solve(N, r, s.mu, tol_gap=1e-8, tol_dual=1e-8, maxit=100)
    assert res.converged and res.iters <= 60
    g = res.gamma.reshape(-1, 3)
    assert np.all(g[:, 0] > 0) and np.all(np.hypot(g[:, 1], g[:, 2]) < s.mu * g[:, 0])
    u = (N @ res.gamma + r).reshape(-1, 3)
    # dual cone: u_n >= mu ||u_t|| up to the residual; complementarity gamma . u ~ 0
    assert np.all(u[:, 0] + 1e-6 >= s.mu * np.hypot(u[:, 1], u[:, 2]) - 1e-6)
    assert abs(float((g * u).sum())) <= 1e-6 * float(np.abs(g).sum())
