"""Oracle: the time step around the CCP and the warm start of the next PDIP.

Test infrastructure (see the package docstring); plain numpy, float64.

Advance (Sec. 2.3, Eqs. force_balance_disc and particle_evolution_disc): with
the contact impulses gamma of the step (momentum units, compact 3Nc layout),

    v^{k+1} = v^k + dt M^-1 f_B + M^-1 D gamma      (f_B = gravity, per body)
    q^{k+1} = q^k + dt v^{k+1}                      (sphere centres; spheres need
                                                     no orientation for contact)

so that D^T v^{k+1} + b = N gamma + r for the step's QP data (Eqs. Ndef, rdef).

Warm start (Sec. 3.3, contacts persisting from one step to the next): a contact
of the new set whose body pair (a, b) was in contact at the previous step takes
that contact's impulse, moved into the interior of its cone (gamma_n at least
gn0, |gamma_t| at most shrink mu gamma_n); a new contact takes the cold start
(gn0, 0, 0).  lambda = -1/f (centred at t = 1), as in the cold start.

Pins: free fall in closed form; the identity D^T v^{k+1} + b = N gamma + r;
zero relative contact velocity of a sticking sphere on a plane after the step
(the closed-form stick impulse); momentum balance of two spheres; a hand-made
warm-start case.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import qp


def advance(scene, con, gamma: np.ndarray):
    """The scene after one step with impulses gamma (compact 3Nc)."""
    D = qp.jacobian(scene, con)
    g = np.asarray(scene.gravity, dtype=np.float64)
    vk = np.concatenate([scene.vel + scene.dt * g, scene.omega], axis=1).reshape(-1)
    vnew = (vk + qp.inv_mass_diag(scene) * (D @ gamma)).reshape(-1, 6)
    vel = vnew[:, :3].copy()
    omega = vnew[:, 3:].copy()
    pos = scene.pos + scene.dt * vel
    out = dataclasses.replace(scene, pos=pos, vel=vel, omega=omega)
    return out


def warm_start(prev_a, prev_b, prev_gamma, new_a, new_b, mu, gn0=1.0, shrink=0.9, prev_plane=None,
               new_plane=None):
    """(gamma, lambda) for the new contact set from the previous step's impulses.
    A contact persists when its (a, b) pair -- and, with walls, its static
    plane (-1 for a pair), since a sphere can touch the floor and a wall at
    once -- occurs in the previous step."""
    pp = np.full(len(prev_a), -1) if prev_plane is None else prev_plane
    npl = np.full(len(new_a), -1) if new_plane is None else new_plane
    prev = {(int(a), int(b), int(w)): c for c, (a, b, w) in enumerate(zip(prev_a, prev_b, pp))}
    Nc = len(new_a)
    gamma = np.zeros(3 * Nc)
    for c in range(Nc):
        j = prev.get((int(new_a[c]), int(new_b[c]), int(npl[c])))
        if j is None:
            gamma[3 * c] = gn0
            continue
        gn = max(float(prev_gamma[3 * j]), gn0)
        t1, t2 = float(prev_gamma[3 * j + 1]), float(prev_gamma[3 * j + 2])
        nt = np.hypot(t1, t2)
        cap = shrink * mu * gn
        if nt > cap:
            t1, t2 = t1 * (cap / nt), t2 * (cap / nt)
        gamma[3 * c:3 * c + 3] = (gn, t1, t2)
    f = qp.constraints(gamma, mu)
    return gamma, -1.0 / f
