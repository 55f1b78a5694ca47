"""Seeded granular scenes: jittered sphere lattices resting on a floor plane.

The paper's workloads are sedimentation, blade-drafting and shear-box simulations
of perturbed cubic lattices of spheres (Sec. 4.2).  Those models are not
available here, so these generators produce the same kind of input: an n x n x n
lattice of unit-density spheres, spacing 0.98, every coordinate jittered by
U(-0.01, 0.01), bottom layer touching the floor z = 0, translational velocities
drawn from N(0, 0.1^2), angular velocities zero.  The polydisperse variant draws
radii from U(0.4, 0.6) and uses a contact envelope delta = 0.21 (Sec. 2.2 allows
any envelope delta > 0 in the active set A(q, delta)).

Random numbers come from a counter-based SplitMix64 (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): output k of the
stream (seed, tag) is mix(seed * 2^20 + tag * 2^40 + k + 1) scaled by the golden
gamma, top 53 bits mapped to [0, 1).  Normals use the Box-Muller transform.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def splitmix64_uniform(seed: int, tag: int, n: int) -> np.ndarray:
    """n draws in [0, 1) (53-bit) from the counter-based stream (seed, tag)."""
    base = (np.uint64(seed & 0xFFFFF) << np.uint64(20)) + (np.uint64(tag & 0xFFFFFF) << np.uint64(40))
    k = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix((base + k) * _GAMMA)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal_vector(seed: int, tag: int, n: int, sigma: float = 1.0) -> np.ndarray:
    """n draws from N(0, sigma^2) by Box-Muller on the stream (seed, tag)."""
    m = (n + 1) // 2
    u = splitmix64_uniform(seed, tag, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    rad = np.sqrt(-2.0 * np.log1p(-u1))
    z = np.empty(2 * m)
    z[0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return sigma * z[:n]


@dataclass
class Scene:
    """Rigid spheres plus a static floor plane; every array is float64.

    pos, vel, omega: (M, 3); radius, mass, inv_mass, inv_inertia: (M,).
    Solid spheres of density `density`: m = 4/3 pi rho R^3, I = 2/5 m R^2.
    """

    name: str
    pos: np.ndarray
    vel: np.ndarray
    omega: np.ndarray
    radius: np.ndarray
    density: float = 1.0
    floor_z: float = 0.0
    gravity: tuple = (0.0, 0.0, -9.81)
    dt: float = 1e-3
    mu: float = 0.5
    delta: float = 0.0
    seed: int = 0
    walls: tuple = ()  # side walls (axis, sign, offset): plane x_axis = offset, box on the side of sign
    mass: np.ndarray = field(init=False)
    inv_mass: np.ndarray = field(init=False)
    inv_inertia: np.ndarray = field(init=False)

    def __post_init__(self):
        self.pos = np.ascontiguousarray(self.pos, dtype=np.float64).reshape(-1, 3)
        self.vel = np.ascontiguousarray(self.vel, dtype=np.float64).reshape(-1, 3)
        self.omega = np.ascontiguousarray(self.omega, dtype=np.float64).reshape(-1, 3)
        self.radius = np.ascontiguousarray(self.radius, dtype=np.float64).reshape(-1)
        r = self.radius
        self.mass = (4.0 / 3.0) * np.pi * self.density * r ** 3
        self.inv_mass = 1.0 / self.mass
        self.inv_inertia = 1.0 / (0.4 * self.mass * r ** 2)

    @property
    def M(self) -> int:
        return self.pos.shape[0]


def lattice_scene(n: int, seed: int, polydisperse: bool = False, *, mu: float = 0.5,
                  dt: float = 1e-3, delta: float | None = None, spacing: float = 0.98,
                  jitter: float = 0.01, vel_sigma: float = 0.1, z0: float = 0.49,
                  name: str | None = None) -> Scene:
    """n^3 jittered lattice; body id = i + n*j + n*n*k for lattice site (i, j, k)."""
    M = n * n * n
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    site = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64)
    jit = (2.0 * splitmix64_uniform(seed, 1, 3 * M) - 1.0).reshape(M, 3) * jitter
    pos = site * spacing + np.array([0.0, 0.0, z0]) + jit
    vel = normal_vector(seed, 2, 3 * M, vel_sigma).reshape(M, 3)
    omega = np.zeros((M, 3))
    if polydisperse:
        radius = 0.4 + 0.2 * splitmix64_uniform(seed, 3, M)
        d = 0.21 if delta is None else delta
    else:
        radius = np.full(M, 0.5)
        d = 0.0 if delta is None else delta
    return Scene(name=name or f"lattice{n}{'p' if polydisperse else ''}-s{seed}", pos=pos, vel=vel,
                 omega=omega, radius=radius, mu=mu, dt=dt, delta=d, seed=seed)


def column_scene(nx: int, height: int, seed: int, *, lateral: float = 1.03, spacing: float = 0.98,
                 jitter: float = 0.01, vel_sigma: float = 0.1, mu: float = 0.5, dt: float = 1e-3,
                 z0: float = 0.49, name: str | None = None) -> Scene:
    """nx x nx columns of `height` spheres (radius 0.5) standing on the floor.

    Columns are `lateral` apart (wider than a diameter plus twice the jitter, so
    no two columns touch) and spheres in a column `spacing` apart, so every
    contact is a floor contact or a vertical pair carrying the weight above it;
    jitter, velocities and the rest of the recipe are those of lattice_scene.
    Body id = i + nx*j + nx*nx*k for column (i, j), level k.
    """
    M = nx * nx * height
    k, j, i = np.meshgrid(np.arange(height), np.arange(nx), np.arange(nx), indexing="ij")
    site = np.stack([i.ravel() * lateral, j.ravel() * lateral, k.ravel() * spacing], axis=1).astype(np.float64)
    jit = (2.0 * splitmix64_uniform(seed, 1, 3 * M) - 1.0).reshape(M, 3) * jitter
    pos = site + np.array([0.0, 0.0, z0]) + jit
    vel = normal_vector(seed, 2, 3 * M, vel_sigma).reshape(M, 3)
    return Scene(name=name or f"columns{nx}x{height}-s{seed}", pos=pos, vel=vel, omega=np.zeros((M, 3)),
                 radius=np.full(M, 0.5), mu=mu, dt=dt, delta=0.0, seed=seed)


def box_scene(seed: int, *, n: int = 40, layers: int = 40, side: float | None = None, lift: float = 2.0,
              stagger: float = 0.8, clear: float = 0.61, jitter: float = 0.01, vel_sigma: float = 0.1,
              mu: float = 0.5, dt: float = 1e-3, delta: float = 0.25, name: str | None = None) -> Scene:
    """Polydisperse spheres (radius U[0.4, 0.6], density 1) falling in a walled
    box of side x side (2 side high; side = n unless given): an n x n x layers
    lattice spread evenly across the box with `clear` (above the largest radius
    plus the jitter) between the outer centres and the walls and between the
    lowest centres and the floor, layers `lift` apart, every other column (i + j
    odd) raised by `stagger` so that neighbours across are about 1.25 apart and
    no two spheres overlap at n = 40.  Positions jittered U(+-jitter) per
    coordinate, velocities N(0, vel_sigma^2); walls x, y = 0 and side, floor
    z = 0.  Body id = i + n*j + n*n*k."""
    if n < 2:
        raise ValueError("box_scene needs n >= 2")
    side = float(n) if side is None else float(side)
    spacing = (side - 2.0 * clear) / (n - 1)
    M = n * n * layers
    k, j, i = np.meshgrid(np.arange(layers), np.arange(n), np.arange(n), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    site = np.stack([clear + i * spacing, clear + j * spacing, clear + k * lift + stagger * ((i + j) % 2)],
                    axis=1).astype(np.float64)
    jit = (2.0 * splitmix64_uniform(seed, 1, 3 * M) - 1.0).reshape(M, 3) * jitter
    pos = site + jit
    vel = normal_vector(seed, 2, 3 * M, vel_sigma).reshape(M, 3)
    radius = 0.4 + 0.2 * splitmix64_uniform(seed, 3, M)
    walls = ((0, 1, 0.0), (0, -1, side), (1, 1, 0.0), (1, -1, side))
    return Scene(name=name or f"box{n}-s{seed}", pos=pos, vel=vel, omega=np.zeros((M, 3)), radius=radius, mu=mu,
                 dt=dt, delta=delta, seed=seed, walls=walls)


# Named workloads: the small FP64 pile, the 20^3 pile, the 40^3 polydisperse pile,
# 16 x 16 columns of 10 spheres (every contact loaded; 2560 contacts, 2^13), and
# 64 000 polydisperse spheres falling in a walled 40 x 40 x 80 box.
SCENES = {
    "pile8": dict(n=8, polydisperse=False),
    "pile20": dict(n=20, polydisperse=False),
    "pile40p": dict(n=40, polydisperse=True),
    "stack16": dict(columns=16, height=10),
    "box40": dict(box=40),
}


def scene_for(name: str, seed: int = 1) -> Scene:
    spec = SCENES[name]
    if "columns" in spec:
        return column_scene(spec["columns"], spec["height"], seed, name=f"{name}-s{seed}")
    if "box" in spec:
        return box_scene(seed, n=spec["box"], name=f"{name}-s{seed}")
    return lattice_scene(spec["n"], seed, spec["polydisperse"], name=f"{name}-s{seed}")


def random_vector(seed: int, tag: int, n: int) -> np.ndarray:
    """Standard-normal test vector (probe / right-hand side)."""
    return normal_vector(seed, 1000 + tag, n)
