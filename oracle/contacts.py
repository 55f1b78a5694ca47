"""Oracle: active contact set, contact frames and the contact hierarchy order.

Test infrastructure (see the package docstring); plain numpy, float64.

Follows Sec. 2.2 of the paper: the active set A(q, delta) holds every pair whose
gap Phi = |x_b - x_a| - r_a - r_b is at most delta, plus sphere/floor pairs with
Phi = (z - z_floor) - r <= delta.  Each contact carries a unit normal n (from the
first body towards the second) and two tangents t1, t2 spanning the friction
plane.  Sec. 3.3 orders contacts by a spatial octree of the contact positions; the
readings taken where the paper is silent are:

  * normal n = (x_b - x_a)/d; the floor is body "a" (static, index M), n = +z;
  * contact point p = x_a + n (r_a + Phi/2); for the floor p = (x, y, z_f + Phi/2);
  * side walls (an extension for boxed scenes): axis-aligned static planes
    x_axis = offset with the box on the side `sign`, Phi = sign (x_axis - offset) - r,
    n = sign e_axis, p on that axis = offset + sign Phi/2; static body M as well;
  * tangents: e = coordinate axis minimising |n_e| (lowest index on ties),
    t1 = (n x e)/|n x e|, t2 = n x t1;
  * order: Morton key of p quantised to 21 bits per axis over the bounding box of
    all contact points (x -> bit 3k, y -> 3k+1, z -> 3k+2), ties broken by (a, b),
    a static plane counting as M (floor) or M + 1 + w (wall w).

Every floating-point expression is written with an explicit evaluation order
(numpy never contracts a*b+c into an FMA), so the integer results (pair list and
order) are reproducible bit for bit by any IEEE implementation using the same
order.  Pins: brute-force O(M^2) pair search, hand-computed two-sphere and
sphere-on-floor geometry, Morton interleaving of known bit patterns.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

MORTON_BITS = 21


@dataclass
class Contacts:
    """Contact list in hierarchy (Morton) order.  All arrays have leading dim Nc."""

    a: np.ndarray        # int64, first body (M = static floor)
    b: np.ndarray        # int64, second body
    phi: np.ndarray      # gap function value
    n: np.ndarray        # (Nc, 3) unit normal, from a to b
    t1: np.ndarray       # (Nc, 3)
    t2: np.ndarray       # (Nc, 3)
    p: np.ndarray        # (Nc, 3) contact point
    ra: np.ndarray       # (Nc, 3) arm p - x_a (zero for the floor)
    rb: np.ndarray       # (Nc, 3) arm p - x_b
    key: np.ndarray      # uint64 Morton key
    M: int
    plane: np.ndarray = None  # int64: -1 for a pair, 0 the floor, 1 + w side wall w

    @property
    def Nc(self) -> int:
        return int(self.a.shape[0])


def candidate_pairs_bruteforce(pos: np.ndarray, radius: np.ndarray, delta: float) -> np.ndarray:
    """All pairs a < b within the envelope, by checking every pair (tiny M only)."""
    M = pos.shape[0]
    out = []
    for a in range(M):
        for b in range(a + 1, M):
            dx = pos[b, 0] - pos[a, 0]
            dy = pos[b, 1] - pos[a, 1]
            dz = pos[b, 2] - pos[a, 2]
            d2 = (dx * dx + dy * dy) + dz * dz
            s = (radius[a] + radius[b]) + delta
            if d2 <= s * s:
                out.append((a, b))
    return np.array(out, dtype=np.int64).reshape(-1, 2)


def _pairs_within(pos: np.ndarray, radius: np.ndarray, delta: float) -> np.ndarray:
    """Exact pair test d^2 <= (r_a + r_b + delta)^2 on k-d tree candidates."""
    from scipy.spatial import cKDTree

    M = pos.shape[0]
    if M < 2:
        return np.zeros((0, 2), dtype=np.int64)
    reach = (2.0 * float(radius.max()) + delta) * 1.001 + 1e-12
    cand = cKDTree(pos).query_pairs(reach, output_type="ndarray").astype(np.int64)
    if cand.size == 0:
        return np.zeros((0, 2), dtype=np.int64)
    a = np.minimum(cand[:, 0], cand[:, 1])
    b = np.maximum(cand[:, 0], cand[:, 1])
    dx = pos[b, 0] - pos[a, 0]
    dy = pos[b, 1] - pos[a, 1]
    dz = pos[b, 2] - pos[a, 2]
    d2 = (dx * dx + dy * dy) + dz * dz
    s = (radius[a] + radius[b]) + delta
    keep = d2 <= s * s
    pairs = np.stack([a[keep], b[keep]], axis=1)
    order = np.lexsort((pairs[:, 1], pairs[:, 0]))
    return pairs[order]


def tangent_frame(n: np.ndarray):
    """t1 = normalize(n x e), e the axis minimising |n_e|; t2 = n x t1."""
    an = np.abs(n)
    # lowest-index argmin of |n_e|
    e = np.where(an[:, 1] < an[:, 0], 1, 0)
    best = np.where(e == 1, an[:, 1], an[:, 0])
    e = np.where(an[:, 2] < best, 2, e)
    nx, ny, nz = n[:, 0], n[:, 1], n[:, 2]
    zero = np.zeros_like(nx)
    c0 = np.where(e == 0, zero, np.where(e == 1, -nz, ny))
    c1 = np.where(e == 0, nz, np.where(e == 1, zero, -nx))
    c2 = np.where(e == 0, -ny, np.where(e == 1, nx, zero))
    L = np.sqrt((c0 * c0 + c1 * c1) + c2 * c2)
    t1 = np.stack([c0 / L, c1 / L, c2 / L], axis=1)
    t2 = np.stack([
        ny * t1[:, 2] - nz * t1[:, 1],
        nz * t1[:, 0] - nx * t1[:, 2],
        nx * t1[:, 1] - ny * t1[:, 0],
    ], axis=1)
    return t1, t2


def morton_interleave(qx: np.ndarray, qy: np.ndarray, qz: np.ndarray) -> np.ndarray:
    """Interleave three 21-bit integers: x -> bit 3k, y -> 3k+1, z -> 3k+2."""
    key = np.zeros(qx.shape, dtype=np.uint64)
    for k in range(MORTON_BITS):
        sh = np.uint64(k)
        key |= ((qx.astype(np.uint64) >> sh) & np.uint64(1)) << np.uint64(3 * k)
        key |= ((qy.astype(np.uint64) >> sh) & np.uint64(1)) << np.uint64(3 * k + 1)
        key |= ((qz.astype(np.uint64) >> sh) & np.uint64(1)) << np.uint64(3 * k + 2)
    return key


def morton_keys(p: np.ndarray) -> np.ndarray:
    """Quantise each contact point over the bounding box of all points, interleave."""
    if p.shape[0] == 0:
        return np.zeros(0, dtype=np.uint64)
    lo = p.min(axis=0)
    hi = p.max(axis=0)
    q = np.zeros(p.shape, dtype=np.int64)
    top = (1 << MORTON_BITS) - 1
    for ax in range(3):
        ext = hi[ax] - lo[ax]
        if ext > 0.0:
            v = np.floor(((p[:, ax] - lo[ax]) / ext) * float(1 << MORTON_BITS))
            q[:, ax] = np.minimum(v, top).astype(np.int64)
    return morton_interleave(q[:, 0], q[:, 1], q[:, 2])


def detect(scene, pairs: np.ndarray | None = None) -> Contacts:
    """Active set A(q, delta) with frames, arms and keys, in (key, a, b) order."""
    pos, rad, delta = scene.pos, scene.radius, float(scene.delta)
    M = pos.shape[0]
    if pairs is None:
        pairs = _pairs_within(pos, rad, delta)
    pa, pb = pairs[:, 0], pairs[:, 1]

    # sphere-sphere contacts
    dx = pos[pb, 0] - pos[pa, 0]
    dy = pos[pb, 1] - pos[pa, 1]
    dz = pos[pb, 2] - pos[pa, 2]
    d = np.sqrt((dx * dx + dy * dy) + dz * dz)
    phi_p = d - (rad[pa] + rad[pb])
    n_p = np.stack([dx / d, dy / d, dz / d], axis=1)
    h = rad[pa] + phi_p * 0.5
    p_p = np.stack([pos[pa, 0] + n_p[:, 0] * h, pos[pa, 1] + n_p[:, 1] * h,
                    pos[pa, 2] + n_p[:, 2] * h], axis=1)

    # sphere-floor contacts (floor = static body a = M)
    fz = float(scene.floor_z)
    phi_all = (pos[:, 2] - fz) - rad
    fb = np.nonzero(phi_all <= delta)[0].astype(np.int64)
    phi_f = phi_all[fb]
    n_f = np.zeros((fb.size, 3))
    n_f[:, 2] = 1.0
    p_f = np.stack([pos[fb, 0], pos[fb, 1], fz + phi_f * 0.5], axis=1)

    # sphere-wall contacts: static planes x_axis = offset, the box on the side of
    # `sign`; like the floor, a wall is body "a" (static, index M), its normal
    # sign * e_axis points into the box, and p = offset + sign * Phi/2 on that axis
    aw, bw, phw, nw, pw = [], [], [], [], []
    for w, (axis, sign, off) in enumerate(getattr(scene, "walls", ()) or ()):
        x = pos[:, axis]
        ph_all = ((x - off) if sign > 0 else (off - x)) - rad
        sel = np.nonzero(ph_all <= delta)[0].astype(np.int64)
        ph = ph_all[sel]
        nv = np.zeros((sel.size, 3))
        nv[:, axis] = float(sign)
        pv = pos[sel].copy()
        pv[:, axis] = off + ((ph * 0.5) if sign > 0 else -(ph * 0.5))
        aw.append(np.full(sel.size, M + 1 + w, dtype=np.int64))  # plane index breaks ties below
        bw.append(sel)
        phw.append(ph)
        nw.append(nv)
        pw.append(pv)

    a = np.concatenate([pa, np.full(fb.size, M, dtype=np.int64)] + aw)
    b = np.concatenate([pb, fb] + bw)
    phi = np.concatenate([phi_p, phi_f] + phw)
    n = np.concatenate([n_p, n_f] + nw).reshape(-1, 3)
    p = np.concatenate([p_p, p_f] + pw).reshape(-1, 3)

    key = morton_keys(p)
    order = np.lexsort((b, a, key))
    a, b, phi, n, p, key = a[order], b[order], phi[order], n[order], p[order], key[order]
    plane = np.where(a >= M, a - M, -1)  # which static plane, before it is folded into body M
    a = np.minimum(a, M)  # every static plane is body M
    t1, t2 = tangent_frame(n)
    stat = a == M
    xa = np.where(stat[:, None], 0.0, pos[np.minimum(a, M - 1)] if M > 0 else 0.0)
    ra = np.where(stat[:, None], 0.0, p - xa)
    rb = p - pos[b] if b.size else np.zeros((0, 3))
    return Contacts(a=a, b=b, phi=phi, n=n, t1=t1, t2=t2, p=p, ra=ra, rb=rb, key=key, M=M, plane=plane)
