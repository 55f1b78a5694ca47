"""Oracle: the learned warm start's message-passing network (not in the paper;
an extension that predicts PDIP impulses to start from), forward and backward.

Test infrastructure (see the package docstring); plain numpy, float64.

Graph and network.  Contacts are the nodes; a message goes from a contact to
each of its (dynamic) bodies and back: m_b = sum of h_c over the contacts c of
body b, s_c = m_{a(c)} + m_{b(c)} (the static floor contributes nothing).
Features of contact c (F = 8, each multiplied by its scale): the normal n (3,
world frame), Phi/dt, the relative velocity D_c^T v in the contact frame (3:
r_c - b_c, Eq. rdef) and mu.

    h0 = relu(W0 x + b0)                           W0: 64 x 8
    hl = relu(Wl [h(l-1); s(h(l-1))] + bl)         Wl: 64 x 128, l = 1, 2, 3
    o  = Wo h3 + bo                                Wo: 3 x 64

o is the contact's impulse divided by out_scale.  Loss: mean over the 3 Nc
entries of (o - y)^2 with y = target / out_scale.  Parameters are one flat
vector [W0, b0, W1, b1, W2, b2, W3, b3, Wo, bo] (row-major weights); the
forward pass uses them as given (the GPU path rounds its weights to BF16 first;
tests hand the oracle the same rounded values).

Warm start: gamma = out_scale * o moved into the cone's interior (gamma_n >=
gn_min, |gamma_t| <= shrink mu gamma_n), lambda = -1/f (centred at t = 1).

Pins: the backward pass against central finite differences of the loss;
permutation equivariance (relabelled contacts give permuted outputs); the
message as a hand-computed body sum; the features of a sphere on a plane in
closed form; the warm start lies strictly inside the cones.
"""
from __future__ import annotations

import numpy as np

from . import qp

F, W, OUT, LAYERS = 8, 64, 3, 3
SHAPES = [(W, F), (W,)] + [(W, 2 * W), (W,)] * LAYERS + [(OUT, W), (OUT,)]
NPARAM = int(sum(np.prod(s) for s in SHAPES))


def unpack(theta: np.ndarray) -> list:
    out, k = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(theta[k:k + n].reshape(s))
        k += n
    return out


def init_params(seed: int) -> np.ndarray:
    """He-style initial weights from a seeded generator, zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in SHAPES:
        if len(s) == 2:
            parts.append(rng.standard_normal(s).reshape(-1) * np.sqrt(2.0 / s[1]))
        else:
            parts.append(np.zeros(s[0]))
    return np.concatenate(parts)


def features(scene, con, r: np.ndarray, scale: np.ndarray) -> np.ndarray:
    """(Nc, 8) scaled features; r is the compact 3Nc vector of Eq. rdef."""
    Nc = con.Nc
    x = np.zeros((Nc, F))
    x[:, 0:3] = con.n
    x[:, 3] = con.phi / scene.dt
    u = r.reshape(Nc, 3).copy()
    u[:, 0] -= con.phi / scene.dt
    x[:, 4:7] = u
    x[:, 7] = scene.mu
    return x * scale[None, :]


def _relu(z):
    return np.maximum(z, 0.0)


def message(h: np.ndarray, a: np.ndarray, b: np.ndarray, M: int) -> np.ndarray:
    """s_c = m_a + m_b with m_body = sum of h over the body's contacts."""
    m = np.zeros((M + 1, h.shape[1]))
    np.add.at(m, a, h)
    np.add.at(m, b, h)
    m[M] = 0.0  # the static floor sends nothing
    return m[a] + m[b]


def forward(theta, x, a, b, M):
    """Outputs (Nc, 3) and the activations kept for the backward pass."""
    P = unpack(theta)
    h = _relu(x @ P[0].T + P[1])
    acts = [(x, None, h)]
    for l in range(LAYERS):
        Wl, bl = P[2 + 2 * l], P[3 + 2 * l]
        s = message(h, a, b, M)
        hn = _relu(np.concatenate([h, s], axis=1) @ Wl.T + bl)
        acts.append((h, s, hn))
        h = hn
    o = h @ P[-2].T + P[-1]
    return o, acts


def loss(theta, x, a, b, M, y) -> float:
    o, _ = forward(theta, x, a, b, M)
    return float(np.mean((o - y) ** 2))


def grad(theta, x, a, b, M, y):
    """(loss, d loss / d theta) by the chain rule written out layer by layer."""
    P = unpack(theta)
    o, acts = forward(theta, x, a, b, M)
    n = o.size
    g = [np.zeros_like(p) for p in P]
    do = 2.0 * (o - y) / n
    h3 = acts[-1][2]
    g[-2] = do.T @ h3
    g[-1] = do.sum(0)
    dh = do @ P[-2]
    for l in reversed(range(LAYERS)):
        hin, s, hout = acts[l + 1]
        dz = dh * (hout > 0)
        Wl = P[2 + 2 * l]
        g[2 + 2 * l] = dz.T @ np.concatenate([hin, s], axis=1)
        g[3 + 2 * l] = dz.sum(0)
        dcat = dz @ Wl
        dhin, ds = dcat[:, :W], dcat[:, W:]
        # s = message(hin): its adjoint is the same sum over the shared bodies
        dh = dhin + message(ds, a, b, M)
    x0, _, h0 = acts[0]
    dz = dh * (h0 > 0)
    g[0] = dz.T @ x0
    g[1] = dz.sum(0)
    return float(np.mean((o - y) ** 2)), np.concatenate([q.reshape(-1) for q in g])


def warm_start(o: np.ndarray, out_scale: float, mu: float, gn_min: float, shrink: float = 0.9):
    """(gamma, lambda) from the network outputs (compact 3Nc)."""
    g = (out_scale * o).copy()
    g[:, 0] = np.maximum(g[:, 0], gn_min)
    nt = np.hypot(g[:, 1], g[:, 2])
    cap = shrink * mu * g[:, 0]
    sc = np.where(nt > cap, cap / np.maximum(nt, 1e-300), 1.0)
    g[:, 1] *= sc
    g[:, 2] *= sc
    gamma = g.reshape(-1)
    return gamma, -1.0 / qp.constraints(gamma, mu)
