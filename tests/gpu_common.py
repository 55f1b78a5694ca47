"""Shared helpers of the GPU parity tests (oracle on the CPU, library on cuda:0)."""
import numpy as np
import torch

from oracle import contacts as oc, pdip, qp
from paper_1808_02558_gb300 import binding, workload


def to_np(t):
    return t.detach().cpu().numpy()


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).cuda()


class Problem:
    """A scene assembled by both the oracle and the library."""

    def __init__(self, ctx, scene, slots=3):
        # a context holds one contact set: every problem gets its own context
        self.scene = scene
        self.slots = slots
        self.ctx = binding.Context()
        ctx = self.ctx
        self.dev, self.con = workload.assemble(ctx, scene, slots)
        self.oc = oc.detect(scene)
        self.D, self.N, self.r = qp.qp_data(scene, self.oc)
        self.Nc = self.oc.Nc
        self.L, self.P = qp.padded_size(self.Nc, slots)

    def pad(self, x):
        return qp.to_padded(x, self.Nc, self.slots, self.P)

    def unpad(self, y):
        return qp.from_padded(y, self.Nc, self.slots)

    def oracle_iterates(self, k, newton_solver=None):
        """(gamma, lambda) after k oracle PDIP iterations from the cold start."""
        g, lam = qp.initial_point(self.Nc, self.scene.mu)
        for _ in range(k):
            g, lam, _ = pdip.pdip_step(self.N, self.r, self.scene.mu, g, lam, newton_solver=newton_solver)
        return g, lam

    def state(self, gamma, lam):
        gd = dev(self.pad(gamma))
        ld = dev(lam)
        return gd, ld, self.ctx.state(gd, ld)


def relerr(a, b):
    """Norm-wise relative error; used only where the quantity itself is a norm
    (a residual) or as extra information next to an element-wise check."""
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def assert_close(got, want, rtol, floor_rel=None, floor=None, scale=None, what=""):
    """Element-wise check |got_i - want_i| <= rtol * max(|want_i|, F_i).

    F_i is the stated floor below which an entry is checked in absolute terms:
    `floor` (absolute), `floor_rel` * max|want| (a fraction of the largest
    entry), or `scale` (a per-entry array, e.g. |S| |x| for an operator apply,
    which bounds the rounding error of the sum when its terms cancel).  The
    largest of those given is used; with none, the check is purely relative.
    """
    got = np.asarray(got, dtype=np.float64).reshape(-1)
    want = np.asarray(want, dtype=np.float64).reshape(-1)
    assert got.shape == want.shape, (got.shape, want.shape)
    F = np.zeros_like(want)
    if floor is not None:
        F = np.maximum(F, floor)
    if floor_rel is not None and want.size:
        F = np.maximum(F, floor_rel * np.abs(want).max())
    if scale is not None:
        F = np.maximum(F, np.abs(np.asarray(scale, dtype=np.float64).reshape(-1)))
    bound = rtol * np.maximum(np.abs(want), F)
    err = np.abs(got - want)
    bad = np.nonzero(~(err <= bound))[0]
    if bad.size:
        i = bad[np.argmax(err[bad] / np.maximum(bound[bad], 1e-300))]
        raise AssertionError(f"{what}: {bad.size} of {want.size} entries off; worst [{i}] got {got[i]!r} "
                             f"want {want[i]!r} |err| {err[i]:.3e} > bound {bound[i]:.3e} "
                             f"(rtol {rtol}, floor {F[i]:.3e})")
    return float((err / np.maximum(np.maximum(np.abs(want), F), 1e-300)).max()) if want.size else 0.0
