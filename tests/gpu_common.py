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

    def oracle_iterates(self, k):
        """(gamma, lambda) after k oracle PDIP iterations from the cold start."""
        g, lam = qp.initial_point(self.Nc, self.scene.mu)
        for _ in range(k):
            g, lam, _ = pdip.pdip_step(self.N, self.r, self.scene.mu, g, lam)
        return g, lam

    def state(self, gamma, lam):
        gd = dev(self.pad(gamma))
        ld = dev(lam)
        return gd, ld, self.ctx.state(gd, ld)


def relerr(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
