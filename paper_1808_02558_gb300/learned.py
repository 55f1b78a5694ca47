"""Learned warm start (an extension; the paper has no counterpart): training and
use of the message-passing network of `mpnn_*` in include/qttpdip.h.

Marshalling and the optimisation loop only: features, forward and backward
passes, the Adam update and the warm start all run in the library's kernels.
"""
from __future__ import annotations

import math

import torch

from . import binding

NPARAM = 25539
SHAPES = [(64, 8), (64,)] + [(64, 128), (64,)] * 3 + [(3, 64), (3,)]


def init_params(seed: int, device="cuda") -> torch.Tensor:
    """He-scaled normal weights, zero biases (FP32 master vector)."""
    g = torch.Generator().manual_seed(seed)
    parts = []
    for s in SHAPES:
        if len(s) == 2:
            parts.append(torch.randn(s, generator=g, dtype=torch.float64).reshape(-1) * math.sqrt(2.0 / s[1]))
        else:
            parts.append(torch.zeros(s[0], dtype=torch.float64))
    return torch.cat(parts).to(torch.float32).to(device)


class WarmStartNet:
    """Parameters, Adam moments and the two scales of the network."""

    def __init__(self, seed: int, feat_scale, out_scale: float, device="cuda"):
        self.params = init_params(seed, device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.feat_scale = [float(x) for x in feat_scale]
        self.out_scale = float(out_scale)
        self.step = 0

    def train_step(self, ctx: binding.Context, target_gamma: torch.Tensor, lr: float) -> float:
        """One Adam step on one scene; target_gamma: compact (3 Nc) impulses."""
        y = (target_gamma / self.out_scale).to(torch.float32).contiguous()
        loss = ctx.mpnn_grad(self.params, self.feat_scale, y, self.grad)
        self.step += 1
        ctx.mpnn_adam(self.params, self.m, self.v, self.grad, self.step, lr)
        return loss

    def predict(self, ctx: binding.Context, Nc: int) -> torch.Tensor:
        out = torch.empty(3 * Nc, dtype=torch.float32, device=self.params.device)
        ctx.mpnn_forward(self.params, self.feat_scale, out)
        return out

    def warm_start(self, ctx: binding.Context, st: binding.State, Nc: int, gn_min: float, shrink: float = 0.9):
        ctx.mpnn_warm_start(st, self.predict(ctx, Nc), self.out_scale, gn_min, shrink)

    def start(self, ctx: binding.Context, st: binding.State, Nc: int, gn_min: float, shrink: float = 0.9):
        """Set the PDIP iterate to the network's warm start; returns (eta, r_dual) of
        the cold start and of the learned start (for reporting)."""
        ctx.pdip_init(st, 1.0)
        cold = ctx.pdip_measure(st)
        self.warm_start(ctx, st, Nc, gn_min, shrink)
        return cold, ctx.pdip_measure(st)

    def solve(self, ctx: binding.Context, st: binding.State, Nc: int, opts: binding.PdipOpts, gn_min: float,
              cap: int, gap_tol: float = 1e-8, dual_tol: float = 1e-8, max_iter: int = 200, shrink: float = 0.9):
        """PDIP to the tolerances from the learned start, with the cold start as the
        fallback: when the PDIP from the learned start has not converged within
        `cap` iterations, it is restarted from the cold start (Sec. 3.3 initial
        point) with the full budget.  Neither the dual residual nor the objective
        at the starting point predicts the PDIP's iteration count, so the fallback
        is decided by the outcome.  Returns ("learned" or "cold", total PDIP
        iterations, final PdipStats)."""
        self.warm_start(ctx, st, Nc, gn_min, shrink)
        stats, n = ctx.pdip_solve(st, opts, gap_tol=gap_tol, dual_tol=dual_tol, max_iter=cap,
                                  allow=(binding.QP_NOT_CONVERGED, binding.QP_LINESEARCH_FAIL))
        if stats.status == binding.QP_OK:
            return "learned", n, stats
        ctx.pdip_init(st, 1.0)
        stats2, n2 = ctx.pdip_solve(st, opts, gap_tol=gap_tol, dual_tol=dual_tol, max_iter=max_iter)
        return "cold", n + n2, stats2
