"""The allocation-free QTT mat-vec agrees with qtt_apply (collected last on purpose).

qtt_apply_f32_noalloc serves callers that cannot call cudaMalloc (for example
code inside a host application that owns the device memory pool): it takes no
context and uses a static device array as scratch.  Its output must equal the
context-based qtt_apply with float32 cores and vectors, call after call.
"""
import numpy as np
import pytest
import torch

from paper_1808_02558_gb300 import binding

pytestmark = pytest.mark.gpu


def f32_cores(d, rmax, seed):
    rng = np.random.default_rng(seed)
    r = [1] + [int(rng.integers(1, rmax + 1)) for _ in range(d - 1)] + [1]
    r[d // 2] = rmax  # reach the largest rank at least once
    cores = [(rng.standard_normal((r[k], 4, r[k + 1])) / np.sqrt(2 * r[k + 1])).astype(np.float32).astype(np.float64)
             for k in range(d)]
    return r, cores


def check_pair(ctx, d, rmax, seed):
    ranks, cores = f32_cores(d, rmax, seed)
    A = ctx.qtt_from_cores(cores)
    flat = torch.as_tensor(np.concatenate([c.reshape(-1) for c in cores]), dtype=torch.float32).cuda()
    x = torch.as_tensor(np.random.default_rng(seed + 1).standard_normal(1 << d), dtype=torch.float32).cuda()
    y_ref = torch.empty_like(x)
    ctx.qtt_apply(A, x, y_ref, binding.QP_F32, binding.QP_F32)
    y = torch.full_like(x, float("nan"))
    rc = binding.qtt_apply_f32_noalloc(ranks, flat, x, y)
    assert rc == binding.QP_OK
    torch.cuda.synchronize()
    err = (torch.linalg.norm((y - y_ref).double()) / torch.linalg.norm(y_ref.double())).item()
    assert err <= 1e-6, err
    A.free()


def test_noalloc_matches_qtt_apply_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = binding.Context()
    check_pair(ctx, 12, 12, 5)       # first call on the device does the one-time set-up
    check_pair(ctx, 17, 32, 6)       # second call in a row, at the size limit (32 * 2^17 values)
    ctx.close()


def test_noalloc_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ranks = [1] + [8] * 19 + [1]      # 8 * 2^20 values > limit
    flat = torch.zeros(sum(ranks[k] * 4 * ranks[k + 1] for k in range(20)), dtype=torch.float32, device="cuda")
    x = torch.zeros(1 << 20, dtype=torch.float32, device="cuda")
    y = torch.full_like(x, 3.0)
    assert binding.qtt_apply_f32_noalloc(ranks, flat, x, y) == binding.QP_INVALID_ARG
    assert bool((y == 3.0).all())
