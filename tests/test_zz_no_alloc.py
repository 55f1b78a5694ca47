"""The allocation-free QTT mat-vec against the oracle (collected last on purpose).

qtt_apply_f32_noalloc serves callers that cannot call cudaMalloc (for example
code inside a host application that owns the device memory pool): it takes no
context and uses a static device array as scratch.  Its output is checked entry
by entry against the oracle's FP64 core-by-core contraction (oracle/tt.py
qtt_matvec) of the same float32-representable cores and input, and against the
context-based qtt_apply with float32 cores and vectors, on two calls in a row.

Tolerance: an FP32 chain of d core contractions (sums of 2 r terms each) has a
per-entry error of about 1e-5 (d = 12) to 3e-5 (d = 17) relative to
max(|y_i|, 1e-2 max|y|) on these cores (float32 emulation of the chain in
numpy); the check allows 1e-4 on that scale.
"""
import numpy as np
import pytest
import torch

from gpu_common import assert_close, relerr, to_np
from oracle import tt
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
    x64 = np.random.default_rng(seed + 1).standard_normal(1 << d).astype(np.float32).astype(np.float64)
    want = tt.qtt_matvec(cores, x64)
    flat = torch.as_tensor(np.concatenate([c.reshape(-1) for c in cores]), dtype=torch.float32).cuda()
    x = torch.as_tensor(x64, dtype=torch.float32).cuda()
    y = torch.full_like(x, float("nan"))
    rc = binding.qtt_apply_f32_noalloc(ranks, flat, x, y)
    assert rc == binding.QP_OK
    torch.cuda.synchronize()
    got = to_np(y).astype(np.float64)
    assert_close(got, want, 1e-4, floor_rel=1e-2, what=f"noalloc vs oracle d={d}")
    assert relerr(got, want) <= 1e-5
    # the context-based apply: FP32 too, but it fuses two cores per pass at ranks
    # <= 12, so its sums run in another order; same tolerance as against the oracle
    A = ctx.qtt_from_cores(cores)
    y_ref = torch.empty_like(x)
    ctx.qtt_apply(A, x, y_ref, binding.QP_F32, binding.QP_F32)
    assert_close(got, to_np(y_ref), 1e-4, floor_rel=1e-2, what=f"noalloc vs qtt_apply d={d}")
    A.free()


def test_noalloc_matches_oracle_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = binding.Context()
    check_pair(ctx, 12, 12, 5)       # first call on the device does the one-time set-up
    check_pair(ctx, 17, 32, 6)       # second call in a row, at the size limit (32 * 2^17 values)
    ctx.close()


def test_noalloc_rejects_oversize_and_bad_buffers():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ranks = [1] + [8] * 19 + [1]      # 8 * 2^20 values > limit
    flat = torch.zeros(sum(ranks[k] * 4 * ranks[k + 1] for k in range(20)), dtype=torch.float32, device="cuda")
    x = torch.zeros(1 << 20, dtype=torch.float32, device="cuda")
    y = torch.full_like(x, 3.0)
    assert binding.qtt_apply_f32_noalloc(ranks, flat, x, y) == binding.QP_INVALID_ARG
    assert bool((y == 3.0).all())
    # the wrapper checks what the C entry point cannot see: sizes, dtype, device
    small = [1, 2, 1]
    c = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        binding.qtt_apply_f32_noalloc(small, c, torch.zeros(3, device="cuda"), torch.zeros(4, device="cuda"))
    with pytest.raises(ValueError):
        binding.qtt_apply_f32_noalloc(small, c[:15], torch.zeros(4, device="cuda"), torch.zeros(4, device="cuda"))
    with pytest.raises(TypeError):
        binding.qtt_apply_f32_noalloc(small, c, torch.zeros(4, dtype=torch.float64, device="cuda"),
                                      torch.zeros(4, device="cuda"))
