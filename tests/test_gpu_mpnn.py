"""GPU parity of the learned warm start's network against the FP64 oracle:
forward pass, hand-written backward pass, Adam step, warm start, training."""
import numpy as np
import pytest
import torch

from gpu_common import Problem, assert_close, relerr, to_np
from oracle import mpnn, qp
from paper_1808_02558_gb300 import binding, learned
from synth import lattice_scene, scene_for

pytestmark = pytest.mark.gpu

SCALE = [1.0, 1.0, 1.0, 0.05, 0.05, 0.5, 0.5, 2.0]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return binding.Context()


def bf16_round(x):
    """Round float32 values to bfloat16 (nearest, ties to even), as float64."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def setup(ctx, seed=4):
    pb = Problem(ctx, lattice_scene(3, seed, polydisperse=True))
    params = learned.init_params(seed)
    theta = bf16_round(to_np(params))
    x = mpnn.features(pb.scene, pb.oc, pb.r, np.array(SCALE))
    return pb, params, theta, x


def test_forward_matches_oracle(ctx):
    pb, params, theta, x = setup(ctx)
    out = torch.empty(3 * pb.Nc, dtype=torch.float32, device="cuda")
    pb.ctx.mpnn_forward(params, SCALE, out)
    want, _ = mpnn.forward(theta, x, pb.oc.a, pb.oc.b, pb.scene.M)
    # FP32 width-64 layers against FP64 with the same bf16 weights
    assert_close(to_np(out), want.reshape(-1), 1e-4, floor_rel=1e-2, what="forward")
    assert relerr(to_np(out).astype(np.float64), want.reshape(-1)) <= 1e-5


def test_backward_matches_oracle(ctx):
    pb, params, theta, x = setup(ctx, 5)
    y = np.random.default_rng(1).standard_normal((pb.Nc, 3))
    g = torch.empty_like(params)
    loss = pb.ctx.mpnn_grad(params, SCALE, torch.tensor(y.reshape(-1), dtype=torch.float32, device="cuda"), g)
    L, want = mpnn.grad(theta, x, pb.oc.a, pb.oc.b, pb.scene.M, y.astype(np.float32).astype(np.float64))
    assert abs(loss - L) <= 1e-5 * L
    assert relerr(to_np(g).astype(np.float64), want) <= 1e-4
    # every parameter block gets its own share right
    k = 0
    for s in mpnn.SHAPES:
        n = int(np.prod(s))
        assert_close(to_np(g)[k:k + n], want[k:k + n], 1e-3, floor_rel=1e-2, what=f"gradient block {s}")
        k += n


def test_adam_step(ctx):
    pb, params, theta, x = setup(ctx)
    g = torch.randn_like(params)
    m = torch.randn_like(params) * 0.1
    v = torch.rand_like(params) * 0.1
    p0, m0, v0 = to_np(params).astype(np.float64), to_np(m).astype(np.float64), to_np(v).astype(np.float64)
    gg = to_np(g).astype(np.float64)
    pb.ctx.mpnn_adam(params, m, v, g, 3, lr=1e-2)
    m1 = 0.9 * m0 + 0.1 * gg
    v1 = 0.999 * v0 + 0.001 * gg * gg
    p1 = p0 - 1e-2 * (m1 / (1 - 0.9 ** 3)) / (np.sqrt(v1 / (1 - 0.999 ** 3)) + 1e-8)
    # the update itself, entry by entry: the FP32 bias correction 1 - beta2^3 cancels to
    # about 2e-5 relative, so the step is checked to 1e-4 of max(|dp_i|, 1e-3 max|dp|)
    assert_close(to_np(params).astype(np.float64) - p0, p1 - p0, 1e-4, floor_rel=1e-3, what="Adam update")


def test_warm_start_matches_oracle(ctx):
    pb, params, theta, x = setup(ctx)
    out = torch.randn(3 * pb.Nc, dtype=torch.float32, device="cuda") * 3
    g = torch.zeros(pb.P, dtype=torch.float64, device="cuda")
    lam = torch.zeros(2 * pb.Nc, dtype=torch.float64, device="cuda")
    st = pb.ctx.state(g, lam)
    pb.ctx.mpnn_warm_start(st, out, 2.5, gn_min=1e-2, shrink=0.9)
    wg, wl = mpnn.warm_start(to_np(out).astype(np.float64).reshape(-1, 3), 2.5, pb.scene.mu, 1e-2, 0.9)
    assert_close(pb.unpad(to_np(g)), wg, 1e-14, floor_rel=1e-6, what="warm-start gamma")
    assert_close(to_np(lam), wl, 1e-12, floor_rel=1e-9, what="warm-start lambda")


def test_training_fits_pdip_iterates(ctx):
    """A few hundred Adam steps on PDIP iterates of two 8^3 piles lower the loss."""
    net = learned.WarmStartNet(7, SCALE, out_scale=100.0)
    data = []
    for seed in (2, 3):
        pb = Problem(ctx, scene_for("pile8", seed))
        g, lam = pb.oracle_iterates(6)
        data.append((pb, torch.tensor(g, dtype=torch.float64, device="cuda")))
    first = [net.train_step(pb.ctx, t, 1e-3) for pb, t in data]
    for _ in range(150):
        for pb, t in data:
            net.train_step(pb.ctx, t, 1e-3)
    last = [net.train_step(pb.ctx, t, 1e-3) for pb, t in data]
    assert max(last) <= 0.2 * min(first)


def test_start_never_worse_than_cold(ctx):
    """net.start keeps the learned start only when its dual residual is below the
    cold start's; an untrained network falls back to the cold start exactly."""
    pb = Problem(ctx, scene_for("pile8", 1))
    g = torch.zeros(pb.P, dtype=torch.float64, device="cuda")
    lam = torch.zeros(2 * pb.Nc, dtype=torch.float64, device="cuda")
    st = pb.ctx.state(g, lam)
    pb.ctx.pdip_init(st, 1.0)
    _, rd_cold = pb.ctx.pdip_measure(st)
    g0 = g.clone()
    net = learned.WarmStartNet(3, SCALE, out_scale=1e4)  # wildly scaled: far from the cold start
    used, cold, warm = net.start(pb.ctx, st, pb.Nc, gn_min=1.0)
    _, rd = pb.ctx.pdip_measure(st)
    assert rd <= rd_cold and cold[1] == rd_cold
    if used == "cold":
        assert torch.equal(g, g0)
