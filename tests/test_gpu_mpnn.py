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


def test_forward_and_backward_full_size(ctx):
    """The 40^3 pile (191 806 contacts, 1499 row tiles of the tensor-core GEMM,
    the last one partial): forward pass and gradient against the oracle, with
    the same tolerances as the small case."""
    pb = Problem(ctx, scene_for("pile40p", 1))
    params = learned.init_params(9)
    theta = bf16_round(to_np(params))
    x = mpnn.features(pb.scene, pb.oc, pb.r, np.array(SCALE))
    out = torch.empty(3 * pb.Nc, dtype=torch.float32, device="cuda")
    pb.ctx.mpnn_forward(params, SCALE, out)
    want, _ = mpnn.forward(theta, x, pb.oc.a, pb.oc.b, pb.scene.M)
    assert_close(to_np(out), want.reshape(-1), 1e-4, floor_rel=1e-2, what="forward, 40^3 pile")
    y = np.random.default_rng(2).standard_normal((pb.Nc, 3))
    g = torch.empty_like(params)
    loss = pb.ctx.mpnn_grad(params, SCALE, torch.tensor(y.reshape(-1), dtype=torch.float32, device="cuda"), g)
    L, gw = mpnn.grad(theta, x, pb.oc.a, pb.oc.b, pb.scene.M, y.astype(np.float32).astype(np.float64))
    assert abs(loss - L) <= 1e-5 * L
    k = 0
    for shp in mpnn.SHAPES:
        n = int(np.prod(shp))
        assert_close(to_np(g)[k:k + n], gw[k:k + n], 1e-3, floor_rel=1e-2, what=f"gradient block {shp}, 40^3 pile")
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
    # entry by entry: the FP32 bias correction 1 - beta2^3 cancels to about 2e-5
    # relative, so the step dp is held to 1e-4 of max(|dp_i|, 1e-3 max|dp|); the
    # parameter is stored in FP32, which adds one rounding of |p1| (2^-24 |p1|)
    got = to_np(params).astype(np.float64)
    dp = np.abs(p1 - p0)
    bound = 1e-4 * np.maximum(dp, 1e-3 * dp.max()) + 2.0 ** -23 * np.abs(p1)
    err = np.abs(got - p1)
    assert np.all(err <= bound), (int(np.argmax(err / bound)), float((err / bound).max()))


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


COL_SCALE = [1.0, 1.0, 1.0, 0.05, 0.05, 0.05, 0.05, 2.0]


def column_system(seed):
    """A 16 x 16 x 10 column scene in its own context, PDIP state at the cold start."""
    from paper_1808_02558_gb300 import workload

    sc = scene_for("stack16", seed)
    c = binding.Context()
    _, con = workload.assemble(c, sc)
    g = torch.zeros(con.P, dtype=torch.float64, device="cuda")
    lam = torch.zeros(2 * con.Nc, dtype=torch.float64, device="cuda")
    st = c.state(g, lam)
    rows = (3 * torch.arange(con.Nc, device="cuda")[:, None] + torch.arange(3, device="cuda")[None, :]).reshape(-1)
    return c, con, g, lam, st, rows


def cold_solve(c, st):
    opts = c.pdip_opts(c.solve_opts(tol=1e-10, maxit=200000))
    c.pdip_init(st, 1.0)
    stats, n = c.pdip_solve(st, opts, gap_tol=1e-8, dual_tol=1e-8, max_iter=200)
    assert stats.status == binding.QP_OK
    return opts, n


def test_learned_start_cuts_pdip_iterations(ctx):
    """The network, trained on converged PDIP solutions that the library itself
    computes for columns of seeds 2-9, starts the PDIP of the unseen seed 1: it
    converges (gap and dual residual 1e-8) in fewer iterations than the cold
    start, to the same impulses (1e-6 per entry)."""
    train, cold_its = [], []
    for seed in range(2, 10):
        c, con, g, lam, st, rows = column_system(seed)
        _, n = cold_solve(c, st)
        cold_its.append(n)
        train.append((c, g[rows].clone()))
    out_scale = float(torch.cat([t[0::3] for _, t in train]).mean())
    net = learned.WarmStartNet(11, COL_SCALE, out_scale)
    first = net.train_step(train[0][0], train[0][1], 1e-3)
    for _ in range(300):
        for c, t in train:
            last = net.train_step(c, t, 1e-3)
    assert last <= 0.01 * first
    c, con, g, lam, st, rows = column_system(1)
    opts, n_cold = cold_solve(c, st)
    g_cold = g[rows].cpu().numpy()
    used, n_learned, stats = net.solve(c, st, con.Nc, opts, gn_min=1e-3 * out_scale, cap=max(cold_its))
    print(f"PDIP iterations: cold {n_cold}, learned start {n_learned} ({used})")
    assert used == "learned" and stats.status == binding.QP_OK
    assert n_learned < n_cold
    assert_close(g[rows].cpu().numpy(), g_cold, 1e-6, what="impulses from the learned start")
    for c_, _ in train:
        c_.close()
    c.close()


def test_learned_start_falls_back_to_cold(ctx):
    """An untrained, wildly scaled network: the PDIP from its start does not
    converge within the cap, the solve restarts from the cold start and ends at
    the cold start's solution."""
    c, con, g, lam, st, rows = column_system(1)
    opts, n_cold = cold_solve(c, st)
    g_cold = g[rows].cpu().numpy()
    net = learned.WarmStartNet(3, COL_SCALE, out_scale=1e6)
    used, n, stats = net.solve(c, st, con.Nc, opts, gn_min=1.0, cap=3)
    assert used == "cold" and stats.status == binding.QP_OK
    assert n == 3 + n_cold
    assert_close(g[rows].cpu().numpy(), g_cold, 1e-6, what="impulses after the fallback")
    c.close()
