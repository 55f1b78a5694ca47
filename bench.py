"""Benchmark: PDIP Newton solves/s at 1e-8 relative residual on the 40^3 pile.

Workload: 40x40x40 polydisperse jittered lattice (radius U[0.4, 0.6], delta =
0.21, mu = 0.5, dt = 1e-3), padded to 2^20 unknowns.  A step is a fixed window
of the time step's PDIP: reset to the cold start (Sec. 3.3), then `--window`
PDIP iterations (default 8), each with the Schur blocks and rhs, the Newton solve
to ||rhs - S dx|| <= 1e-8 ||rhs|| (FP32 inner PCG + FP64 refinement, Jacobi or
QTT preconditioner), dlambda, ratio test, backtracking and update.  Every step
does the same work, so the value does not depend on K.  The L2 is flushed
(512 MiB write) before every timed step, outside the step's events.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--precond jacobi|qtt] [--workload pile40p|pile20|pile8]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PDIP Newton solves/s at 1e-8 residual, QTT vs plain PCG; HBM GB/s fraction"
UNIT = "Newton solves/s"
WORKLOADS = {
    "pile40p": "40^3 polydisperse lattice, r~U[0.4,0.6], delta=0.21, mu=0.5, dt=1e-3, 2^20 padded unknowns",
    "pile20": "20^3 monodisperse lattice, r=0.5, mu=0.5, dt=1e-3, 2^17 padded unknowns",
    "pile8": "8^3 monodisperse lattice, r=0.5, mu=0.5, dt=1e-3, 2^13 padded unknowns",
    "stack16": "16x16 columns of 10 spheres, r=0.5, mu=0.5, dt=1e-3, 2^13 padded unknowns",
}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n_gpus):
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def _reduce(v, world, op):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    device = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(v, world):
    """Slowest rank's time: the job finishes when the last replica does."""
    import torch.distributed as dist

    return _reduce(v, world, dist.ReduceOp.MAX) if world > 1 else v


def sum_over_ranks(v, world):
    """Work done by all replicas together."""
    import torch.distributed as dist

    return _reduce(v, world, dist.ReduceOp.SUM) if world > 1 else v


def job_throughput(local_units, local_ms, world):
    """Whole-job throughput: units of all ranks / the slowest rank's time."""
    total = sum_over_ranks(local_units, world)
    ms = max_over_ranks(local_ms, world)
    return total / (ms / 1e3), ms


# ---------------------------------------------------------------------- our arm
STATUS_NAMES = {0: "ok", -4: "not_converged", -5: "breakdown", -6: "linesearch_fail", -7: "timeout"}
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one k_pcg<float, void>
# launch of the 40^3 window (mean of three consecutive launches), from an ncu capture of
# this kernel version (caches flushed by ncu before each launch).  Reset to None when the
# kernel changes.
KPCG_DRAM_BYTES_PER_LAUNCH = 137.2e6


# FP32 CUDA-core peak of the part from its unit counts: 152 SMs x 128 FP32 lanes x
# 2 flop per FMA x the maximum SM clock (2070 MHz).
FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def qtt_apply_roofline(t, nbytes, flops, passes, d):
    """Roofline entry of one QTT apply: HBM-bound when its flop/byte is below the
    ridge of the FP32 ALU peak over the measured HBM peak, ALU-bound above."""
    hbm, src = peaks()[0], peaks()[1]
    ridge = FP32_ALU_TFLOPS * 1e12 / (hbm * 1e9)
    out = {"us": t * 1e6, "bytes": nbytes, "flops": flops, "flop_per_byte": flops / nbytes,
           "ridge_flop_per_byte": ridge, "gbs": nbytes / t / 1e9, "tflops": flops / t / 1e12,
           "schedule": f"{passes} passes for {d} cores (two cores per pass where ranks <= 12)"}
    if flops / nbytes < ridge:
        out.update({"bound": "hbm", "achieved": nbytes / t / 1e9, "peak": hbm, "unit": "GB/s",
                    "frac": nbytes / t / 1e9 / hbm, "peak_source": src})
    else:
        out.update({"bound": "alu", "achieved": flops / t / 1e12, "peak": FP32_ALU_TFLOPS, "unit": "TFLOP/s",
                    "frac": flops / t / 1e12 / FP32_ALU_TFLOPS, "peak_source": "derived: 152 SM x 128 FP32 x 2 x 2.07 GHz"})
    return out


def solve_bytes(Nc, M, nrow, iters, outer):
    """Algorithmic bytes of one Newton solve: S-apply per contact/body plus the
    PCG vector passes, FP32 inner iterations and FP64 outer residuals."""
    inner = iters * (Nc * 100 + M * 48 + 10 * 4 * nrow)
    outer_b = (outer + 1) * (Nc * 200 + M * 96 + 5 * 8 * nrow)
    return inner + outer_b


def run_ours(args):
    import numpy as np
    import torch

    from paper_1808_02558_gb300 import binding, workload
    from synth import scene_for

    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", torch.cuda.current_device())
    scene = scene_for(args.workload, seed=1 + rank)
    ctx = binding.Context()
    _, con = workload.assemble(ctx, scene)
    Nc, M, P = con.Nc, con.M, con.P
    gamma = torch.zeros(P, dtype=torch.float64, device=dev)
    lam = torch.zeros(2 * Nc, dtype=torch.float64, device=dev)
    st = ctx.state(gamma, lam)
    ctx.pdip_init(st, 1.0)
    mixed = 1 if args.workload == "pile40p" else 0
    qtt = args.precond == "qtt"
    sopts = ctx.solve_opts(binding.QP_QTT_PCG if qtt else binding.QP_JACOBI_PCG, None, tol=1e-8, maxit=200000,
                           mixed=mixed, inner_tol=1e-3 if mixed else 0.0, max_outer=60,
                           core_dtype=binding.QP_BF16 if mixed else binding.QP_F32)
    opts = ctx.pdip_opts(sopts, qtt_refresh=1 if qtt else 0, qtt_eps=args.qtt_eps, qtt_rmax=args.qtt_rmax)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    ok = (binding.QP_NOT_CONVERGED, binding.QP_LINESEARCH_FAIL)

    def window(c, state, o, record=None, o_rest=None):
        """pdip_init, then args.window PDIP iterations (o for the first, o_rest, if
        given, for the others)."""
        c.pdip_init(state, 1.0)
        for i in range(args.window):
            s_ = c.pdip_step(state, o if (i == 0 or o_rest is None) else o_rest, allow=ok)
            if record is not None:
                record.append(s_)

    for _ in range(args.warmup):
        window(ctx, st, opts)
    torch.cuda.synchronize()
    barrier(world)
    step_ms, pcg_ms, iters, outer, relres, refresh_ms = [], [], [], [], [], []
    status_counts, solved, stepped = {}, 0, 0
    launches = 0
    with ClockSampler(local) as clk:
        time.sleep(0.5)  # let the sampler start before the timed region
        torch.cuda.synchronize()
        barrier(world)
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            rec = []
            e0.record(stream)
            window(ctx, st, opts, rec)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            for s in rec:
                pcg_ms.append(s.solve.ms)
                iters.append(s.solve.iters)
                outer.append(s.solve.outer)
                relres.append(s.solve.rel_res)
                refresh_ms.append(s.ms_refresh)
                name = STATUS_NAMES.get(s.status, str(s.status))
                status_counts[name] = status_counts.get(name, 0) + 1
                # a Newton solve counts when it reached the tolerance; a PDIP step
                # counts when its line search accepted a step (status OK)
                solved += int(s.solve.status == binding.QP_OK and s.solve.rel_res <= 1e-8)
                stepped += int(s.status == binding.QP_OK)
            launches += 1 + 4 * args.window  # init; pre-step, Jacobi diagonal, Krylov kernel, post-step
        torch.cuda.synchronize()
        barrier(world)
    value, total_ms = job_throughput(float(solved), sum(step_ms), world)
    pdip_steps_per_s, _ = job_throughput(float(stepped), sum(step_ms), world)

    # roofline of the dominant kernel (persistent PCG)
    nrow = 3 * Nc
    bytes_per = [solve_bytes(Nc, M, nrow, it, ou) for it, ou in zip(iters, outer)]
    ach = sum(bytes_per) / (sum(pcg_ms) / 1e3) / 1e9
    peak, src = peaks()

    # QTT leg (Sec. 3.3): the same PDIP iterates solved with the QTT-preconditioned
    # PCG, the preconditioner refreshed (compressed + inverted, warm-started) each step
    qtt_out = None
    if not qtt and args.qtt_steps > 0:
        ctxq = binding.Context()
        workload.assemble(ctxq, scene)
        gq, lq = gamma.clone(), lam.clone()
        stq = ctxq.state(gq, lq)
        soq = ctxq.solve_opts(binding.QP_QTT_PCG, None, tol=1e-8, maxit=args.qtt_maxit, mixed=mixed,
                              inner_tol=1e-3 if mixed else 0.0, max_outer=60,
                              core_dtype=binding.QP_BF16 if mixed else binding.QP_F32,
                              krylov=binding.QP_BICGSTAB if args.qtt_krylov == "bicgstab" else binding.QP_CG)
        optq = ctxq.pdip_opts(soq, qtt_refresh=1, qtt_eps=args.qtt_eps, qtt_rmax=args.qtt_rmax)
        q_ms, q_it, q_ref, q_solve, q_fb = [], [], [], [], 0
        for _ in range(args.qtt_steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            rec = []
            e0.record(stream)
            window(ctxq, stq, optq, rec)
            e1.record(stream)
            e1.synchronize()
            q_ms.append(e0.elapsed_time(e1))
            for sq in rec:
                q_it.append(sq.solve.iters)
                q_ref.append(sq.ms_refresh)
                q_solve.append(sq.solve.ms)
                q_fb += sq.solve.fallback
        # re-use across Newton iterations (Sec. 3.3): refresh at the window's first
        # iteration only, the other iterations reuse that inverse
        optr = ctxq.pdip_opts(soq, qtt_refresh=0, qtt_eps=args.qtt_eps, qtt_rmax=args.qtt_rmax)
        r_ms, r_it, r_fb = [], [], 0
        for _ in range(args.qtt_steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            rec = []
            e0.record(stream)
            window(ctxq, stq, optq, rec, o_rest=optr)
            e1.record(stream)
            e1.synchronize()
            r_ms.append(e0.elapsed_time(e1))
            for sq in rec:
                r_it.append(sq.solve.iters)
                r_fb += sq.solve.fallback
        rv = args.window * 1e3 / statistics.mean(r_ms)
        # standalone QTT apply of the refreshed preconditioner (FP32 vectors, BF16 or FP32 cores)
        S_tt = ctxq.qtt_compress(stq, args.qtt_eps, args.qtt_rmax)
        X = ctxq.qtt_inverse(S_tt, args.qtt_eps, args.qtt_rmax, sweeps=2)
        ranks = X.ranks()
        xin = torch.randn(P, dtype=torch.float32, device=dev)
        yout = torch.empty_like(xin)
        cdt = binding.QP_BF16 if mixed else binding.QP_F32
        for _ in range(3):
            ctxq.qtt_apply(X, xin, yout, cdt, binding.QP_F32)
        ap_ms = []
        for _ in range(10):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctxq.qtt_apply(X, xin, yout, cdt, binding.QP_F32)
            e1.record(stream)
            e1.synchronize()
            ap_ms.append(e0.elapsed_time(e1))
        # schedule of qtt_apply: cores d, d-1, ... in passes of two where both ranks of
        # the pair and the rank below are <= 12 (else one); a pass reads r_in * N and
        # writes r_out * N FP32 values.  Flops: core k is applied to N/2 column items,
        # each a (2 r_{k-1}) x (2 r_k) matrix times a 2 r_k vector, i.e. 4 r_{k-1} r_k
        # multiply-adds = 8 r_{k-1} r_k flops, so 4 r_{k-1} r_k N flops per core
        ap_bytes, ap_passes, k = 0, 0, len(ranks) - 1
        while k >= 1:
            fuse = k >= 2 and max(ranks[k - 1], ranks[k]) <= 12 and \
                ranks[k - 1] * ranks[k] + ranks[k - 2] * ranks[k - 1] <= 288
            nxt = k - 2 if fuse else k - 1
            ap_bytes += (ranks[k] + ranks[nxt]) * P * 4
            ap_passes += 1
            k = nxt
        ap_flops = sum(4 * ranks[k] * ranks[k + 1] * P for k in range(len(ranks) - 1))
        ap_t = statistics.median(ap_ms) / 1e3
        qv = args.window * 1e3 / statistics.mean(q_ms)
        qtt_out = {"value": qv, "unit": UNIT, "factor_vs_jacobi": qv / value,
                   "solve_only_factor_vs_jacobi": statistics.mean(pcg_ms) / statistics.mean(q_solve),
                   "krylov_iters_per_solve": statistics.mean(q_it), "refresh_ms": statistics.mean(q_ref),
                   "solve_ms": statistics.mean(q_solve), "eps": args.qtt_eps, "rmax": args.qtt_rmax,
                   "krylov": args.qtt_krylov, "maxit": args.qtt_maxit, "jacobi_fallbacks": q_fb,
                   "inverse_ranks_max": max(ranks),
                   "refresh_once_per_window": {"value": rv, "unit": UNIT, "factor_vs_jacobi": rv / value,
                                               "krylov_iters_per_solve": statistics.mean(r_it),
                                               "jacobi_fallbacks": r_fb,
                                               "note": "refresh at the first PDIP iteration, reused by the others"},
                   "qtt_apply": qtt_apply_roofline(ap_t, ap_bytes, ap_flops, ap_passes, len(ranks) - 1)}
        for h in (X, S_tt):
            h.free()
        ctxq.close()

    # end to end through the C ABI with host buffers: H2D scene + state, assemble, step, D2H state
    host = {k: v.cpu().pin_memory() for k, v in workload.scene_to_device(scene, dev).items()}
    ctx.pdip_init(st, 1.0)
    g_h = gamma.cpu().pin_memory()
    l_h = lam.cpu().pin_memory()
    ddev = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
    g2 = torch.empty_like(gamma)
    l2 = torch.empty_like(lam)
    g_out = torch.empty_like(g_h).pin_memory()
    l_out = torch.empty_like(l_h).pin_memory()
    h2d = sum(v.numel() * v.element_size() for v in host.values()) + g_h.numel() * 8 + l_h.numel() * 8
    d2h = g_out.numel() * 8 + l_out.numel() * 8
    ctx2 = binding.Context()
    e2e_ms = []
    for i in range(max(1, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in host:
            ddev[k].copy_(host[k], non_blocking=True)
        g2.copy_(g_h, non_blocking=True)
        l2.copy_(l_h, non_blocking=True)
        ctx2.assemble(ddev, scene.floor_z, scene.gravity, scene.dt, scene.delta, scene.mu, 3)
        st2 = ctx2.state(g2, l2)
        for _ in range(args.window):
            ctx2.pdip_step(st2, opts, allow=ok)
        g_out.copy_(g2, non_blocking=True)
        l_out.copy_(l2, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_ms_max = max_over_ranks(statistics.median(e2e_ms), world)

    apply_out = n_apply_leg(binding, ctx, st, Nc, M, P, flush, stream, args.apply_reps) if args.apply_reps > 0 else None
    ts_out = time_stepping_leg(args, binding, workload, scene, opts, ok, flush, stream) if args.ts_steps > 0 else None
    batch_out = batched_leg(args, binding, workload) if args.batch_scenes > 0 else None
    learned_out = learned_leg(args, binding, workload) if args.learned_steps > 0 else None
    if learned_out is not None:
        learned_out["network_at_bench_scale"] = mpnn_scale_leg(binding, workload, scene, flush, stream)
    box_out = box_leg(args, binding, workload, flush, stream) if args.box_steps > 0 else None
    dense_out = qtt_dense_leg(binding, flush, stream) if args.qtt_dense else None
    configs_out = None
    if args.config_legs:
        cpu_ok = rank == 0 and not args.no_cpu_baseline
        configs_out = {
            "pile8_fp64": config_leg(binding, workload, "pile8", 1e-10, args.window, [(1e-2, 10)], flush, stream,
                                     cpu=cpu_ok),
            "stack16_pdip_to_gap": stack_leg(binding, workload, flush, stream, cpu=cpu_ok),
            "pile20_fp64_qtt": config_leg(binding, workload, "pile20", 1e-8, 4, [(1e-3, 64), (1e-2, 10)], flush,
                                          stream, reps=2, cpu=cpu_ok),
        }

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if mixed else "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "contacts": Nc, "bodies": M,
                   "padded_unknowns": P, "precond": args.precond, "newton_tol": 1e-8,
                   "solver": "PCG, FP32 inner + FP64 refinement" if mixed else "PCG FP64",
                   "pdip_iterates": f"each step: cold start, then PDIP iterations 0..{args.window - 1}",
                   "newton_solves_per_step": args.window,
                   "l2": "flushed (512 MiB write) before every timed step", "parallelism": f"replicas x{world}"},
        "newton_solves_converged": solved, "newton_solves_attempted": args.steps * args.window,
        "pdip_steps_per_s": pdip_steps_per_s, "pdip_step_status_counts": status_counts,
        "krylov_iters_per_solve": statistics.mean(iters), "refinements_per_solve": statistics.mean(outer),
        "max_rel_res": max(relres), "pcg_ms_per_solve": statistics.mean(pcg_ms),
        "qtt_refresh_ms_per_step": statistics.mean(refresh_ms) if qtt else None,
        "roofline": {"kernel": "k_pcg (persistent PCG)", "bound": "hbm", "achieved": ach, "peak": peak,
                     "unit": "GB/s", "frac": ach / peak, "peak_source": src,
                     "traffic": KPCG_DRAM_BYTES_PER_LAUNCH if args.workload == "pile40p" else None,
                     "traffic_unit": "bytes per launch (one Newton solve)"},
        "qtt_pcg": qtt_out,
        "n_apply": apply_out,
        "e2e": {"value": args.window * 1e3 / e2e_ms_max * world, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "time_stepping": ts_out,
        "batched": batch_out,
        "learned_warm_start": learned_out,
        "configs": configs_out,
        "box_time_stepping": box_out,
        "qtt_apply_rank64": dense_out,
    }
    if rank == 0 and not args.no_cpu_baseline:
        its = gpu_window_iterates(ctx, st, gamma, lam, opts, args.window, ok, Nc)
        sample = list(range(1, args.window, 2)) if args.workload == "pile40p" else list(range(args.window))
        out["cpu_baseline"] = cpu_baseline(scene, its, sample)
        if args.cpu_all_cores:
            out["cpu_baseline_all_cores"] = cpu_baseline_all_cores(args.workload, its, sample)
    ctx2.close()
    ctx.close()
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


FP64_TFLOPS_NOMINAL = 1.25  # GB300 FP64 (nominal; no measured figure)


def n_apply_leg(binding, ctx, st, Nc, M, P, flush, stream, reps=20):
    """The standalone operator apply y = S x (newton_apply, one fused launch) on
    the bench's scene, FP64 and FP32, with and without the PDIP state, L2 flushed
    before every timed call.  Algorithmic bytes (vb = 8 or 4 bytes per value):
    per contact x 3 vb + y 3 vb + frame 6 vb (n and t1; t2 = n x t1) + arms 6 vb
    = 18 vb, ids 8 B and incidence codes 8 B; with the state, gamma 24 B and
    lambda 16 B (FP64; the 3x3 block is formed in registers, never stored); per
    body 1/m and 1/I 2 vb and its CSR offset 4 B (the body intermediate stays in
    shared memory).  Pad
    rows are excluded.  Flops: 33 per incidence (two per contact), 47 per contact
    in the contact pass, 6 per body, and 45 per contact for forming and applying
    the block.  The bound is HBM when flop/byte is below the ridge of the dtype's
    ALU peak over the measured HBM peak (FP32: 80.5 TFLOP/s derived; FP64: 1.25
    TFLOP/s nominal), else that ALU peak."""
    import torch

    hbm, src = peaks()
    out = {}
    for name, dt, vb in (("f64", binding.QP_F64, 8), ("f32", binding.QP_F32, 4)):
        tdt = torch.float64 if vb == 8 else torch.float32
        alu = FP64_TFLOPS_NOMINAL if vb == 8 else FP32_ALU_TFLOPS
        alu_src = "nominal" if vb == 8 else "derived: 152 SM x 128 FP32 x 2 x 2.07 GHz"
        x = torch.randn(P, dtype=tdt, device="cuda")
        y = torch.empty_like(x)
        for with_state in (False, True):
            s_ = st if with_state else None
            for _ in range(3):
                ctx.newton_apply(s_, x, y, dt)
            ms = []
            for _ in range(reps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.newton_apply(s_, x, y, dt)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            per_c = 18 * vb + 16 + (40 if with_state else 0)
            # FP32: one launch, w stays in shared memory; FP64: two launches, w (6 values
            # per body) is written by the gather and read back by the contact pass
            nbytes = Nc * per_c + M * (2 * vb + 4 + (12 * vb if vb == 8 else 0))
            flops = Nc * (2 * 33 + 47 + (45 if with_state else 0)) + M * 6
            t = statistics.median(ms) / 1e3
            if flops / nbytes < alu * 1e12 / (hbm * 1e9):
                roof = {"bound": "hbm", "achieved": nbytes / t / 1e9, "peak": hbm, "unit": "GB/s",
                        "frac": nbytes / t / 1e9 / hbm, "peak_source": src}
            else:
                roof = {"bound": "alu", "achieved": flops / t / 1e12, "peak": alu, "unit": "TFLOP/s",
                        "frac": flops / t / 1e12 / alu, "peak_source": alu_src}
            key = name + ("_with_state" if with_state else "")
            out[key] = {"us": t * 1e6, "bytes": nbytes, "flops": flops, "launches": 2 if vb == 8 else 1,
                        "gbs": nbytes / t / 1e9, "roofline": roof}
    out["note"] = ("median of %d calls, L2 flushed before each; FP32 one fused launch, FP64 two (body "
                   "gather, contact pass); with_state forms each contact's Schur block from (gamma, lambda) in "
                   "registers" % reps)
    return out


def config_leg(binding, workload, name, tol, window, qtt_variants, flush, stream, reps=3, cpu=True):
    """One of the smaller configurations, FP64 throughout: `window` PDIP
    iterations from the cold start solved with Jacobi-PCG to `tol`, then with the
    QTT-preconditioned PCG for each (eps, rmax) in `qtt_variants` (S compressed
    and inverted at every Newton iteration, the inverse warm-started from the
    previous one, Sec. 3.3), each against the same iterates; plus the oracle's
    PDIP iteration on the GPU window's own iterates (one host core)."""
    import torch

    from synth import scene_for

    scene = scene_for(name, 1)
    ctx = binding.Context()
    _, con = workload.assemble(ctx, scene)
    g = torch.zeros(con.P, dtype=torch.float64, device="cuda")
    lam = torch.zeros(2 * con.Nc, dtype=torch.float64, device="cuda")
    st = ctx.state(g, lam)
    ok = (binding.QP_NOT_CONVERGED, binding.QP_LINESEARCH_FAIL)

    def timed(opts, n):
        ms, rec = [], []
        for _ in range(n):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            one = []
            e0.record(stream)
            ctx.pdip_init(st, 1.0)
            for _ in range(window):
                one.append(ctx.pdip_step(st, opts, allow=ok))
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            rec += one
        conv = sum(1 for r in rec if r.solve.status == binding.QP_OK and r.solve.rel_res <= tol)
        return conv / (sum(ms) / 1e3), rec, ms

    jo = ctx.pdip_opts(ctx.solve_opts(tol=tol, maxit=200000))
    timed(jo, 1)
    jv, jrec, jms = timed(jo, reps)
    out = {"workload": f"{name}: {WORKLOADS[name]}", "contacts": con.Nc, "padded_unknowns": con.P, "dtype": "f64",
           "newton_tol": tol, "pdip_iterates": f"cold start, then PDIP iterations 0..{window - 1}",
           "jacobi_pcg": {"value": jv, "unit": UNIT, "ms_per_window": statistics.mean(jms),
                          "krylov_iters_per_solve": statistics.mean(r.solve.iters for r in jrec)},
           "qtt_pcg": []}
    for eps, rmax in qtt_variants:
        so = ctx.solve_opts(binding.QP_QTT_PCG, None, tol=tol, maxit=20000)
        qo = ctx.pdip_opts(so, qtt_refresh=1, qtt_eps=eps, qtt_rmax=rmax)
        timed(qo, 1)
        qv, qrec, qms = timed(qo, 1)
        ro = ctx.pdip_opts(so, qtt_refresh=0)
        # re-use across Newton iterations: refresh at the first iteration only
        ctx.pdip_init(st, 1.0)
        rr = []
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(window):
            rr.append(ctx.pdip_step(st, qo if i == 0 else ro, allow=ok))
        e1.record(stream)
        e1.synchronize()
        rms = e0.elapsed_time(e1)
        rconv = sum(1 for r in rr if r.solve.status == binding.QP_OK and r.solve.rel_res <= tol)
        out["qtt_pcg"].append({
            "eps": eps, "rmax": rmax, "value": qv, "unit": UNIT, "factor_vs_jacobi": qv / jv,
            "refresh_ms": statistics.mean(r.ms_refresh for r in qrec),
            "solve_ms": statistics.mean(r.solve.ms for r in qrec),
            "solve_only_factor_vs_jacobi": statistics.mean(r.solve.ms for r in jrec) / statistics.mean(
                r.solve.ms for r in qrec),
            "krylov_iters_per_solve": statistics.mean(r.solve.iters for r in qrec),
            "jacobi_fallbacks": sum(r.solve.fallback for r in qrec),
            "refresh_once_per_window": {"value": rconv / (rms / 1e3), "factor_vs_jacobi": rconv / (rms / 1e3) / jv,
                                        "krylov_iters_per_solve": statistics.mean(r.solve.iters for r in rr)}})
    if cpu:
        its = gpu_window_iterates(ctx, st, g, lam, jo, window, ok, con.Nc)
        out["cpu_baseline"] = cpu_baseline(scene, its, list(range(window)), tol)
    ctx.close()
    return out


def stack_leg(binding, workload, flush, stream, cpu=True):
    """PDIP to convergence (gap 1e-8 and dual residual 1e-8, Sec. 2.4) on 16 x 16
    columns of 10 spheres (2560 contacts, 2^13), where every contact carries load
    and the method converges: FP64 Jacobi-PCG Newton solves to 1e-10."""
    import torch

    from synth import scene_for

    scene = scene_for("stack16", 1)
    ctx = binding.Context()
    _, con = workload.assemble(ctx, scene)
    g = torch.zeros(con.P, dtype=torch.float64, device="cuda")
    lam = torch.zeros(2 * con.Nc, dtype=torch.float64, device="cuda")
    st = ctx.state(g, lam)
    opts = ctx.pdip_opts(ctx.solve_opts(tol=1e-10, maxit=200000))
    ms, n, stats = [], 0, None
    for rep in range(4):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.pdip_init(st, 1.0)
        stats, n = ctx.pdip_solve(st, opts, gap_tol=1e-8, dual_tol=1e-8, max_iter=200)
        e1.record(stream)
        e1.synchronize()
        if rep:
            ms.append(e0.elapsed_time(e1))
    out = {"workload": "stack16: 16x16 columns of 10 spheres, r=0.5, mu=0.5, dt=1e-3, 2^13 padded unknowns",
           "contacts": con.Nc, "converged": stats.status == binding.QP_OK, "pdip_iterations": n,
           "eta": stats.eta, "r_dual": stats.r_dual, "ms_per_pdip_solve": statistics.mean(ms),
           "pdip_solves_per_s": 1e3 / statistics.mean(ms), "newton_solves_per_s": n * 1e3 / statistics.mean(ms)}
    ctx.close()
    if cpu:
        from oracle import krylov, pdip

        c_o, N, r = oracle_data(scene)

        def solver(S, b):
            x, info = krylov.jacobi_pcg(S, b, tol=1e-10, maxit=100000)
            return x, info["iters"]

        t0 = time.perf_counter()
        res = pdip.pdip_solve(N, r, scene.mu, tol_gap=1e-8, tol_dual=1e-8, maxit=200, newton_solver=solver)
        el = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": 1.0 / el, "unit": "PDIP solves/s", "cores": 1, "kind": "oracle",
                               "newton_solves_per_s": res.iters / el,
                               "sample": f"oracle FP64 PDIP loop with Jacobi-PCG to 1e-10, {res.iters} iterations, "
                                         f"converged={res.converged}, {el:.1f} s"}
    return out


def learned_leg(args, binding, workload):
    """Learned warm start: the network is trained on the converged PDIP solutions
    (gap and dual residual 1e-8) that the library itself computes for 16 x 16 x
    10 column scenes of seeds 2..9, then starts the PDIP of unseen seeds (1, 10,
    11), with the cold start as the fallback (restart from the cold start when
    the PDIP from the learned start has not converged within the training
    scenes' largest cold-start count).  Reported per unseen scene: PDIP
    iterations and device time to convergence from the cold and from the
    learned start (network inference included)."""
    import torch

    from paper_1808_02558_gb300 import learned
    from synth import scene_for

    scale = [1.0, 1.0, 1.0, 0.05, 0.05, 0.05, 0.05, 2.0]
    stream = torch.cuda.current_stream()

    def system(seed):
        sc = scene_for("stack16", seed)
        c = binding.Context()
        _, con = workload.assemble(c, sc)
        g = torch.zeros(con.P, dtype=torch.float64, device="cuda")
        lam = torch.zeros(2 * con.Nc, dtype=torch.float64, device="cuda")
        rows = (3 * torch.arange(con.Nc, device="cuda")[:, None] + torch.arange(3, device="cuda")[None, :]).reshape(-1)
        return c, con, g, lam, c.state(g, lam), rows

    def cold(c, st):
        opts = c.pdip_opts(c.solve_opts(tol=1e-10, maxit=200000))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c.pdip_init(st, 1.0)
        stats, n = c.pdip_solve(st, opts, gap_tol=1e-8, dual_tol=1e-8, max_iter=200)
        e1.record(stream)
        e1.synchronize()
        return opts, n, stats, e0.elapsed_time(e1)

    train, cold_its = [], []
    for seed in range(2, 10):
        c, con, g, lam, st, rows = system(seed)
        _, n, stats, _ = cold(c, st)
        cold_its.append(n)
        train.append((c, g[rows].clone()))
    out_scale = float(torch.cat([t[0::3] for _, t in train]).mean())
    net = learned.WarmStartNet(11, scale, out_scale)
    t0 = time.perf_counter()
    losses = []
    for _ in range(args.learned_steps):
        for c, t in train:
            losses.append(net.train_step(c, t, 1e-3))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    evals = []
    for seed in (1, 10, 11):
        c, con, g, lam, st, rows = system(seed)
        opts, n_cold, s_cold, ms_cold = cold(c, st)
        g_cold = g[rows].clone()
        cold(c, st)  # warm-up of the timed pair
        _, n_cold, s_cold, ms_cold = cold(c, st)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        used, n_l, s_l = net.solve(c, st, con.Nc, opts, gn_min=1e-3 * out_scale, cap=max(cold_its))
        e1.record(stream)
        e1.synchronize()
        dev = float(((g[rows] - g_cold).abs() / g_cold.abs().clamp_min(1e-300)).max())
        evals.append({"seed": seed, "cold_iters": n_cold, "cold_ms": ms_cold, "learned_iters": n_l,
                      "learned_ms": e0.elapsed_time(e1), "start_used": used,
                      "converged": s_l.status == binding.QP_OK, "eta": s_l.eta, "r_dual": s_l.r_dual,
                      "max_rel_impulse_diff_vs_cold": dev})
        c.close()
    for c, _ in train:
        c.close()
    return {"train": {"scenes": "stack16 seeds 2..9", "targets": "converged PDIP solutions (gap, dual 1e-8)",
                      "steps": len(losses), "first_loss": losses[0], "final_loss": losses[-1],
                      "seconds": t_train, "out_scale": out_scale, "cold_iters": cold_its},
            "eval": evals,
            "iters_saved_mean": statistics.mean(e["cold_iters"] - e["learned_iters"] for e in evals),
            "speedup_mean": statistics.mean(e["cold_ms"] / e["learned_ms"] for e in evals)}


def mpnn_scale_leg(binding, workload, scene, flush, stream, reps=10):
    """The warm-start network on the bench's scene (the 40^3 pile, 191 806
    contacts): one forward pass and one gradient (forward + backward), device
    time with the L2 flushed before each call.  The three hidden layers are
    Nc x 128 by 128 x 64 products on the tensor cores (tcgen05, split TF32), the
    backward's input gradients Nc x 64 by 64 x 128 likewise; flops counted are
    those of the dense layers (2 Nc K J per product)."""
    import torch

    from paper_1808_02558_gb300 import learned

    ctx = binding.Context()
    _, con = workload.assemble(ctx, scene)
    Nc = con.Nc
    params = learned.init_params(5)
    scale = [1.0, 1.0, 1.0, 0.05, 5.0, 5.0, 5.0, 2.0]
    out = torch.empty(3 * Nc, dtype=torch.float32, device="cuda")
    grad = torch.empty_like(params)
    target = torch.randn(3 * Nc, dtype=torch.float32, device="cuda")

    def timed(fn):
        fn()
        ms = []
        for _ in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    f_ms = timed(lambda: ctx.mpnn_forward(params, scale, out))
    g_ms = timed(lambda: ctx.mpnn_grad(params, scale, target, grad))
    dense_f = 2 * Nc * (8 * 64 + 3 * 128 * 64 + 64 * 3)
    dense_g = dense_f + 2 * Nc * (3 * 2 * 128 * 64 + 64 * 8 + 2 * 64 * 3)
    ctx.close()
    return {"contacts": Nc, "forward_ms": f_ms, "grad_ms": g_ms, "forward_dense_flops": dense_f,
            "grad_dense_flops": dense_g, "forward_tflops": dense_f / f_ms / 1e9, "grad_tflops": dense_g / g_ms / 1e9,
            "note": "median of %d calls each, L2 flushed before each; times include the message passing, "
                    "the small input/output layers and (grad) the loss read-back" % reps}


def batched_leg(args, binding, workload):
    """Many small scenes (sides U{4..16}, mu U[0.2, 0.8], seeded): the Newton system
    at the cold start of each, solved to 1e-8 by one launch over the scene table
    (clusters of two thread blocks: a large scene on both, small scenes one per block),
    by the same launch with one block per scene, and by one newton_solve per scene."""
    import torch

    from synth import lattice_scene, splitmix64_uniform

    n = args.batch_scenes
    u = splitmix64_uniform(7, 31, 2 * n)
    sides = [4 + min(12, int(x * 13)) for x in u[:n]]
    mus = [0.2 + 0.6 * x for x in u[n:]]
    ctxs, states, rhs, dx, keep = [], [], [], [], []
    nc_tot, p_tot = 0, 0
    for i in range(n):
        sc = lattice_scene(sides[i], 100 + i, mu=mus[i])
        c = binding.Context()
        _, con = workload.assemble(c, sc)
        g = torch.zeros(con.P, dtype=torch.float64, device="cuda")
        lam = torch.zeros(2 * con.Nc, dtype=torch.float64, device="cuda")
        st = c.state(g, lam)
        c.pdip_init(st, 1.0)
        r = torch.empty(con.P, dtype=torch.float64, device="cuda")
        c.newton_rhs(st, r)
        ctxs.append(c)
        states.append(st)
        rhs.append(r)
        dx.append(torch.empty_like(r))
        keep.append((g, lam, con.Nc, con.M, con.P))
        nc_tot += con.Nc
        p_tot += con.P
    torch.cuda.synchronize()
    kw = dict(tol=1e-8, maxit=100000, inner_tol=1e-3, max_outer=60)
    stats, used = binding.newton_solve_batched(ctxs, states, rhs, dx, block_threads=0, **kw)  # measures the block size
    t_b = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        stats, used = binding.newton_solve_batched(ctxs, states, rhs, dx, block_threads=used, **kw)
        t_b.append(time.perf_counter() - t0)
    so = [c.solve_opts(tol=1e-8, maxit=100000, mixed=1, inner_tol=1e-3, max_outer=60) for c in ctxs]
    one = [torch.empty_like(r) for r in rhs]
    for c, st, r, x, o in zip(ctxs, states, rhs, one, so):  # warm-up pass
        c.newton_solve(st, r, x, o)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c, st, r, x, o in zip(ctxs, states, rhs, one, so):
        c.newton_solve(st, r, x, o)
    torch.cuda.synchronize()
    t_s = time.perf_counter() - t0
    tb = statistics.median(t_b)
    # the same batch with one block per scene (no scene split over a cluster)
    _, used1 = binding.newton_solve_batched(ctxs, states, rhs, dx, block_threads=0, split=1, **kw)
    s1, _ = binding.newton_solve_batched(ctxs, states, rhs, dx, block_threads=used1, split=1, **kw)
    plan = binding.newton_batch_plan([k[4] + k[2] for k in keep], torch.cuda.get_device_properties(0).multi_processor_count)
    # algorithmic bytes of all solves (same per-scene count as the single-scene kernel)
    nbytes = sum(solve_bytes(k[2], k[3], 3 * k[2], s.iters, s.outer) for k, s in zip(keep, stats))
    hbm, src = peaks()
    ach = nbytes / (stats[0].ms / 1e3) / 1e9
    out = {"scenes": n, "sides": "U{4..16}", "mu": "U[0.2, 0.8]", "contacts": nc_tot, "padded_unknowns": p_tot,
           "block_threads": used, "tol": 1e-8, "batched_ms": tb * 1e3, "batched_device_ms": stats[0].ms,
           "scenes_on_two_blocks": sum(1 for _, b in plan if b == -2), "clusters": len(plan),
           "one_block_per_scene_device_ms": s1[0].ms, "one_block_per_scene_threads": used1,
           "batched_solves_per_s": n / tb, "sequential_ms": t_s * 1e3, "sequential_solves_per_s": n / t_s,
           "speedup": t_s / tb, "max_rel_res": max(s.rel_res for s in stats),
           "not_converged": sum(1 for s in stats if s.status != binding.QP_OK),
           "iters_mean": statistics.mean(s.iters for s in stats),
           "roofline": {"kernel": "k_pcg_batched", "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                        "frac": ach / hbm, "peak_source": src, "bytes": nbytes,
                        "time": "device time of the launch (events)"}}
    # every scene with its own QTT preconditioner: the inverse of its Jacobi-scaled
    # Schur matrix at the paper's operating point (eps 1e-2, r <= 10), BF16 cores,
    # the tile shapes from the measured table
    t0 = time.perf_counter()
    X = []
    for c, st in zip(ctxs, states):
        S_tt = c.qtt_compress(st, 1e-2, 10)
        X.append(c.qtt_inverse(S_tt, 1e-2, 10, sweeps=2))
        S_tt.free()
    torch.cuda.synchronize()
    t_refresh = time.perf_counter() - t0
    qkw = dict(kw, precond=X, core_dtype=binding.QP_BF16, allow=(binding.QP_NOT_CONVERGED, binding.QP_BREAKDOWN))
    qs, qused = binding.newton_solve_batched(ctxs, states, rhs, dx, block_threads=0, **qkw)
    t_q = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        qs, qused = binding.newton_solve_batched(ctxs, states, rhs, dx, block_threads=qused, **qkw)
        t_q.append(time.perf_counter() - t0)
    fixed = {}
    for tile in (1, 2):
        fs, _ = binding.newton_solve_batched(ctxs, states, rhs, dx, block_threads=qused, qtt_tile=tile, **qkw)
        fixed[f"tile_{tile}_device_ms"] = fs[0].ms
    out["qtt"] = {"eps": 1e-2, "rmax": 10, "core_dtype": "bf16", "block_threads": qused,
                  "tiles_measured": ctxs[0].batch_qtt_tiles(qused), "batched_ms": statistics.median(t_q) * 1e3,
                  "batched_device_ms": qs[0].ms, "batched_solves_per_s": n / statistics.median(t_q),
                  "factor_vs_jacobi_batched": tb / statistics.median(t_q),
                  "iters_mean": statistics.mean(s.iters for s in qs),
                  "converged": sum(1 for s in qs if s.status == binding.QP_OK),
                  "max_rel_res": max(s.rel_res for s in qs), "refresh_s_all_scenes": t_refresh, **fixed,
                  "note": "tiles_measured: column items per thread for input ranks <= 4, <= 8, <= 16, above"}
    for x in X:
        x.free()
    for c in ctxs:
        c.close()
    return out


def time_stepping_leg(args, binding, workload, scene, opts, ok, flush, stream):
    """Time steps of the scene (Sec. 2.3): assemble, PDIP init (cold at the first
    step, warm from the persisting contacts after), a window of PDIP iterations,
    advance.  Reports the time per step and its parts, the fraction of contacts
    that persist, and, at every warm-started step, the surrogate gap and dual
    residual after the window against a cold start of the same system."""
    import torch

    ctx = binding.Context()
    dev_s = workload.scene_to_device(scene, "cuda")
    rows, prev = [], None
    for step in range(args.ts_steps):
        dev_before = {k: v.clone() for k, v in dev_s.items()}  # this step's scene (for the fresh-context refresh)
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        con = ctx.assemble(dev_s, scene.floor_z, scene.gravity, scene.dt, scene.delta, scene.mu, 3)
        ev[1].record(stream)
        g = torch.zeros(con.P, dtype=torch.float64, device="cuda")
        lam = torch.zeros(2 * con.Nc, dtype=torch.float64, device="cuda")
        st = ctx.state(g, lam)
        if prev is None:
            ctx.pdip_init(st, 1.0)
        else:
            ctx.pdip_init_warm(st, prev[0], prev[1], prev[2], 3)
        for _ in range(args.window):
            ctx.pdip_step(st, opts, allow=ok)
        ev[2].record(stream)
        ab = (workload.view(con, "body_a"), workload.view(con, "body_b"))
        eta, rd = ctx.pdip_measure(st)
        cold = None
        if prev is not None:
            # the same system from the cold start, for comparison (not timed)
            g2 = torch.zeros_like(g)
            l2 = torch.zeros_like(lam)
            st2 = ctx.state(g2, l2)
            ctx.pdip_init(st2, 1.0)
            for _ in range(args.window):
                ctx.pdip_step(st2, opts, allow=ok)
            cold = ctx.pdip_measure(st2)
        ev3 = torch.cuda.Event(enable_timing=True)
        ev3.record(stream)
        ctx.advance(st)
        ev[3].record(stream)
        ev[3].synchronize()
        keys = set(zip(ab[0].tolist(), ab[1].tolist()))
        persist = None if prev is None else len(keys & prev[3]) / max(1, len(keys))
        # QTT refresh of the first Newton system of the step (compress + invert):
        # warm-started by the previous step's inverse in this context, and from
        # scratch in a fresh context (the reuse speed-up across time steps)
        qtt_ms = None
        if args.ts_qtt:
            def refresh_ms(c):
                g3 = torch.zeros_like(g)
                l3 = torch.zeros_like(lam)
                s3 = c.state(g3, l3)
                c.pdip_init(s3, 1.0)
                so = c.solve_opts(binding.QP_QTT_PCG, None, tol=1e-8, maxit=args.qtt_maxit, mixed=1,
                                  inner_tol=1e-3, max_outer=60, core_dtype=binding.QP_BF16)
                po = c.pdip_opts(so, qtt_refresh=1, qtt_eps=args.qtt_eps, qtt_rmax=args.qtt_rmax)
                return c.pdip_step(s3, po, allow=ok).ms_refresh
            warm_ms = refresh_ms(ctx)
            fresh = binding.Context()
            fresh.assemble(dev_before, scene.floor_z, scene.gravity, scene.dt, scene.delta, scene.mu, 3)
            cold_ms = refresh_ms(fresh)
            fresh.close()
            qtt_ms = {"refresh_ms_reusing_previous": warm_ms if step > 0 else None, "refresh_ms_from_scratch": cold_ms}
        rows.append({"step": step, "contacts": con.Nc, "persisting": persist,
                     "ms_assemble": ev[0].elapsed_time(ev[1]), "ms_pdip_window": ev[1].elapsed_time(ev[2]),
                     "ms_advance": ev3.elapsed_time(ev[3]), "eta": eta, "r_dual": rd,
                     "cold_eta": None if cold is None else cold[0], "cold_r_dual": None if cold is None else cold[1],
                     "qtt": qtt_ms})
        prev = (ab[0], ab[1], g.clone(), keys)
    ctx.close()
    ms = [r["ms_assemble"] + r["ms_pdip_window"] + r["ms_advance"] for r in rows]
    return {"steps": args.ts_steps, "pdip_iterations_per_step": args.window,
            "ms_per_time_step": sum(ms) / len(ms), "per_step": rows,
            "note": "Jacobi-PCG windows; warm start = previous impulses of persisting pairs moved into the cone"}


def qtt_dense_leg(binding, flush, stream, reps=10):
    """QTT apply at rank cap 64 (d = 20: 2^20 unknowns, ranks min(64, 4^k,
    4^(d-k)), BF16 cores, FP32 vectors), the profile of a Schur inverse
    compressed at eps 1e-3, r <= 64: the CUDA-core steps against the tensor-core
    steps (tcgen05, split TF32) of the dense cores.  Bytes: each core's pass
    reads r_k N and writes r_{k-1} N FP32 values; flops 4 r_{k-1} r_k N per core
    (N/2 column items, each a (2 r_{k-1}) x (2 r_k) matrix-vector product)."""
    import numpy as np
    import torch

    d, N = 20, 1 << 20
    ranks = [min(64, 4 ** min(k, d - k)) for k in range(d + 1)]
    rng = np.random.default_rng(7)
    cores = [rng.standard_normal((ranks[k], 4, ranks[k + 1])) / np.sqrt(2 * ranks[k + 1]) for k in range(d)]
    ctx = binding.Context()
    A = ctx.qtt_from_cores(cores)
    x = torch.randn(N, dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    nbytes = sum((ranks[k] + ranks[k + 1]) * N * 4 for k in range(d))
    flops = sum(4 * ranks[k] * ranks[k + 1] * N for k in range(d))
    dense = [k + 1 for k in range(d) if ranks[k] * ranks[k + 1] >= 512]
    dense_bytes = sum((ranks[k - 1] + ranks[k]) * N * 4 for k in dense)
    out = {"d": d, "ranks": ranks, "core_dtype": "bf16", "bytes": nbytes, "flops": flops,
           "tensor_core_cores": len(dense), "tensor_core_bytes": dense_bytes}
    hbm, src = peaks()
    for mode, name in ((0, "cuda_cores"), (1, "tensor_cores")):
        ctx.qtt_set_tensor_cores(mode)
        for _ in range(3):
            ctx.qtt_apply(A, x, y, binding.QP_BF16, binding.QP_F32)
        ms = []
        for _ in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.qtt_apply(A, x, y, binding.QP_BF16, binding.QP_F32)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        t = statistics.median(ms) / 1e3
        out[name] = {"us": t * 1e6, "gbs": nbytes / t / 1e9, "hbm_frac": nbytes / t / 1e9 / hbm,
                     "tflops": flops / t / 1e12, "fp32_alu_frac": flops / t / 1e12 / FP32_ALU_TFLOPS}
    out["speedup"] = out["cuda_cores"]["us"] / out["tensor_cores"]["us"]
    out["peak_source"] = src
    A.free()
    ctx.close()
    return out


def box_leg(args, binding, workload, flush, stream):
    """Time stepping of 64 000 polydisperse spheres falling in the walled 40 x 40
    x 80 box (Sec. 2.3), args.box_steps steps of seed 1.  A step: assemble (pairs,
    floor, side walls), start the PDIP from the previous step's impulses on the
    persisting pairs (cold at the first step), args.box_window PDIP iterations
    with mixed-precision Jacobi-PCG Newton solves at 1e-8, advance.  Alongside,
    outside the step time:
    * QTT reuse across steps (Sec. 3.3): the inverse of every step's first Newton
      system is refreshed (compressed, then inverted warm-started from the
      previous step's inverse) and used by one QTT-PCG solve; every 25th step
      the same refresh and solve run from scratch in a fresh context;
    * learned start: the network is trained on the window solutions of the
      first args.box_train_steps steps of seeds 2 and 3 and, every 10th step of
      seed 1, starts the same window, compared with the cold start and with the
      warm start of the trajectory (gap and dual residual after the window)."""
    import torch

    from paper_1808_02558_gb300 import learned
    from synth import scene_for

    ok = (binding.QP_NOT_CONVERGED, binding.QP_LINESEARCH_FAIL)
    W = args.box_window
    scale = [1.0, 1.0, 1.0, 0.05, 0.05, 0.05, 0.05, 2.0]

    def opts_for(c):
        return c.pdip_opts(c.solve_opts(tol=1e-8, maxit=200000, mixed=1, inner_tol=1e-3, max_outer=60))

    def qtt_opts(c):
        so = c.solve_opts(binding.QP_QTT_PCG, None, tol=1e-8, maxit=args.qtt_maxit, mixed=1, inner_tol=1e-3,
                          max_outer=60, core_dtype=binding.QP_BF16)
        return c.pdip_opts(so, qtt_refresh=1, qtt_eps=args.qtt_eps, qtt_rmax=args.qtt_rmax)

    def fresh_state(con):
        g = torch.zeros(con.P, dtype=torch.float64, device="cuda")
        lam = torch.zeros(2 * con.Nc, dtype=torch.float64, device="cuda")
        return g, lam, binding.Context.state(g, lam)

    def trajectory(seed, steps, hook=None, timed=False):
        sc = scene_for("box40", seed)
        ctx = binding.Context()
        dev_s = workload.scene_to_device(sc, "cuda")
        opts = opts_for(ctx)
        prev, rows = None, []
        for step in range(steps):
            dev_before = {k: v.clone() for k, v in dev_s.items()} if hook else None
            if timed:
                flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(stream)
            con = ctx.assemble(dev_s, sc.floor_z, sc.gravity, sc.dt, sc.delta, sc.mu, 3, sc.walls)
            ev[1].record(stream)
            g, lam, st = fresh_state(con)
            if prev is None:
                ctx.pdip_init(st, 1.0)
            else:
                ctx.pdip_init_warm(st, prev[0], prev[1], prev[2], 3, prev_plane=prev[4])
            stats = [ctx.pdip_step(st, opts, allow=ok) for _ in range(W)]
            ev[2].record(stream)
            ab = (workload.view(con, "body_a"), workload.view(con, "body_b"), workload.view(con, "plane"))
            eta, rd = ctx.pdip_measure(st)
            side = hook(step, ctx, con, g, dev_before, sc) if hook else None
            ev[3].record(stream)
            ctx.advance(st)
            ev4 = torch.cuda.Event(enable_timing=True)
            ev4.record(stream)
            ev4.synchronize()
            keys = set(zip(ab[0].tolist(), ab[1].tolist(), ab[2].tolist()))
            rows.append({"step": step, "contacts": con.Nc, "padded_unknowns": con.P,
                         "persisting": None if prev is None else len(keys & prev[3]) / max(1, len(keys)),
                         "ms_assemble": ev[0].elapsed_time(ev[1]), "ms_pdip_window": ev[1].elapsed_time(ev[2]),
                         "ms_advance": ev[3].elapsed_time(ev4), "eta": eta, "r_dual": rd,
                         "pdip_ok": sum(int(s_.status == binding.QP_OK) for s_ in stats),
                         "solves_converged": sum(int(s_.solve.status == binding.QP_OK and s_.solve.rel_res <= 1e-8)
                                                 for s_ in stats),
                         "krylov_iters": statistics.mean(s_.solve.iters for s_ in stats), "side": side})
            prev = (ab[0], ab[1], g.clone(), keys, ab[2])
        return ctx, rows

    # training data: window solutions along the trajectories of seeds 2 and 3
    train = []

    def keep(step, c, con, g, dev_before, sc):
        if step % max(1, args.box_train_steps // 3) == 0:
            tc = binding.Context()
            tcon = tc.assemble(dev_before, sc.floor_z, sc.gravity, sc.dt, sc.delta, sc.mu, 3, sc.walls)
            assert tcon.Nc == con.Nc
            train.append((tc, g[:3 * con.Nc].clone()))
        return None

    t0 = time.perf_counter()
    for seed in (2, 3):
        c, _ = trajectory(seed, args.box_train_steps, keep)
        c.close()
    gn_all = torch.cat([t[0::3] for _, t in train])
    out_scale = max(float(gn_all.mean()), 1e-6)
    net = learned.WarmStartNet(11, scale, out_scale)
    losses = []
    for _ in range(args.box_train_epochs):
        for c, t in train:
            losses.append(net.train_step(c, t, 1e-3))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0

    # seed 1: the timed trajectory, with the QTT and learned-start comparisons beside it
    def side(step, c, con, g, dev_before, sc):
        out = {}
        g3, l3, s3 = fresh_state(con)
        c.pdip_init(s3, 1.0)
        r = c.pdip_step(s3, qtt_opts(c), allow=ok)
        out["qtt_reuse"] = {"refresh_ms": r.ms_refresh, "krylov_iters": r.solve.iters, "solve_ms": r.solve.ms}
        if step % 25 == 0:
            fc = binding.Context()
            fcon = fc.assemble(dev_before, sc.floor_z, sc.gravity, sc.dt, sc.delta, sc.mu, 3, sc.walls)
            g5, l5, s5 = fresh_state(fcon)
            fc.pdip_init(s5, 1.0)
            r5 = fc.pdip_step(s5, qtt_opts(fc), allow=ok)
            out["qtt_scratch"] = {"refresh_ms": r5.ms_refresh, "krylov_iters": r5.solve.iters,
                                  "solve_ms": r5.solve.ms}
            fc.close()
        if step % 10 == 0:
            o = opts_for(c)
            g4, l4, s4 = fresh_state(con)
            c.pdip_init(s4, 1.0)
            for _ in range(W):
                c.pdip_step(s4, o, allow=ok)
            cold = c.pdip_measure(s4)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            net.warm_start(c, s4, con.Nc, gn_min=1e-3 * out_scale)
            e1.record(stream)
            start = c.pdip_measure(s4)
            for _ in range(W):
                c.pdip_step(s4, o, allow=ok)
            learned_end = c.pdip_measure(s4)
            # control: the cold start scaled to the learned start's impulse floor
            # (the targets are near zero, so the network's output is too)
            c.pdip_init(s4, 1e-3 * out_scale)
            for _ in range(W):
                c.pdip_step(s4, o, allow=ok)
            out["starts"] = {"cold": cold, "learned": learned_end, "learned_at_start": start,
                             "cold_scaled_to_learned": c.pdip_measure(s4),
                             "learned_start_ms": e0.elapsed_time(e1)}
        return out

    ctx, rows = trajectory(1, args.box_steps, side, timed=True)
    ctx.close()
    for c, _ in train:
        c.close()
    ms = [r["ms_assemble"] + r["ms_pdip_window"] + r["ms_advance"] for r in rows]
    warm = [r for r in rows if r["step"] > 0]
    reuse = [r["side"]["qtt_reuse"] for r in warm]
    scratch = [r["side"]["qtt_scratch"] for r in rows if "qtt_scratch" in r["side"]]
    starts = [dict(step=r["step"], warm=(r["eta"], r["r_dual"]), **r["side"]["starts"]) for r in rows
              if "starts" in r["side"]]
    steps_total = sum(ms) / 1e3
    return {"scene": "box40 seed 1: 64 000 spheres, radius U[0.4, 0.6], walls x, y = 0, 40, floor z = 0",
            "steps": len(rows), "pdip_iterations_per_step": W,
            "ms_per_time_step": statistics.mean(ms), "time_steps_per_s": len(rows) / steps_total,
            "pdip_steps_per_s": sum(r["pdip_ok"] for r in rows) / steps_total,
            "newton_solves_per_s": sum(r["solves_converged"] for r in rows) / steps_total,
            "ms_assemble": statistics.mean(r["ms_assemble"] for r in rows),
            "ms_pdip_window": statistics.mean(r["ms_pdip_window"] for r in rows),
            "ms_advance": statistics.mean(r["ms_advance"] for r in rows),
            "contacts_first_last": [rows[0]["contacts"], rows[-1]["contacts"]],
            "padded_unknowns": rows[0]["padded_unknowns"],
            "persisting_mean": statistics.mean(r["persisting"] for r in warm) if warm else None,
            "eta_r_dual_first_last": [[rows[0]["eta"], rows[0]["r_dual"]], [rows[-1]["eta"], rows[-1]["r_dual"]]],
            "krylov_iters_per_solve": statistics.mean(r["krylov_iters"] for r in rows),
            "qtt": {"refresh_ms_reusing_previous_step": statistics.mean(x["refresh_ms"] for x in reuse)
                    if reuse else None,
                    "krylov_iters_reusing": statistics.mean(x["krylov_iters"] for x in reuse) if reuse else None,
                    "refresh_ms_from_scratch": statistics.mean(x["refresh_ms"] for x in scratch),
                    "krylov_iters_from_scratch": statistics.mean(x["krylov_iters"] for x in scratch),
                    "eps": args.qtt_eps, "rmax": args.qtt_rmax},
            "learned": {"train": {"scenes": f"box40 seeds 2, 3, window solutions of steps 0..{args.box_train_steps - 1}",
                                  "snapshots": len(train), "epochs": args.box_train_epochs,
                                  "first_loss": losses[0] if losses else None,
                                  "final_loss": losses[-1] if losses else None, "seconds": t_train,
                                  "out_scale": out_scale},
                        "eval": starts},
            "l2": "flushed (512 MiB write) before every step",
            "note": "the step time excludes the QTT and learned-start comparisons run beside it"}


# ---------------------------------------------------------------------- oracle arm
def oracle_data(scene):
    from oracle import contacts as oc, qp

    con = oc.detect(scene)
    D, N, r = qp.qp_data(scene, con)
    return con, N, r


def oracle_pdip_times(scene, iterates, tol=1e-8, data=None):
    """The oracle's PDIP iteration (Sec. 2.4: Schur blocks and rhs, Jacobi-PCG
    Newton solve to `tol`, dlambda, ratio test, backtracking, update) timed at
    each given (gamma, lambda) iterate (compact layout).  Returns a list of
    (seconds, krylov iterations)."""
    from oracle import krylov, pdip

    con, N, r = data or oracle_data(scene)

    def solver(S, b):
        x, info = krylov.jacobi_pcg(S, b, tol=tol, maxit=100000)
        return x, info["iters"]

    out = []
    for g, lam in iterates:
        t0 = time.perf_counter()
        _, _, info = pdip.pdip_step(N, r, scene.mu, g, lam, newton_solver=solver)
        out.append((time.perf_counter() - t0, info.krylov_iters))
    return out


def oracle_window(scene, window, tol=1e-8, data=None):
    """The oracle's own PDIP window: iterates 0..window-1 from the cold start."""
    from oracle import krylov, pdip, qp

    con, N, r = data or oracle_data(scene)

    def solver(S, b):
        x, info = krylov.jacobi_pcg(S, b, tol=tol, maxit=100000)
        return x, info["iters"]

    g, lam = qp.initial_point(con.Nc, scene.mu)
    its = []
    for _ in range(window):
        its.append((g.copy(), lam.copy()))
        g, lam, _ = pdip.pdip_step(N, r, scene.mu, g, lam, newton_solver=solver)
    return its


def gpu_window_iterates(ctx, st, gamma, lam, opts, window, ok, Nc):
    """(gamma, lambda) before each PDIP iteration of one window, in the compact
    layout the oracle uses (read back from the device, untimed)."""
    idx = None
    out = []
    ctx.pdip_init(st, 1.0)
    for _ in range(window):
        g = gamma.cpu().numpy()
        if idx is None:
            import numpy as np

            idx = (3 * np.arange(Nc)[:, None] + np.arange(3)[None, :]).reshape(-1)
        out.append((g[idx].copy(), lam.cpu().numpy().copy()))
        ctx.pdip_step(st, opts, allow=ok)
    return out


def cpu_baseline(scene, iterates, sample, tol=1e-8):
    """The oracle as it stands on one host core: its PDIP iteration at the GPU
    window's own iterates `sample` (indices into `iterates`)."""
    times = oracle_pdip_times(scene, [iterates[i] for i in sample], tol)
    el = sum(t for t, _ in times)
    return {"value": len(times) / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "iterations_per_solve": statistics.mean(k for _, k in times),
            "sample": (f"oracle FP64 PDIP iteration (numpy/scipy, 1 thread; Schur blocks, rhs, Jacobi-PCG to "
                       f"{tol:g}, update) at PDIP iterates {list(sample)} of the GPU's own timed window "
                       f"(read back after timing): {len(times)} iterations in {el:.1f} s, "
                       f"{statistics.mean(k for _, k in times):.0f} CG iterations per solve; one Newton solve "
                       f"per PDIP iteration")}


def _oracle_worker(job):
    """One host core of the all-cores CPU baseline: the oracle's PDIP iteration
    at one iterate, repeated for `seconds`.  Returns (iterations, seconds)."""
    workload, seed, it, tol, seconds = job
    from synth import scene_for

    scene = scene_for(workload, seed=seed)
    data = oracle_data(scene)
    n, t0 = 0, time.perf_counter()
    while True:
        oracle_pdip_times(scene, [it], tol, data)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            return n, el


def cpu_baseline_all_cores(workload, iterates, sample, tol=1e-8, seconds=10.0):
    """The oracle on every host core: one spawned single-thread process per core,
    process i repeating the PDIP iteration at iterate sample[i mod len(sample)];
    the job's rate is the sum of the per-process rates."""
    import concurrent.futures as cf
    import multiprocessing as mp

    cores = os.cpu_count() or 1
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    jobs = [(workload, 1, iterates[sample[i % len(sample)]], tol, seconds) for i in range(cores)]
    try:
        # a worker that dies breaks the executor (an error, not a hang)
        with cf.ProcessPoolExecutor(cores, mp_context=mp.get_context("spawn")) as ex:
            res = list(ex.map(_oracle_worker, jobs))
    except Exception as e:  # reported in the line instead of failing the bench
        return {"value": None, "unit": UNIT, "cores": cores, "kind": "oracle", "error": repr(e)[:200]}
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    rate = sum(n / e for n, e in res)
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"oracle FP64 PDIP iteration (numpy/scipy), {cores} spawned processes of one thread, "
                       f"process i repeating PDIP iterate {list(sample)}[i mod {len(sample)}] of the GPU's window "
                       f"for {seconds:.0f} s ({sum(n for n, _ in res)} iterations in all); rate = sum of "
                       f"per-process iterations/s (one Newton solve each)")}


def run_reference(args):
    """The oracle as it stands, on the host cores, on the benchmark's workload:
    the oracle computes its own PDIP window (iterates 0..window-1 from the cold
    start, untimed set-up); timed step j is the oracle's PDIP iteration at
    iterate j mod window, one Newton solve each, a bounded sample of the GPU
    step's `window` iterations."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from synth import scene_for

    scene = scene_for(args.workload, seed=1)
    tol = 1e-8 if args.workload != "pile8" else 1e-10
    data = oracle_data(scene)
    its = oracle_window(scene, args.window, tol, data)
    times, kry = [], []
    for j in range(args.warmup + args.steps):
        (t, k), = oracle_pdip_times(scene, [its[j % args.window]], tol, data)
        if j >= args.warmup:
            times.append(t)
            kry.append(k)
    per = statistics.mean(times)
    value = 1.0 / per
    sample = (f"oracle FP64 PDIP iteration (numpy/scipy, 1 thread; Schur blocks, rhs, Jacobi-PCG to {tol:g}, "
              f"update) at its own iterates j mod {args.window} of the cold-start window; "
              f"{statistics.mean(kry):.0f} CG iterations per solve")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "precond": "jacobi",
                      "newton_tol": tol,
                      "pdip_iterates": f"PDIP iterations 0..{args.window - 1} from the cold start (the GPU "
                                       f"step's window), one per timed step"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--window", type=int, default=8, help="PDIP iterations (Newton solves) per step")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precond", default="jacobi", choices=["jacobi", "qtt"])
    ap.add_argument("--workload", default="pile40p", choices=list(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-all-cores", type=int, default=1, help="also time the oracle on every host core (0: skip)")
    ap.add_argument("--apply-reps", type=int, default=20, help="timed newton_apply calls per variant (0: skip)")
    ap.add_argument("--qtt-eps", type=float, default=1e-2)
    ap.add_argument("--qtt-rmax", type=int, default=10)
    ap.add_argument("--qtt-steps", type=int, default=1, help="PDIP steps of the QTT-PCG comparison leg (0: skip)")
    ap.add_argument("--ts-steps", type=int, default=3, help="time steps of the time-stepping leg (0: skip)")
    ap.add_argument("--ts-qtt", type=int, default=1, help="time-stepping leg: measure the QTT refresh reuse (0: skip)")
    ap.add_argument("--batch-scenes", type=int, default=256, help="scenes of the batched leg (0: skip)")
    ap.add_argument("--learned-steps", type=int, default=300, help="training epochs of the learned leg (0: skip)")
    ap.add_argument("--box-steps", type=int, default=100, help="time steps of the walled-box leg (0: skip)")
    ap.add_argument("--qtt-dense", type=int, default=1, help="time the rank-64 QTT apply, CUDA vs tensor cores (0: skip)")
    ap.add_argument("--box-window", type=int, default=20, help="walled-box leg: PDIP iterations per time step")
    ap.add_argument("--box-train-steps", type=int, default=30, help="walled-box leg: steps of each training seed")
    ap.add_argument("--box-train-epochs", type=int, default=100, help="walled-box leg: training epochs")
    ap.add_argument("--config-legs", type=int, default=1,
                    help="also run the 8^3 FP64, the columns PDIP-to-gap and the 20^3 FP64 QTT legs (0: skip)")
    ap.add_argument("--qtt-krylov", default="cg", choices=["bicgstab", "cg"],
                    help="Krylov method of the QTT leg (the paper uses BiCGSTAB)")
    ap.add_argument("--qtt-maxit", type=int, default=2000,
                    help="iteration cap of the QTT leg before the Jacobi fallback")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
