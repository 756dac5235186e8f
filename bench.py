#!/usr/bin/env python3
"""Throughput of the implicit LISL HJB solver: grid-point·steps/s at 2049 x 2049, 65 controls.

Workload (the mixed-precision configuration): uncertain-correlation HJB on [-2, 2]^2,
2049 x 2049 nodes, 65 controls rho in [-0.95, 0.95], (s1, s2) ~ U[0.15, 0.4]^2 from seed 0,
dt = 1/128.  A bench step is one implicit time step of the whole hot path: source tables,
Howard policy iteration (FP64 policy decision with an FP32 screen), Galerkin hierarchy
rebuilds, and FP64 iterative refinement around an FP32 BiCGSTAB with an FP32 multigrid
V-cycle.  The W warm-up steps are the first W steps of the 128-step horizon; the K timed
steps continue the march (K = 125 covers the rest of the horizon).  The working set
(about 1 GB of vectors, tables and coarse levels) is far larger than L2, so no flush is
needed between steps.

Output: one JSON line (rank 0).  `value` is the device-timed rate of all ranks together;
`e2e` repeats the measurement through the public API with the state in pinned host memory
(H2D before and D2H after every step); `fp64` times the FP64 path on the same steps and
`mixed_vs_fp64_rel_err` compares the two.  `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SL-HJB grid-point·steps/s at 2049², 65 controls: mixed vs FP64 GPU at 1e-8 rel"
UNIT = "grid-point·steps/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=125)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=2049)
    p.add_argument("--fp64-steps", type=int, default=8)
    p.add_argument("--e2e-steps", type=int, default=-1,
                   help="steps of the end-to-end timing (default: the same steps as the device timing)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-adjoint", action="store_true")
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--no-amg", action="store_true")
    p.add_argument("--no-smoother", action="store_true")
    p.add_argument("--amg-steps", type=int, default=8)
    p.add_argument("--batched-instances", type=int, default=256)
    p.add_argument("--batched-workers", type=int, default=16)
    p.add_argument("--batched-graphs", type=int, default=1, choices=[1, 2],
                   help="graph mode of the batch's handles (sl_opts.use_graphs)")
    p.add_argument("--batched-one-worker", action="store_true",
                   help="also time the batch with a single worker thread (about 25 s)")
    p.add_argument("--adjoint-steps", type=int, default=64,
                   help="steps of 1/64 in the adjoint workload's march (64: T = 1)")
    p.add_argument("--opt", action="append", default=[],
                   help="solver option override key=value (sl_opts field), repeatable")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def traffic_record(kernel: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary (None if absent)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        if line.startswith(kernel + ":"):
            try:
                return float(line.split(":", 1)[1].split()[0])
            except ValueError:
                return None
    return None


# ------------------------------------------------------------------------------- CPU oracle

def oracle_rate(n_sample: int, steps: int, t_start_steps: int = 0):
    """Times the CPU oracle (as it stands) on the same PDE family at n_sample^2."""
    import workloads as W
    from oracle import lisl
    full = W.mixed_2049(seed=0)
    dt = 1.0 / 128
    p = W.manufactured(n_sample, 65, -0.95, 0.95, full.s1, full.s2, T=dt * steps, n_steps=steps)
    t0 = time.perf_counter()
    lisl.solve(p)
    wall = time.perf_counter() - t0
    return n_sample * n_sample * steps / wall, wall


def cpu_baseline_record():
    rate, wall = oracle_rate(257, 1)
    return {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"1 implicit step of the same PDE family on a 257x257 grid (65 controls, "
                      f"dt=1/128, direct sparse solve), {wall:.1f} s wall; NumPy/SciPy on one host "
                      f"core ({os.cpu_count()} available)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    # bounded per-step sample: 129^2 steps of the oracle, W + K of them
    n_sample = 129
    import workloads as W
    from oracle import lisl
    full = W.mixed_2049(seed=0)
    dt = 1.0 / 128
    total = args.warmup + args.steps
    p = W.manufactured(n_sample, 65, -0.95, 0.95, full.s1, full.s2, T=dt * total, n_steps=total)
    U = p.g.copy()
    pol = None
    t_steps = []
    for s in range(1, total + 1):
        t0 = time.perf_counter()
        r = lisl.howard_step(p, U, s * dt, dt, policy0=pol)
        t_steps.append(time.perf_counter() - t0)
        U, pol = r.X, r.policy
    timed = sum(t_steps[args.warmup:])
    value = n_sample * n_sample * args.steps / timed
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * timed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"oracle sample: {n_sample}x{n_sample} grid of the 2049x2049 "
                                   f"65-control uncertain-correlation workload, dt=1/128"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"each step one implicit step at {n_sample}x{n_sample}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------- GPU path

def run_ours(args):
    import numpy as np
    import torch

    import paper_1605_04821_gb300 as slp
    import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    else:
        dist = None

    def barrier():
        if dist is not None:
            dist.barrier()

    prob = W.mixed_2049(seed=0) if args.n == 2049 else W.scaled(args.n, 65, 128, seed=0,
                                                                   rho_range=(-0.95, 0.95))
    n = prob.n
    dt = 1.0 / 128
    stream = torch.cuda.current_stream()

    # V(1,1) for both precisions: the fastest cycle for this workload in either (V(2,2) costs
    # 11 % more in FP64 and 14 % more in mixed precision); --opt overrides
    extra = {"nu1": 1, "nu2": 1}
    for kv in args.opt:
        k, v = kv.split("=", 1)
        extra[k] = float(v) if "." in v or "e" in v else int(v)

    def make(precision):
        kw = dict(precision=precision, argmin_screen=1)  # the screen's decision is the FP64 one
        kw.update(extra)
        return slp.solver_from_problem(prob, device=dev, **kw)

    # ---- mixed path (the metric)
    s = make(1)
    g = torch.as_tensor(prob.g, dtype=torch.float64, device=dev)
    u = g.clone()
    for i in range(1, args.warmup + 1):
        s.step(u, i * dt, dt)
    torch.cuda.synchronize()
    u_after_warm = u.clone()
    compare_at = min(args.fp64_steps, args.steps)
    u_cmp = None
    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    launches0 = slp.launch_count()
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = {"pi_iters": 0, "krylov_iters": 0, "ir_iters": 0, "rebuilds": 0, "policy_changes": 0}
    for i in range(1, args.steps + 1):
        st = s.step(u, (args.warmup + i) * dt, dt)
        for kk in stats:
            stats[kk] += st[kk]
        if i == compare_at:
            u_cmp = u.clone()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = slp.launch_count() - launches0
    ms = e0.elapsed_time(e1)
    barrier()
    if dist is not None:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * n * n * args.steps / (ms / 1e3)
    explicit_rows = [s.level_info(l)[1] for l in range(s.num_levels())]

    # ---- roofline: the fine-level FP32 operator (matrix-free SpMV), timed alone with events
    m = n - 2
    x = torch.zeros((n, n), dtype=torch.float32, device=dev)
    x[1:-1, 1:-1] = torch.rand((m, m), device=dev)
    y = torch.zeros_like(x)
    for _ in range(3):
        s.apply(0, x, y)
    reps = 50
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    timing = "CUDA graph of 50 back-to-back launches, CUDA events around the replay"
    try:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            for _ in range(reps):
                s.apply(0, x, y)
        graph.replay()
        torch.cuda.synchronize()
        r0.record(stream)
        graph.replay()
        r1.record(stream)
        torch.cuda.synchronize()
    except Exception:
        timing = "50 stream-ordered launches, CUDA events around them"
        r0.record(stream)
        for _ in range(reps):
            s.apply(0, x, y)
        r1.record(stream)
        torch.cuda.synchronize()
    warm_ms = r0.elapsed_time(r1) / reps
    # cold: every operand evicted from L2 before each launch (a 256 MB write, larger than the
    # 129 MB L2), CUDA events around the launch alone; the median of 20 launches
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    cold = []
    for _ in range(20):
        flush.zero_()
        r0.record(stream)
        s.apply(0, x, y)
        r1.record(stream)
        torch.cuda.synchronize()
        cold.append(r0.elapsed_time(r1))
    kern_ms = statistics.median(cold)
    del flush
    bytes_per_launch = m * m * (1 + 4 + 4)   # policy byte, x_j, y_j (taps hit L1/L2)
    peak, peak_kind = measured_peaks()
    achieved = bytes_per_launch / (kern_ms / 1e3) / 1e9
    roofline = {"kernel": "k_fine_op_tma1<OP_APPLY,12> (fine-level matrix-free operator, FP32, "
                          "TMA-staged tiles)",
                "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs (burst copy)",
                "traffic": traffic_record("k_fine_op_tma1_apply_2049"),
                "algorithmic_bytes_per_launch": bytes_per_launch, "launch_ms": kern_ms,
                "timing": "cold: L2 flushed (256 MB write) before each launch, CUDA events around "
                          "the launch, median of 20",
                "warm_launch_ms": warm_ms, "warm_timing": timing,
                "warm_achieved": bytes_per_launch / (warm_ms / 1e3) / 1e9}
    del s
    torch.cuda.empty_cache()

    # ---- e2e through the public API with host-resident state
    se = make(1)
    ue = u_after_warm.clone()
    # replay the warm-up so that the handle's policy matches the timed run's starting point
    ue.copy_(g)
    for i in range(1, args.warmup + 1):
        se.step(ue, i * dt, dt)
    host = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
    host.copy_(ue)
    ke = args.steps if args.e2e_steps < 0 else min(args.e2e_steps, args.steps)
    torch.cuda.synchronize()
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0.record(stream)
    for i in range(1, ke + 1):
        ue.copy_(host, non_blocking=True)
        se.step(ue, (args.warmup + i) * dt, dt)
        host.copy_(ue, non_blocking=True)
    h1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = h0.elapsed_time(h1)
    e2e = {"value": world * n * n * ke / (e2e_ms / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": n * n * 8, "d2h_bytes_per_step": n * n * 8, "steps": ke}
    del se
    torch.cuda.empty_cache()

    # ---- FP64 path on the first steps of the same timed range
    fp64 = None
    err = None
    if not args.no_fp64:
        s64 = make(0)
        u64 = g.clone()
        for i in range(1, args.warmup + 1):
            s64.step(u64, i * dt, dt)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for i in range(1, compare_at + 1):
            s64.step(u64, (args.warmup + i) * dt, dt)
        f1.record(stream)
        torch.cuda.synchronize()
        f_ms = f0.elapsed_time(f1)
        fp64 = {"value": n * n * compare_at / (f_ms / 1e3), "unit": UNIT, "steps": compare_at,
                "ms_per_step": f_ms / compare_at}
        if u_cmp is not None:
            err = float((u_cmp - u64).abs().max() / u64.abs().max())
        del s64

    # ---- discrete adjoint: gradients of J = sum w U(T) on 1025^2, 33 controls, 64 steps
    adjoint = None
    if not args.no_adjoint:
        torch.cuda.nvtx.range_push("adjoint")  # lets a profiler select this part alone
        adjoint = adjoint_record(slp, W, dev, stream, extra, args.adjoint_steps)
        torch.cuda.nvtx.range_pop()

    # ---- aggregation AMG against the V-cycle on the same steps
    amg = None
    if not args.no_amg:
        torch.cuda.nvtx.range_push("amg")
        amg = amg_record(slp, prob, dev, stream, args, extra, g)
        torch.cuda.nvtx.range_pop()

    # ---- the plain FP64 configuration (513^2, 33 controls, 64 steps)
    fp64_513 = None
    if not args.no_fp64:
        torch.cuda.nvtx.range_push("fp64_513")
        fp64_513 = fp64_513_record(slp, W, dev, stream)
        torch.cuda.nvtx.range_pop()

    # ---- two-colour Gauss-Seidel against damped Jacobi on the same steps
    smoother = None
    if not args.no_smoother:
        torch.cuda.nvtx.range_push("smoother")
        smoother = smoother_record(slp, prob, dev, stream, args, extra, g)
        torch.cuda.nvtx.range_pop()

    # ---- batched: many independent instances, LPT-sharded over the ranks
    batched = None
    if not args.no_batched:
        torch.cuda.nvtx.range_push("batched")
        batched = batched_record(slp, W, dev, args, extra, rank, world, barrier, dist)
        torch.cuda.nvtx.range_pop()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_record()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"uncertain-correlation HJB, {n}x{n} grid, 65 controls rho in "
                                   f"[-0.95,0.95], s1={prob.s1:.4f} s2={prob.s2:.4f} (seed 0), "
                                   f"dt=1/128, steps {args.warmup + 1}..{args.warmup + args.steps}",
                       "precision": "mixed: FP32 V-cycle/inner BiCGSTAB, FP64 residual, argmin "
                                    "decision and refinement",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "working set > L2 (no flush needed)",
                       "levels": int(make_levels(n)), "pi_iters": stats["pi_iters"],
                       "krylov_iters": stats["krylov_iters"], "ir_iters": stats["ir_iters"],
                       "rebuilds": stats["rebuilds"], "opts": extra,
                       "explicit_rows_per_level": explicit_rows},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "fp64": fp64,
            "mixed_vs_fp64_rel_err": err,
            "adjoint": adjoint,
            "batched": batched,
            "amg": amg,
            "smoother": smoother,
            "fp64_513": fp64_513,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def adjoint_record(slp, W, dev, stream, extra, steps=64):
    """Forward march with recording, then the backward pass, each timed with CUDA events.
    The workload's checkpoint interval is 8 (the backward pass re-solves the 7 steps between
    two checkpoints); every U^n kept (interval 1) is timed beside it."""
    import copy

    import torch
    pa, wa = W.adjoint_1025(seed=0)
    if steps != pa.n_steps:
        pa = copy.copy(pa)
        pa.T = pa.T * steps / pa.n_steps
        pa.n_steps = steps
    dirs = W.sigma_directions(pa)
    na, nt = pa.n, pa.n_steps
    dta = pa.T / nt
    wd = torch.as_tensor(wa, dtype=torch.float64, device=dev)
    out = {"workload": f"uncertain-correlation HJB, {na}x{na} grid, 33 controls rho in "
                       f"[-0.9,0.9], s1=0.3 s2=0.2, {nt} steps of {dta:g}; J = sum w U(T) with a "
                       "seeded Gaussian bump w; checkpoints every 8 steps (every step in the "
                       "ckpt_every_1 entries)",
           "unit": UNIT}
    for prec, key in ((1, "mixed"), (0, "fp64")):
        kw = dict(precision=prec, argmin_screen=1)
        kw.update(extra)
        sa = slp.solver_from_problem(pa, device=dev, **kw)
        ua0 = torch.as_tensor(pa.g, dtype=torch.float64, device=dev)
        dg = torch.zeros_like(ua0)
        sa.solve_record(ua0.clone(), 0.0, 3 * dta, 3, 1)   # warm-up: buffers and graphs
        sa.adjoint(wd, dg, None, dirs)
        for ckpt in (8, 1):
            ua = ua0.clone()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            torch.cuda.synchronize()
            l0 = slp.launch_count()
            ev[0].record(stream)
            stf = sa.solve_record(ua, 0.0, pa.T, nt, ckpt)
            ev[1].record(stream)
            dth, stb = sa.adjoint(wd, dg, None, dirs)
            ev[2].record(stream)
            torch.cuda.synchronize()
            fwd, bwd = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
            rec = {"value": na * na * nt / (bwd / 1e3), "ckpt_every": ckpt, "backward_ms": bwd,
                   "backward_ms_per_step": bwd / nt, "forward_record_ms": fwd,
                   "forward_ms_per_step": fwd / nt, "backward_krylov_iters": stb["krylov_iters"],
                   "forward_krylov_iters": stf["krylov_iters"],
                   "gpu_launches": slp.launch_count() - l0,
                   "dJ_dtheta": [float(v) for v in dth],
                   "J": float((wd * ua).sum())}
            if ckpt == 8:
                out[key] = rec
            else:
                out[key]["ckpt_every_1"] = rec
        del sa
        torch.cuda.empty_cache()
    out["value"] = out["mixed"]["value"]
    return out


def amg_record(slp, prob, dev, stream, args, extra, g):
    """Mixed-precision steps W+1 .. W+K of the headline workload with the aggregation K-cycle
    (precond 1) and with the V-cycle (precond 0), each timed with CUDA events."""
    import torch
    n = prob.n
    dt = 1.0 / 128
    k = args.amg_steps
    out = {"workload": f"steps {args.warmup + 1}..{args.warmup + k} of the headline workload, mixed precision",
           "unit": UNIT}
    for pc, key in ((1, "aggregation_kcycle"), (0, "geometric_vcycle")):
        kw = dict(precision=1, argmin_screen=1, precond=pc)
        kw.update(extra)
        s = slp.solver_from_problem(prob, device=dev, **kw)
        u = g.clone()
        for i in range(1, args.warmup + 1):
            s.step(u, i * dt, dt)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st = {"pi_iters": 0, "krylov_iters": 0, "ir_iters": 0}
        e0.record(stream)
        for i in range(1, k + 1):
            r = s.step(u, (args.warmup + i) * dt, dt)
            for kk in st:
                st[kk] += r[kk]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[key] = {"value": n * n * k / (ms / 1e3), "ms_per_step": ms / k, **st}
        del s
        torch.cuda.empty_cache()
    out["value"] = out["aggregation_kcycle"]["value"]
    return out


def fp64_513_record(slp, W, dev, stream):
    """The plain FP64 workload: 513 x 513 grid, 33 controls, 64 implicit steps to T = 1, V(2,2)
    damped Jacobi (omega 0.8), BiCGSTAB to the default tolerance, every step FP64.  The whole
    march is timed with CUDA events, its first step included (it is part of the workload); the
    GPU tests compare the same march with the oracle's stored one."""
    import torch
    p = W.plain_fp64()
    s = slp.solver_from_problem(p, device=dev, precision=0, nu1=2, nu2=2, omega=0.8)
    dt = p.T / p.n_steps
    u = torch.as_tensor(p.g, dtype=torch.float64, device=dev)
    s.step(u.clone(), dt, dt)  # builds the graphs of this step size once (not timed)
    s.reset()                  # the timed march starts like a new handle's
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st = {"pi_iters": 0, "krylov_iters": 0}
    e0.record(stream)
    for i in range(1, p.n_steps + 1):
        r = s.step(u, i * dt, dt)
        for kk in st:
            st[kk] += r[kk]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    del s
    torch.cuda.empty_cache()
    return {"workload": f"{p.n}x{p.n} grid, {p.K} controls, {p.n_steps} steps to T = {p.T}, FP64, "
                        "V(2,2) damped Jacobi omega 0.8, 8 levels",
            "value": p.n * p.n * p.n_steps / (ms / 1e3), "unit": UNIT, "ms_total": ms,
            "ms_per_step": ms / p.n_steps, **st}


def smoother_record(slp, prob, dev, stream, args, extra, g):
    """Mixed-precision steps W+1 .. W+K of the headline workload with two-colour Gauss-Seidel
    smoothing (relaxation 1) and with damped Jacobi (omega 0.8), each timed with CUDA events."""
    import torch
    n = prob.n
    dt = 1.0 / 128
    k = args.amg_steps
    out = {"workload": f"steps {args.warmup + 1}..{args.warmup + k} of the headline workload, mixed precision",
           "unit": UNIT}
    for sm, om, key in ((1, 1.0, "red_black_gauss_seidel"), (0, 0.8, "damped_jacobi")):
        kw = dict(precision=1, argmin_screen=1)
        kw.update(extra)
        kw.update(smoother=sm, omega=om)
        s = slp.solver_from_problem(prob, device=dev, **kw)
        u = g.clone()
        for i in range(1, args.warmup + 1):
            s.step(u, i * dt, dt)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st = {"pi_iters": 0, "krylov_iters": 0, "ir_iters": 0}
        e0.record(stream)
        for i in range(1, k + 1):
            r = s.step(u, (args.warmup + i) * dt, dt)
            for kk in st:
                st[kk] += r[kk]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[key] = {"value": n * n * k / (ms / 1e3), "ms_per_step": ms / k, "omega": om, **st}
        del s
        torch.cuda.empty_cache()
    out["value"] = out["red_black_gauss_seidel"]["value"]
    return out


def batched_record(slp, W, dev, args, extra, rank, world, barrier, dist):
    """The batched workload (independent instances of the same PDE family), LPT-sharded over the
    ranks and over W worker threads per rank, each with its own stream, every BiCGSTAB iteration
    one graph launch (use_graphs 1: these overlap across streams better than the device-driven
    steps).  Timed on the host around sl_batch_run, which returns when every instance's stream
    is idle: once with the default launch configuration, then with the one sl_batch_autotune
    chooses per grid size (the V-cycle tail, by probe runs of the whole batch)."""
    import torch
    probs = W.batched(n_inst=args.batched_instances, seed=0)
    mine = slp.shard(probs, world, rank)
    sub = [probs[i] for i in mine]
    us = [torch.as_tensor(p.g, dtype=torch.float64, device=dev) for p in sub]
    kw = dict(precision=1, argmin_screen=1)
    kw.update(extra)
    kw["use_graphs"] = args.batched_graphs
    out = {"workload": f"{len(probs)} instances of the uncertain-correlation family: n uniform in "
                       "{65,129,257,513}, (s1,s2) ~ U[0.15,0.4]^2, K ~ U{17..65}, rho in "
                       "[-0.9,0.9], 32 steps of 1/32 (seed 0); mixed precision",
           "unit": UNIT, "instances": len(probs), "scaling": "weak" if world > 1 else None,
           "sharding": "LPT over ranks by n^2 * steps * (K + 32), no collective" if world > 1 else None}
    gp = sum(p.n * p.n * p.n_steps for p in sub)

    def timed_run(b, key, workers):
        for u, p in zip(us, sub):
            u.copy_(torch.as_tensor(p.g, device=dev))
        b.run()   # warm-up: graphs and class tables of every handle
        for u, p in zip(us, sub):
            u.copy_(torch.as_tensor(p.g, device=dev))
        torch.cuda.synchronize()
        barrier()
        l0 = slp.launch_count()
        t0 = time.perf_counter()
        st, stats = b.run()
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        launches = slp.launch_count() - l0
        if dist is not None:
            t = torch.tensor([sec], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            sec = float(t.item())
            g = torch.tensor([gp], device=dev, dtype=torch.float64)
            dist.all_reduce(g)
            total = float(g.item())
        else:
            total = float(gp)
        out[key] = {"workers": workers, "value": total / sec, "seconds": sec,
                    "failed": int(sum(1 for x in st if x != 0)), "gpu_launches": launches,
                    "pi_iters": int(sum(s["pi_iters"] for s in stats)),
                    "krylov_iters": int(sum(s["krylov_iters"] for s in stats))}

    b = slp.Batch(sub, us, workers=args.batched_workers, device=dev, **kw)
    timed_run(b, "default_launch", args.batched_workers)
    t0 = time.perf_counter()
    choices = b.autotune(probe_steps=3)
    out["autotune"] = {"seconds": time.perf_counter() - t0, "probe_steps": 3,
                       "choices": choices, "tunable": "single-block V-cycle tail (coarse_tail_rows) "
                                                      "per grid size"}
    timed_run(b, "concurrent", args.batched_workers)
    b.close()
    del b
    torch.cuda.empty_cache()
    if args.batched_one_worker:
        b = slp.Batch(sub, us, workers=1, device=dev, **kw)
        timed_run(b, "one_worker", 1)
        b.close()
        del b
        torch.cuda.empty_cache()
        out["speedup_vs_one_worker"] = out["concurrent"]["value"] / out["one_worker"]["value"]
    out["value"] = out["concurrent"]["value"]
    return out


def make_levels(n):
    L, nn = 1, n
    while nn > 5 and (nn - 1) % 2 == 0:
        nn = (nn + 1) // 2
        L += 1
    return L


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
