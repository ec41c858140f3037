#!/usr/bin/env python
"""Benchmark: semi-implicit Landau-Lifshitz time steps on one B300 per rank.

Workload (the time-stepping configuration): 3-D 128^3 cells (6.29M unknowns),
h = 1/128, Neumann boundaries, alpha = 0.02, dt = 5e-4; initial state a vortex
core plus 1e-2 Gaussian noise, normalised (seed 0).  One bench step = one
time step through the C ABI (ll_mg_step): numeric setup for m~ = m^n,
aggregation-AMG-preconditioned GCR to relative residual 1e-8, projection
m <- x/|x|.  The metric is unknown-solves per second (3 N unknowns per step).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--precision fp64|mixed]
Prints one JSON line (rank 0).  Ranks are independent replicas (the solve
does not shard); value = unknowns solved by all ranks / max over ranks of the
timed region.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

GRID = (128, 128, 128)
H_SPACING, ALPHA, DT, RTOL = 1.0 / 128, 0.02, 5e-4, 1e-8
N_CELLS = GRID[0] * GRID[1] * GRID[2]
UNKNOWNS = 3 * N_CELLS
METRIC = "unknown-solves/s to rel. residual 1e-8"
UNIT = "unknown-solves/s"
WORKLOAD = "3D 128^3 semi-implicit LL time steps, alpha 0.02, dt 5e-4, vortex + 1e-2 noise, rtol 1e-8"

# FP64 peak derived from unit counts and clocks: 148 SMs x 2 FP64 FMA/clk/SM
# x 2 flop x 2.032 GHz (a DFMA throughput probe on this machine read 1.13 TFLOP/s
# at 1.94 GHz, i.e. the same 2 FMA/clk/SM)
FP64_PEAK_TFLOPS = 148 * 2 * 2 * 2.032e9 / 1e12

# DRAM traffic of the float64 coarse sweeps per launch over the algorithmic
# bytes: ncu dram__bytes_read.sum + dram__bytes_write.sum on 400 kb_sweep
# launches of the --grid 96 case, against the library's byte model for the
# same launches (profiles/kb_sweep_96cube_fp64.md).  Scaled by the bytes a
# launch processes to the traffic of a 128^3 launch.
KB_SWEEP_TRAFFIC_RATIO = 9.679e6 / 9.293e6

KIND_NAMES = ["l0_smooth", "l0_restrict", "outer_apply", "bsr_smooth", "bsr_other", "gcr_vector", "coarsest",
              "numeric", "coarse_tail"]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle sample (the reference arm and the cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_sample(iters_sample: int = 3):
    """Time the FP64 CPU oracle on the full 128^3 workload: its whole setup
    for one step plus `iters_sample` GCR iterations.  Returns (setup_s,
    seconds per GCR iteration)."""
    import oracle
    from paper_2608_09102_b300 import inputs

    m = inputs.vortex(*GRID, seed=0).reshape(-1)
    t0 = time.perf_counter()
    H = oracle.Hierarchy(GRID, H_SPACING, ALPHA, DT, m, oracle.Params(rtol=RTOL, maxit=iters_sample))
    t1 = time.perf_counter()
    b = m / DT
    _, st, it, _ = H.solve(b, m.copy())
    t2 = time.perf_counter()
    return t1 - t0, (t2 - t1) / max(it, 1)


# the oracle's own GCR iteration count on the first step of this workload
# (42, from a full oracle solve); used to extrapolate the reference arm
ORACLE_ITERS_PER_STEP = 42


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    times = []
    setup_s = per_iter = None
    t_all = time.perf_counter()
    steps = max(1, min(args.steps, 3))
    for _ in range(steps):
        s, p = oracle_sample(1)
        setup_s = s if setup_s is None else min(setup_s, s)
        per_iter = p if per_iter is None else min(per_iter, p)
        times.append(s + ORACLE_ITERS_PER_STEP * p)
    step_s = statistics.median(times)
    value = UNKNOWNS / step_s
    sample = ("%d x (oracle setup of one 128^3 step + 1 GCR iteration), extrapolated to %d iterations per step"
              % (steps, ORACLE_ITERS_PER_STEP))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": 0, "ms_per_step": step_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": list(GRID), "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "oracle_setup_s": setup_s, "oracle_s_per_iteration": per_iter,
            "wall_s": time.perf_counter() - t_all}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# replicas: every rank solves its own copy of the workload (the solve does
# not shard); the job's time is the slowest rank's
# ---------------------------------------------------------------------------
def max_over_ranks(v: float, device) -> float:
    """Maximum of v over the ranks of the default process group (v itself
    when there is none)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(v)
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput of `world` replicas that each processed
    units_per_rank in at most `seconds` (the maximum over ranks)."""
    return units_per_rank * world / seconds


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
# kinds that make up the V-cycle preconditioner
VCYCLE_KINDS = ("l0_smooth", "l0_restrict", "bsr_smooth", "bsr_other", "coarsest", "coarse_tail")

# kinds whose arithmetic is float64 whatever the V-cycle precision
FP64_KINDS = {"outer_apply", "gcr_vector", "coarsest", "numeric"}


def roofline(kind: str, ms: float, launches: int, flops: float, byts: float, precision: str, peaks: dict,
             peak_src: str):
    """Roofline entry of one kernel kind from the library's live event timing
    and its algorithmic flop and byte counts (models stated in ll_mg.h).
    float64 kernels are bound by the float64 pipe of this GPU (2 FMA per
    clock per SM, measured); float32 V-cycle kernels by HBM."""
    avg_ms = ms / max(launches, 1)
    per_launch_flops = flops / max(launches, 1)
    per_launch_bytes = byts / max(launches, 1)
    ach_tf = per_launch_flops / (avg_ms * 1e-3) / 1e12 if avg_ms > 0 else None
    ach_gb = per_launch_bytes / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else None
    common = {"kernel_kind": kind, "launches": launches, "avg_launch_ms": avg_ms,
              "flops_per_launch": per_launch_flops, "bytes_per_launch": per_launch_bytes, "traffic": None}
    if precision == "fp64" or kind in FP64_KINDS:
        return dict(bound="alu", achieved=ach_tf, peak=FP64_PEAK_TFLOPS, unit="TFLOP/s",
                    frac=(ach_tf / FP64_PEAK_TFLOPS) if ach_tf else None,
                    peak_source="derived: 148 SMs x 2 FP64 FMA/clk x 2 flop x 2.032 GHz (probe: 1.13 TF at 1.94 GHz)",
                    hbm_gbs=ach_gb, hbm_frac_of_measured=(ach_gb / peaks["hbm_gbs"]) if ach_gb else None, **common)
    return dict(bound="hbm", achieved=ach_gb, peak=peaks["hbm_gbs"], unit="GB/s",
                frac=(ach_gb / peaks["hbm_gbs"]) if ach_gb else None, peak_source=peak_src,
                tflops=ach_tf, **common)


def run_ours(args):
    import torch

    import paper_2608_09102_b300 as ll
    from paper_2608_09102_b300 import build, inputs

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    dev = torch.device("cuda", local)
    precision = {"fp64": ll.LL_FP64, "mixed": ll.LL_MIXED_FP32, "bf16": ll.LL_MIXED_BF16}[args.precision]
    m0 = inputs.vortex(*GRID, seed=0).reshape(-1)
    m = torch.tensor(m0, device=dev)
    error_vs_fp64 = None
    if precision != ll.LL_FP64:  # one step both ways from the same state
        ma, mb = m.clone(), m.clone()
        ll.Hierarchy(ma, ALPHA, DT, H_SPACING, GRID, ll.Params(rtol=RTOL)).step(ma, 1)
        ll.Hierarchy(mb, ALPHA, DT, H_SPACING, GRID, ll.Params(rtol=RTOL, precision=precision,
                                                               kcycle=args.kcycle)).step(mb, 1)
        error_vs_fp64 = float(torch.linalg.norm(mb - ma) / torch.linalg.norm(ma))
        del ma, mb
        torch.cuda.empty_cache()
    t0 = time.perf_counter()
    H = ll.Hierarchy(m, ALPHA, DT, H_SPACING, GRID, ll.Params(rtol=RTOL, precision=precision, kcycle=args.kcycle))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    lib = ll.load_library()
    import ctypes

    def prof_start(mask):
        lib.ll_mg_profile(H._h, ctypes.c_uint(mask))

    def prof_read(kind):
        ms = ctypes.c_double(0)
        cnt = ctypes.c_longlong(0)
        fl = ctypes.c_double(0)
        by = ctypes.c_double(0)
        lib.ll_mg_profile_read(H._h, kind, ctypes.byref(ms), ctypes.byref(cnt), ctypes.byref(fl), ctypes.byref(by))
        return ms.value, cnt.value, fl.value, by.value

    # warm-up steps, with every kernel kind timed to find the dominant kernel
    prof_start((1 << len(KIND_NAMES)) - 1)
    for _ in range(args.warmup):
        H.step(m, 1)
    breakdown = {KIND_NAMES[k]: prof_read(k) for k in range(len(KIND_NAMES))}
    kernel_kinds = [k for k in KIND_NAMES if k != "numeric"]
    dominant = max(kernel_kinds, key=lambda k: breakdown[k][0])
    prof_start(1 << KIND_NAMES.index(dominant))
    H.step(m, 1)  # one more warm-up step: graphs re-captured with the timed kind
    prof_start(1 << KIND_NAMES.index(dominant))

    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    its, rrs = [], []
    launches0 = ll.launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    ev0.record(stream)
    for _ in range(args.steps):
        st, it, rr = H.step(m, 1)
        its += it
        rrs += rr
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if world > 1:
        dist.barrier()
    elapsed_ms = ev0.elapsed_time(ev1)
    launches = ll.launch_count() - launches0
    dom_ms, dom_launches, dom_flops, dom_bytes = prof_read(KIND_NAMES.index(dominant))
    prof_start(0)
    elapsed_ms = max_over_ranks(elapsed_ms, dev)

    # end to end through the public API with host buffers (pinned), copies timed
    e2e_steps = max(1, min(args.steps, 10))
    mh = m.detach().cpu().pin_memory()
    torch.cuda.synchronize()
    te = time.perf_counter()
    for _ in range(e2e_steps):
        H.step(mh, 1)  # copies host -> device, steps, copies back
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - te, dev)

    if rank != 0:
        return
    value = replica_throughput(UNKNOWNS * args.steps, world, elapsed_ms * 1e-3)
    peaks, peak_src = measured_peaks()
    roof = roofline(dominant, dom_ms, dom_launches, dom_flops, dom_bytes, args.precision, peaks, peak_src)
    if dominant == "bsr_smooth" and args.precision == "fp64" and roof.get("bytes_per_launch"):
        roof["traffic"] = KB_SWEEP_TRAFFIC_RATIO * roof["bytes_per_launch"]
        roof["traffic_source"] = ("ncu DRAM bytes of kb_sweep at 96^3 / algorithmic bytes = %.3f, times this "
                                  "launch's algorithmic bytes" % KB_SWEEP_TRAFFIC_RATIO)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "mixed": "f32+f64", "bf16": "bf16+f32+f64"}[args.precision],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": list(GRID), "h": H_SPACING, "alpha": ALPHA, "dt": DT,
                   "rtol": RTOL, "precision": args.precision, "kcycle": args.kcycle, "parallelism": "replicas" if world > 1 else "single",
                   "levels": H.levels, "l2": "working set per step (~3 GB: GCR bases, operators) exceeds the 126 MB L2"},
        "iterations_per_step": {"mean": float(np.mean(its)), "min": int(min(its)), "max": int(max(its))},
        "max_relres": float(max(rrs)),
        "error_vs_fp64": error_vs_fp64,
        "setup_s": setup_s,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "roofline": roof,
        "kernel_breakdown_warmup_ms": {k: round(v[0], 3) for k, v in breakdown.items()},
        # the V-cycle's kernels together (algorithmic bytes over their event time, warm-up steps)
        "vcycle_hbm_gbs": (sum(breakdown[k][3] for k in VCYCLE_KINDS)
                           / max(sum(breakdown[k][0] for k in VCYCLE_KINDS), 1e-9) / 1e6),
        "numeric_setup_ms_per_step": breakdown["numeric"][0] / max(args.warmup, 1),
        "kernel_roofline_warmup": {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv)
                                       for kk, vv in roofline(k, *breakdown[k], args.precision, peaks,
                                                              peak_src).items()
                                       if kk in ("bound", "achieved", "unit", "frac", "hbm_gbs", "tflops")}
                                   for k in KIND_NAMES if breakdown[k][1] > 0},
        "e2e": {"value": replica_throughput(UNKNOWNS * e2e_steps, world, e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": UNKNOWNS * 8 * world, "d2h_bytes_per_step": UNKNOWNS * 8 * world,
                "steps": e2e_steps},
    }
    if not args.no_cpu_baseline:
        s, p = oracle_sample(3)
        it_mean = float(np.mean(its))
        cpu_v = UNKNOWNS / (s + it_mean * p)
        line["cpu_baseline"] = {"value": cpu_v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "oracle setup of one 128^3 step + 3 GCR iterations, extrapolated to "
                                          "the measured %.1f iterations per step" % it_mean}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# ragged batch of independent instances (measured on request)
# ---------------------------------------------------------------------------
BATCH_COUNT = 512
BATCH_WORKLOAD = ("512 independent 2-D instances, sides uniform from {32,48,64,96,128,192,256}, h = 1/side, "
                  "alpha log-uniform [0.005, 1], dt log-uniform [1e-5, 1e-2], smooth unit fields; one step = "
                  "numeric setup + solve of every instance to rtol 1e-8")


def run_batch(args):
    import torch

    import paper_2608_09102_b300 as ll
    from paper_2608_09102_b300 import build, inputs

    build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    precision = {"fp64": ll.LL_FP64, "mixed": ll.LL_MIXED_FP32}[args.precision]
    spec = inputs.batch_instances(args.batch_count, seed=0)
    ms = [torch.tensor(inputs.smooth_field(*s["grid"], seed=s["seed"]).reshape(-1), device=dev) for s in spec]
    alphas = [s["alpha"] for s in spec]
    dts = [s["dt"] for s in spec]
    ns = [int(np.prod(s["grid"])) for s in spec]
    params = ll.Params(rtol=RTOL, precision=precision, maxit=args.batch_maxit)
    t0 = time.perf_counter()
    B = ll.Batch(ms, alphas, dts, [s["h"] for s in spec], [s["grid"] for s in spec], params)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    rhs = [m / dt for m, dt in zip(ms, dts)]
    xs = [torch.zeros_like(m) for m in ms]

    def step():
        B.update(ms, alphas, dts)
        for x in xs:
            x.zero_()
        return B.solve(rhs, xs)

    for _ in range(args.warmup):
        step()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(0)
    launches0 = ll.launch_count()
    torch.cuda.synchronize()
    sampler.start()
    ev0.record(stream)
    for _ in range(args.steps):
        st, its, rrs, sts = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    elapsed_ms = ev0.elapsed_time(ev1)
    launches = ll.launch_count() - launches0
    conv = [k for k in range(len(spec)) if sts[k] == ll.LL_OK]
    solved = 3 * sum(ns[k] for k in conv)
    total = 3 * sum(ns)
    # end to end: host (pinned) right-hand sides in, solutions out, every step
    hr = [r.cpu().pin_memory() for r in rhs]
    hx = [torch.empty_like(h).pin_memory() for h in hr]
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    te = time.perf_counter()
    for _ in range(e2e_steps):
        for d, h in zip(rhs, hr):
            d.copy_(h, non_blocking=True)
        step()
        for h, x in zip(hx, xs):
            h.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - te
    line = {
        "metric": METRIC, "value": solved * args.steps / (elapsed_ms * 1e-3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "mixed": "f32+f64"}[args.precision], "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD, "instances": len(spec), "cells": sum(ns), "unknowns": total,
                   "precision": args.precision, "maxit": args.batch_maxit,
                   "l2": "working set (~6 GB) exceeds the 126 MB L2"},
        "converged": len(conv), "unknowns_converged": solved,
        "not_converged": [{"side": spec[k]["grid"][0], "alpha": spec[k]["alpha"], "dt": spec[k]["dt"],
                           "status": sts[k], "relres": rrs[k], "iterations": its[k]}
                          for k in range(len(spec)) if sts[k] != ll.LL_OK],
        "iterations": {"mean": float(np.mean(its)), "median": float(np.median(its)), "max": int(max(its)),
                       "lockstep": int(max(its))},
        "levels": B.levels, "setup_s": setup_s, "gpu_launches": int(launches), "clocks": clocks,
        "e2e": {"value": solved * e2e_steps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": 8 * total, "d2h_bytes_per_step": 8 * total, "steps": e2e_steps},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# differentiation workload (measured on request)
# ---------------------------------------------------------------------------
GRAD_WORKLOAD = ("3-D 96^3, alpha 0.1, dt 1e-3, 20 steps, loss 0.5|m^20 - m_target|^2 (smooth unit fields, seeds "
                 "0 and 1), gradient in m^0 and alpha by the adjoint with checkpoints every 5 steps, rtol 1e-8")


def run_grad(args):
    import torch

    import paper_2608_09102_b300 as ll
    from paper_2608_09102_b300 import build, inputs

    build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    grid, alpha, dt, n_steps, h = (96, 96, 96), 0.1, 1e-3, 20, 1.0 / 96
    n = 96 ** 3
    m0 = torch.tensor(inputs.smooth_field(*grid, seed=0).reshape(-1), device=dev)
    mt = torch.tensor(inputs.smooth_field(*grid, seed=1).reshape(-1), device=dev)
    precision = {"fp64": ll.LL_FP64, "mixed": ll.LL_MIXED_FP32}[args.precision]
    p = ll.Params(rtol=RTOL, precision=precision)

    def grad():
        m = m0.clone().requires_grad_(True)
        a = torch.tensor(alpha, dtype=torch.float64, requires_grad=True)
        mN = ll.steps_autograd(m, a, n_steps, dt, h, grid, p, checkpoint=5)
        loss = 0.5 * torch.sum((mN - mt) ** 2)
        loss.backward()
        return float(loss.detach()), m.grad, float(a.grad)

    for _ in range(args.warmup):
        grad()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(0)
    launches0 = ll.launch_count()
    torch.cuda.synchronize()
    sampler.start()
    ev0.record(stream)
    for _ in range(args.steps):
        loss, gm, ga = grad()
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    solves = 3 * n_steps  # forward, recomputed forward, adjoint
    line = {"metric": "gradient evaluations/s", "value": 1e3 / ms, "unit": "gradients/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "mixed": "f32+f64"}[args.precision], "data": "synthetic",
            "config": {"workload": GRAD_WORKLOAD, "unknowns": 3 * n, "precision": args.precision},
            "unknown_solves_per_s": solves * 3 * n / (ms * 1e-3), "solves_per_gradient": solves,
            "loss": loss, "grad_norm_m0": float(torch.linalg.norm(gm)), "grad_alpha": ga,
            "gpu_launches": int(ll.launch_count() - launches0), "clocks": clocks}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed", "bf16"], default="fp64")
    ap.add_argument("--kcycle", type=int, default=0,
                    help="coarse levels 1..K solved by two inner GCR steps (K-cycle); 0 = V-cycle")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["step128", "batch512", "grad96"], default="step128",
                    help="step128: the 128^3 time-stepping workload; batch512: the ragged batch; "
                         "grad96: the 96^3 differentiation workload")
    ap.add_argument("--batch-count", type=int, default=BATCH_COUNT)
    ap.add_argument("--batch-maxit", type=int, default=300)
    ap.add_argument("--grid", type=int, default=128,
                    help="cube side of the step workload (default 128; smaller sides are profiling cases)")
    args = ap.parse_args()
    if args.grid != 128:
        global GRID, H_SPACING, N_CELLS, UNKNOWNS, WORKLOAD
        GRID = (args.grid,) * 3
        H_SPACING = 1.0 / args.grid
        N_CELLS = args.grid ** 3
        UNKNOWNS = 3 * N_CELLS
        WORKLOAD = WORKLOAD.replace("128^3", "%d^3 (profiling case)" % args.grid)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch512":
        run_batch(args)
    elif args.workload == "grad96":
        run_grad(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
