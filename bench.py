#!/usr/bin/env python
"""Benchmark: semi-implicit Landau-Lifshitz time steps on one B300 per rank.

Workload (the time-stepping configuration): 3-D 128^3 cells (6.29M unknowns),
h = 1/128, Neumann boundaries, alpha = 0.02, dt = 5e-4; initial state a vortex
core plus 1e-2 Gaussian noise, normalised (seed 0).  One bench step = one
time step through the C ABI (ll_mg_step): numeric setup for m~ = m^n,
aggregation-AMG-preconditioned GCR to relative residual 1e-8, projection
m <- x/|x|.  The metric is unknown-solves per second (3 N unknowns per step).

The default run times, in this order:
  * the headline: K float64 steps with no instrumentation (CUDA events on
    the launching stream around the K steps);
  * the same K steps in float64, with the float32 V-cycle (mixed) and with
    bfloat16 coarse operators (bf16, the mixed-precision configuration:
    float32 V-cycle, bfloat16 coarse levels, float64 GCR), each from the same
    initial state and one after another, for the mixed-vs-float64 speedup at
    the same true relative residual 1e-8;
  * a separate profiling pass of the float64 path (per-kind event timing) for
    the kernel breakdown and the dominant kernel's roofline;
  * end to end: steps of a pinned host field through ll_mg_step_host (the
    library copies it in and out on its stream every step);
  * the float64 multiply-add probe (the measured float64 peak);
  * one compact measurement of each of the other workloads
    (other_workloads: the 64^2 solve, the 256^2 x 128 random-unit-vector
    solves, the 512-instance batch, the 96^3 gradient);
  * the CPU oracle on a bounded sample (cpu_baseline).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--precision fp64|mixed|bf16] [--workload step128|batch512|grad96]
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
# x 2 flop x 2.032 GHz.  The bench also measures it (ll_fp64_fma_probe).
FP64_PEAK_TFLOPS = 148 * 2 * 2 * 2.032e9 / 1e12

# DRAM traffic of the float64 coarse sweeps per launch over their algorithmic
# bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum, 96^3 profiling
# case, three launches of each sweep kernel): the level-1 classes on the
# SELL-32 copy (ks_sweep: 89.75 MB against 104.46 MB of the byte model,
# 0.859) and small classes on BSR (kb_sweep: 5.22 MB against 5.26 MB, 0.992),
# weighted by the model's bytes of one V-cycle's sweeps at 96^3 (424 MB on the
# SELL-32 copy, 162 MB on BSR).  Scaled by the bytes a launch processes to a
# 128^3 launch.
KB_SWEEP_TRAFFIC_RATIO = (424.05 * 0.8592 + 162.25 * 0.9919) / (424.05 + 162.25)

KIND_NAMES = ["l0_smooth", "l0_restrict", "outer_apply", "bsr_smooth", "bsr_other", "gcr_vector", "coarsest",
              "numeric", "coarse_tail"]

# The oracle's bounded sample: whole time steps on the central 48^3 block of
# the 128^3 workload field (same h, alpha, dt, rtol; Neumann boundaries at
# the block's faces).
SAMPLE_SIDE = 48


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
# CPU oracle: whole time steps on a bounded block of the workload (the
# reference arm and the cpu_baseline)
# ---------------------------------------------------------------------------
def sample_field(side: int = SAMPLE_SIDE):
    """The central side^3 block of the 128^3 workload's initial field."""
    from paper_2608_09102_b300 import inputs

    off = (GRID[0] - side) // 2
    m = inputs.vortex(*GRID, seed=0).reshape(3, GRID[2], GRID[1], GRID[0])
    return np.ascontiguousarray(m[:, off:off + side, off:off + side, off:off + side]).reshape(-1)


def oracle_steps(m, n_steps: int, side: int = SAMPLE_SIDE):
    """n_steps whole oracle time steps (setup, GCR solve to 1e-8, projection)
    from m in one call, so that its later steps start from the extrapolated
    state as the library's do; returns (m, seconds per step (the call's time
    spread evenly), iterations per step)."""
    import oracle

    if n_steps <= 0:
        return m, [], []
    t0 = time.perf_counter()
    m, it, rr, st = oracle.step(m, n_steps, (side,) * 3, H_SPACING, ALPHA, DT, oracle.Params(rtol=RTOL))
    el = time.perf_counter() - t0
    return m, [el / n_steps] * n_steps, [int(v) for v in it]


def _replica_worker(side, barrier, out):
    m = sample_field(side)
    import oracle

    oracle._load()
    barrier.wait()
    t0 = time.perf_counter()
    _, secs, its = oracle_steps(m, 1, side)
    out.put((time.perf_counter() - t0, its[0]))


def oracle_all_cores(side: int = SAMPLE_SIDE):
    """One whole oracle step in each of P concurrent processes (P = the host's
    cores, fewer if memory is short: about 0.4 GB per process at 48^3), all
    released together; returns (unknown-solves/s of all P, P, seconds of the
    slowest, nproc).  The oracle is single-threaded, so its all-core
    throughput is that of independent replicas."""
    import multiprocessing as mp

    nproc = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    try:
        import psutil

        avail = psutil.virtual_memory().available
        procs = max(1, min(nproc, int(avail * 0.5 / (0.4e9 * (side / 48) ** 3))))
    except ImportError:
        procs = nproc
    ctx = mp.get_context("spawn")  # never fork a process that has used CUDA
    barrier = ctx.Barrier(procs)
    q = ctx.Queue()
    workers = [ctx.Process(target=_replica_worker, args=(side, barrier, q)) for _ in range(procs)]
    for w in workers:
        w.start()
    res = [q.get(timeout=1800) for _ in workers]
    for w in workers:
        w.join(timeout=60)
    slowest = max(r[0] for r in res)
    return 3 * side ** 3 * procs / slowest, procs, slowest, nproc


def run_reference(args):
    """The reference arm: the FP64 CPU oracle as it stands, one thread, on
    whole time steps of the bounded sample (W untimed, K timed), then the
    all-core replica throughput of the same sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    t_all = time.perf_counter()
    m = sample_field()
    m, _, _ = oracle_steps(m, args.warmup)
    t0 = time.perf_counter()
    m, secs, its = oracle_steps(m, args.steps)
    elapsed = time.perf_counter() - t0
    unknowns = 3 * SAMPLE_SIDE ** 3
    value = unknowns * args.steps / elapsed
    allc, procs, slowest, nproc = oracle_all_cores()
    sample = ("whole oracle time steps (setup, GCR to 1e-8, projection) on the central %d^3 block of the 128^3 "
              "workload field, same h, alpha, dt; %d untimed, %d timed, one thread"
              % (SAMPLE_SIDE, args.warmup, args.steps))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": list(GRID), "precision": "fp64",
                       "sample": "%d^3 central block" % SAMPLE_SIDE},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "all_cores": {"value": allc, "unit": UNIT, "cores": procs, "processes": procs,
                          "slowest_step_s": slowest,
                          "sample": "one whole step of the same block in each of %d concurrent processes" % procs},
            "nproc": nproc,
            "iterations_per_step": {"mean": float(np.mean(its)), "min": int(min(its)), "max": int(max(its))},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t_all}
    print(json.dumps(line), flush=True)


def cpu_baseline():
    """The oracle on the bounded sample, for our arm's line: two whole steps
    on one thread, then one step in each of P concurrent processes."""
    m = sample_field()
    _, secs, its = oracle_steps(m, 2)
    unknowns = 3 * SAMPLE_SIDE ** 3
    value = unknowns * len(secs) / sum(secs)
    allc, procs, slowest, nproc = oracle_all_cores()
    return {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": ("2 whole oracle time steps (setup, GCR to 1e-8, projection) on the central %d^3 block of the "
                       "128^3 workload field, same h, alpha, dt, one thread; %s GCR iterations"
                       % (SAMPLE_SIDE, its)),
            "all_cores": {"value": allc, "cores": procs, "slowest_step_s": slowest,
                          "sample": "one whole step of the same block in each of %d concurrent processes" % procs},
            "nproc": nproc}


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

# What bounds the dominant kernel, from its ncu counters (float64 coarse
# sweeps): the small colour classes of levels 2-3 run at a few per cent
# achieved occupancy with long-scoreboard stalls taking about two thirds of
# the cycles between issues (latency); the level-1 classes keep the float64
# pipe about three quarters busy.
DOMINANT_LIMITER = "latency (small classes: dependent-load chains) and the float64 pipe (level-1 classes)"


def roofline(kind: str, ms: float, launches: int, flops: float, byts: float, peaks: dict, peak_src: str,
             fp64_peak: float):
    """Roofline entry of one kernel kind from its event timing and the
    library's algorithmic flop and byte counts (models stated in ll_mg.h).
    The V-cycle kernels move about 0.18 float64 flop per byte: at the HBM
    roofline they would need about 1.2 TFLOP/s, the float64 pipe's peak, so
    the HBM roof is the lower of the two and is the bound reported; the
    float64 rate is given beside it."""
    avg_ms = ms / max(launches, 1)
    per_launch_flops = flops / max(launches, 1)
    per_launch_bytes = byts / max(launches, 1)
    ach_tf = per_launch_flops / (avg_ms * 1e-3) / 1e12 if avg_ms > 0 else None
    ach_gb = per_launch_bytes / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else None
    return {"bound": "hbm", "achieved": ach_gb, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": (ach_gb / peaks["hbm_gbs"]) if ach_gb else None, "peak_source": peak_src,
            "traffic": None, "kernel_kind": kind, "launches": launches, "avg_launch_ms": avg_ms,
            "flops_per_launch": per_launch_flops, "bytes_per_launch": per_launch_bytes,
            "fp64_tflops": ach_tf, "fp64_frac": (ach_tf / fp64_peak) if ach_tf else None}


def fp64_probe(ll, torch, dev):
    """Measured float64 multiply-add throughput (TFLOP/s, best of 5)."""
    sink = torch.zeros(1, dtype=torch.float64, device=dev)
    blocks = 148 * 8
    ll.fp64_fma_probe(sink, 256, blocks)
    best = 0.0
    stream = torch.cuda.current_stream()
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fl = ll.fp64_fma_probe(sink, 8192, blocks)
        e1.record(stream)
        torch.cuda.synchronize()
        best = max(best, fl / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    return best


def timed_steps(H, m, steps, stream, torch, ll, sampler=None):
    """K steps of m on H between two CUDA events on `stream` (no profiling
    scopes are active); returns (ms, iterations, relres, launches, clocks)."""
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    its, rrs = [], []
    launches0 = ll.launch_count()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    ev0.record(stream)
    for _ in range(steps):
        st, it, rr = H.step(m, 1)
        its += it
        rrs += rr
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    return ev0.elapsed_time(ev1), its, rrs, ll.launch_count() - launches0, clocks


def run_ours(args):
    import ctypes

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
    stream = torch.cuda.current_stream()
    lib = ll.load_library()
    prec_code = {"fp64": ll.LL_FP64, "mixed": ll.LL_MIXED_FP32, "bf16": ll.LL_MIXED_BF16}
    m0 = inputs.vortex(*GRID, seed=0).reshape(-1)

    def hierarchy(m, precision):
        return ll.Hierarchy(m, ALPHA, DT, H_SPACING, GRID, ll.Params(rtol=RTOL, precision=prec_code[precision],
                                                                     kcycle=args.kcycle))

    # ---- the headline: K steps, no instrumentation -------------------------
    m = torch.tensor(m0, device=dev)
    t0 = time.perf_counter()
    H = hierarchy(m, args.precision)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        H.step(m, 1)
    m_start = m.clone()  # the end-to-end leg repeats these K steps from here
    if world > 1:
        dist.barrier()
    elapsed_ms, its, rrs, launches, clocks = timed_steps(H, m, args.steps, stream, torch, ll, ClockSampler(local))
    if world > 1:
        dist.barrier()
    elapsed_ms = max_over_ranks(elapsed_ms, dev)

    # ---- the precisions side by side on the same K steps --------------------
    # Every hierarchy set up after a second one in the same process runs about
    # 2 % slower than the first (measured; not from allocations, streams,
    # events, pinned memory or module loading), so the headline (the first
    # hierarchy) is not compared with later ones: the three precisions are
    # timed here one after another in the same process state, and the
    # speed-ups divide these.
    others = {}
    if not args.no_mixed:
        for prec in ("fp64", "mixed", "bf16"):
            mp_ = torch.tensor(m0, device=dev)
            Hp = hierarchy(mp_, prec)
            for _ in range(args.warmup):
                Hp.step(mp_, 1)
            ms_p, its_p, rrs_p, _, clk_p = timed_steps(Hp, mp_, args.steps, stream, torch, ll, ClockSampler(local))
            ms_p = max_over_ranks(ms_p, dev)
            # error against the float64 path: one step from the same state
            ma, mb = torch.tensor(m0, device=dev), torch.tensor(m0, device=dev)
            hierarchy(ma, "fp64").step(ma, 1)
            hierarchy(mb, prec).step(mb, 1)
            others[prec] = {"value": replica_throughput(UNKNOWNS * args.steps, world, ms_p * 1e-3),
                            "ms_per_step": ms_p / args.steps,
                            "iterations_per_step": float(np.mean(its_p)), "max_relres": float(max(rrs_p)),
                            "error_vs_fp64": float(torch.linalg.norm(mb - ma) / torch.linalg.norm(ma)),
                            "clocks_sm_mhz": clk_p["sm_mhz"], "clock_reasons": clk_p["reasons"]}
            del Hp, mp_, ma, mb
            torch.cuda.empty_cache()
        fp64_ms = others["fp64"]["ms_per_step"]
        for prec in ("mixed", "bf16"):
            others[prec]["speedup_vs_fp64"] = fp64_ms / others[prec]["ms_per_step"]

    # ---- profiling pass: per-kind breakdown, then the dominant kind alone ----
    def prof_start(mask):
        lib.ll_mg_profile(H._h, ctypes.c_uint(mask))

    def prof_read(kind):
        ms, cnt, fl, by = ctypes.c_double(0), ctypes.c_longlong(0), ctypes.c_double(0), ctypes.c_double(0)
        lib.ll_mg_profile_read(H._h, kind, ctypes.byref(ms), ctypes.byref(cnt), ctypes.byref(fl), ctypes.byref(by))
        return ms.value, cnt.value, fl.value, by.value

    prof_steps = max(1, min(args.steps, 5))
    prof_start((1 << len(KIND_NAMES)) - 1)
    pits = []
    for _ in range(prof_steps):
        pits += H.step(m, 1)[1]
    breakdown = {KIND_NAMES[k]: prof_read(k) for k in range(len(KIND_NAMES))}
    dominant = max((k for k in KIND_NAMES if k != "numeric"), key=lambda k: breakdown[k][0])
    prof_start(1 << KIND_NAMES.index(dominant))
    for _ in range(prof_steps):
        H.step(m, 1)
    dom = prof_read(KIND_NAMES.index(dominant))
    prof_start(0)

    # ---- end to end: the headline's K steps again, the field in pinned host
    # memory, through ll_mg_step_host (one call per step: the library copies
    # the field in and out every step).  The W warm-up steps are repeated
    # first, untimed, from the initial field (a field that is not the last
    # output starts a fresh history), so that the timed steps start from the
    # same state with the same earlier states behind their initial
    # approximations as the headline's ---------------------------------------
    e2e_steps = args.steps
    H.step_host(m.detach().cpu().pin_memory(), 1)  # first call allocates the device copy
    mh = torch.tensor(m0).pin_memory()
    for _ in range(args.warmup):
        H.step_host(mh, 1)
    e2e_start_err = float(torch.abs(mh - m_start.cpu()).max())
    e2e_its = []
    torch.cuda.synchronize()
    te = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_its += H.step_host(mh, 1)[1]
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - te, dev)

    fp64_meas = fp64_probe(ll, torch, dev)
    if rank != 0:
        return
    value = replica_throughput(UNKNOWNS * args.steps, world, elapsed_ms * 1e-3)
    peaks, peak_src = measured_peaks()
    fp64_peak = max(fp64_meas, 1e-9)
    roof = roofline(dominant, *dom, peaks, peak_src, fp64_peak)
    roof["limiter"] = DOMINANT_LIMITER if dominant == "bsr_smooth" else None
    roof["timed_in"] = "a separate profiling pass of %d steps right after the timed region" % prof_steps
    if dominant == "bsr_smooth" and args.precision == "fp64":
        roof["traffic"] = KB_SWEEP_TRAFFIC_RATIO * roof["bytes_per_launch"]
        roof["traffic_source"] = ("ncu DRAM bytes of ks_sweep and kb_sweep launches at 96^3 / algorithmic bytes, "
                                  "weighted by a V-cycle's bytes = %.3f, times this launch's algorithmic bytes"
                                  % KB_SWEEP_TRAFFIC_RATIO)
    vk = [k for k in VCYCLE_KINDS]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "mixed": "f32+f64", "bf16": "bf16+f32+f64"}[args.precision],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": list(GRID), "h": H_SPACING, "alpha": ALPHA, "dt": DT,
                   "rtol": RTOL, "precision": args.precision, "kcycle": args.kcycle,
                   "parallelism": "replicas" if world > 1 else "single", "levels": H.levels,
                   "initial_guess": "m^n and up to 6 earlier states extrapolated with the backward-difference "
                                    "terms that keep shrinking (m^n for a fresh integration's first step)",
                   "l2": "inputs larger than L2: the working set per step (~3 GB: GCR bases, operators) exceeds "
                         "the 126 MB L2"},
        "iterations_per_step": {"mean": float(np.mean(its)), "min": int(min(its)), "max": int(max(its))},
        "max_relres": float(max(rrs)),
        "setup_s": setup_s,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "roofline": roof,
        "precisions": others,
        # the mixed-precision configuration: a float32 V-cycle with bfloat16
        # coarse-level operators inside float64 GCR
        "mixed_vs_fp64_speedup": others.get("bf16", {}).get("speedup_vs_fp64"),
        "mixed_config": "bf16: float32 V-cycle, bfloat16 coarse-level operators, float64 GCR",
        "fp32_vcycle_vs_fp64_speedup": others.get("mixed", {}).get("speedup_vs_fp64"),
        "fp64_peak": {"measured_tflops": fp64_meas, "derived_tflops": FP64_PEAK_TFLOPS,
                      "probe": "ll_fp64_fma_probe: 1184 blocks x 256 threads x 8 chains x 8192 FMA, best of 5"},
        "kernel_breakdown_ms_per_step": {k: round(v[0] / prof_steps, 3) for k, v in breakdown.items()},
        "kernel_launches_per_iteration": {k: round(v[1] / max(sum(pits), 1), 2) for k, v in breakdown.items()},
        "profiling_pass": {"steps": prof_steps, "iterations": int(sum(pits))},
        # the V-cycle's kernels together (algorithmic bytes over their event time)
        "vcycle_hbm_gbs": (sum(breakdown[k][3] for k in vk) / max(sum(breakdown[k][0] for k in vk), 1e-9) / 1e6),
        "numeric_setup_ms_per_step": breakdown["numeric"][0] / prof_steps,
        "kernel_roofline": {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv)
                                for kk, vv in roofline(k, *breakdown[k], peaks, peak_src, fp64_peak).items()
                                if kk in ("achieved", "frac", "fp64_tflops", "fp64_frac")}
                            for k in KIND_NAMES if breakdown[k][1] > 0},
        "e2e": {"value": replica_throughput(UNKNOWNS * e2e_steps, world, e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": UNKNOWNS * 8 * world, "d2h_bytes_per_step": UNKNOWNS * 8 * world,
                "steps": e2e_steps, "iterations_per_step": float(np.mean(e2e_its)),
                "api": "ll_mg_step_host (pinned host field, copies inside the library), the W warm-up steps "
                       "again untimed from the initial field, then the timed K steps, host wall clock",
                "start_state_max_abs_diff": e2e_start_err},
    }
    if not args.no_other_workloads:
        line["other_workloads"] = other_workloads(ll, torch, inputs, dev)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the other workloads, measured compactly in the default run
# ---------------------------------------------------------------------------
TUNING_CACHE = os.path.join(ROOT, "paper_2608_09102_b300", "tuning", "batch512_mixed.txt")
# stagnation stop of the batch workloads: an instance whose true residual at
# a restart is above 0.99 of its value 20 iterations earlier stops as not
# converged (on the oracle, every instance of the 512-instance recipe that
# converges is below 0.5 of its starting residual after 20 iterations, and
# the ones that never do stay above 0.68 from iteration 20 to 300)
STALL_WINDOW, STALL_RATIO = 20, 0.99


def _event_ms(torch, fn):
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), out


def other_workloads(ll, torch, inputs, dev):
    """One compact measurement of each other workload of the list (device
    time by CUDA events on the current stream; every call synchronises):
    the 64^2 solve against a dense-LU-sized problem, the 256^2 x 128 random
    unit vectors with the mixed configuration (K-cycle on level 1), the
    512-instance ragged batch with the autotuner's stored choices, and the
    96^3 gradient.  A workload whose call fails is recorded with its error
    and the others still run."""
    out = {}
    for name, leg in (("config1_64x64", _leg_config1), ("config3_256x256x128_mixed_kcycle1", _leg_config3),
                      ("config4_batch512_mixed_autotuned", _leg_config4), ("config5_grad96_fp64", _leg_config5)):
        try:
            out[name] = leg(ll, torch, inputs, dev)
        except ll.LLError as e:
            out[name] = {"error": str(e)}
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    return out


def _leg_config1(ll, torch, inputs, dev):
    """2-D 64^2, alpha 0.1, dt 1e-3, one solve to 1e-10."""
    g1 = (64, 64, 1)
    m1 = torch.tensor(inputs.smooth_field(*g1, seed=0).reshape(-1), device=dev)
    H1 = ll.Hierarchy(m1, 0.1, 1e-3, 1 / 64, g1, ll.Params(rtol=1e-10))
    b1 = m1 / 1e-3
    x1 = torch.zeros_like(b1)
    H1.solve(b1, x1)
    x1.zero_()
    ms, (st, it, rr) = _event_ms(torch, lambda: H1.solve(b1, x1))
    return {"ms_per_solve": ms, "iterations": it, "relres": rr, "status": st,
            "unknown_solves_per_s": 3 * 64 * 64 / (ms * 1e-3)}


def _leg_config3(ll, torch, inputs, dev):
    """256 x 256 x 128 random unit vectors, h 1/256, dt 1e-4, three alphas."""
    g3 = (256, 256, 128)
    m3 = torch.tensor(inputs.random_sphere(*g3, seed=0).reshape(-1), device=dev)
    b3 = m3 / 1e-4
    c3 = {}
    for alpha in (0.01, 0.1, 1.0):
        H3 = ll.Hierarchy(m3, alpha, 1e-4, 1 / 256, g3, ll.Params(rtol=1e-8, kcycle=1, precision=ll.LL_MIXED_BF16))
        x3 = torch.zeros_like(b3)
        H3.solve(b3, x3)
        x3.zero_()
        ms, (st, it, rr) = _event_ms(torch, lambda: H3.solve(b3, x3))
        c3["alpha_%g" % alpha] = {"ms_per_solve": ms, "iterations": it, "relres": rr, "status": st,
                                  "unknown_solves_per_s": 3 * 256 * 256 * 128 / (ms * 1e-3)}
        del H3, x3
    return c3


def _leg_config4(ll, torch, inputs, dev):
    """The ragged 512-instance batch with the autotuner's stored choices,
    with the stagnation stop (instances whose residual no longer falls stop
    as not converged) and, for comparison, without it."""
    spec = inputs.batch_instances(BATCH_COUNT, seed=0)
    ms4 = [torch.tensor(inputs.smooth_field(*q["grid"], seed=q["seed"]).reshape(-1), device=dev) for q in spec]
    al, dts = [q["alpha"] for q in spec], [q["dt"] for q in spec]
    hs, grids = [q["h"] for q in spec], [q["grid"] for q in spec]
    rhs = [m / d for m, d in zip(ms4, dts)]
    xs = [torch.zeros_like(m) for m in ms4]
    out = {}
    for key, window in (("stall_stop", STALL_WINDOW), ("without_stall_stop", 0)):
        base = ll.Params(rtol=RTOL, precision=ll.LL_MIXED_FP32, maxit=300, stall_window=window,
                         stall_ratio=STALL_RATIO)
        with tempfile.TemporaryDirectory() as td:  # a copy: the stored file is never rewritten
            cache = os.path.join(td, "tune.txt")
            with open(TUNING_CACHE) as f, open(cache, "w") as g:
                g.write(f.read())
            per, tuned = ll.autotune(ms4, al, dts, hs, grids, base=base, cache_path=cache)
        B = ll.Batch(ms4, al, dts, hs, grids, per)

        def bstep():
            B.update(ms4, al, dts)
            for x in xs:
                x.zero_()
            return B.solve(rhs, xs)

        bstep()
        ms, (st, its, rrs, sts) = _event_ms(torch, lambda: [bstep() for _ in range(2)][-1])
        conv = sum(1 for v in sts if v == ll.LL_OK)
        solved = 3 * sum(int(np.prod(q["grid"])) for q, v in zip(spec, sts) if v == ll.LL_OK)
        out[key] = {"ms_per_step": ms / 2, "converged": conv, "instances": len(spec), "classes_tuned_now": tuned,
                    "groups": B.groups, "converged_unknown_solves_per_s": solved / (ms / 2 * 1e-3),
                    "stall_window": window, "stall_ratio": STALL_RATIO if window else None,
                    "iterations_max": int(max(its))}
        B.close()
        del B
        torch.cuda.synchronize()
    return out


def _leg_config5(ll, torch, inputs, dev):
    """The 96^3 gradient (20 steps, checkpoints every 5)."""
    g5, n5 = (96, 96, 96), 96 ** 3
    m0 = torch.tensor(inputs.smooth_field(*g5, seed=0).reshape(-1), device=dev)
    mt = torch.tensor(inputs.smooth_field(*g5, seed=1).reshape(-1), device=dev)

    def grad():
        m = m0.clone().requires_grad_(True)
        a = torch.tensor(0.1, dtype=torch.float64, requires_grad=True)
        mN = ll.steps_autograd(m, a, 20, 1e-3, 1 / 96, g5, ll.Params(rtol=RTOL), checkpoint=5)
        loss = 0.5 * torch.sum((mN - mt) ** 2)
        loss.backward()
        return float(loss.detach())

    grad()
    ms, loss = _event_ms(torch, grad)
    return {"ms_per_gradient": ms, "loss": loss, "unknown_solves_per_s": 60 * 3 * n5 / (ms * 1e-3)}


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
    params = ll.Params(rtol=RTOL, precision=precision, maxit=args.batch_maxit, stall_window=args.stall_window,
                       stall_ratio=STALL_RATIO)
    hs, grids = [s["h"] for s in spec], [s["grid"] for s in spec]
    tune_s, tuned, per = None, 0, params
    if not args.no_autotune:  # per class of instances: cycle and coarse-kernel shape
        t0 = time.perf_counter()
        if args.tune_cache:  # earlier choices reused, new classes added
            per, tuned = ll.autotune(ms, alphas, dts, hs, grids, base=params, cache_path=args.tune_cache)
        else:  # tuned from scratch
            with tempfile.TemporaryDirectory() as td:
                per, tuned = ll.autotune(ms, alphas, dts, hs, grids, base=params,
                                         cache_path=os.path.join(td, "tune.txt"))
        tune_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    B = ll.Batch(ms, alphas, dts, hs, grids, per)
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
                   "stall_stop": {"window": args.stall_window, "ratio": STALL_RATIO} if args.stall_window else None,
                   "l2": "working set (~6 GB) exceeds the 126 MB L2"},
        "converged": len(conv), "unknowns_converged": solved,
        "not_converged": [{"side": spec[k]["grid"][0], "alpha": spec[k]["alpha"], "dt": spec[k]["dt"],
                           "status": sts[k], "relres": rrs[k], "iterations": its[k]}
                          for k in range(len(spec)) if sts[k] != ll.LL_OK],
        "iterations": {"mean": float(np.mean(its)), "median": float(np.median(its)), "max": int(max(its)),
                       "lockstep": int(max(its))},
        "levels": B.levels, "setup_s": setup_s, "gpu_launches": int(launches), "clocks": clocks,
        "autotune": None if args.no_autotune else {
            "classes_tuned": tuned, "tune_s": tune_s, "groups": B.groups,
            "choices": sorted({(p.nu_pre, p.nu_post, p.kcycle, p.coarse_lanes, p.coarse_block) for p in per}),
            "key": "(grid, floor(log2(dt/h^2))); candidates V(1,1), V(2,2), K1+V(1,1), K1+V(2,2), then lanes 8 "
                   "and/or 128-thread blocks"},
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
    ap.add_argument("--no-mixed", action="store_true", help="time only the --precision path")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="skip the compact measurements of the other workloads of the list")
    ap.add_argument("--workload", choices=["step128", "batch512", "grad96"], default="step128",
                    help="step128: the 128^3 time-stepping workload; batch512: the ragged batch; "
                         "grad96: the 96^3 differentiation workload")
    ap.add_argument("--batch-count", type=int, default=BATCH_COUNT)
    ap.add_argument("--batch-maxit", type=int, default=300)
    ap.add_argument("--stall-window", type=int, default=STALL_WINDOW,
                    help="batch512: stagnation stop window in iterations (0: off)")
    ap.add_argument("--no-autotune", action="store_true", help="batch512: one parameter set for every instance")
    ap.add_argument("--tune-cache", default=None, help="batch512: the autotuner's cache file (default: a fresh one)")
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
