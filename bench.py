"""Throughput of the fused D2Q5Q4Q4 step (MLUPS and fraction of the HBM roofline).

Workload: the 2D unsteady circular dam-break on a 4096 x 4096 periodic grid (depth 2
inside radius 0.2 of the centre of the unit square, 1 outside, at rest, plus a seeded
uniform perturbation of +-1e-3), D2Q5Q4Q4 with lambda = 8, s = 1.8, a = 0.05, g = 1,
FP32 populations.  One bench step is one time step of the scheme over the whole grid
(pull streaming, boundaries, moments, equilibria, relaxation), run by the library's
default kernel for this workload: temporal blocking, 6 time steps per launch of one
fused kernel that updates two cells per thread with paired FP32 instructions (results
bit-identical to one step per launch).  The two 872 MB population
buffers exceed the 129 MB L2, so every launch streams the state from HBM and back.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line on rank 0.  Under torchrun (N > 1) the grid is split into N bands of
rows, one per GPU, with ghost rows exchanged over NCCL (strong scaling; --replicas runs
independent replicas instead); `value` is the whole grid's cell updates per second.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "MLUPS and % of HBM roofline per step (FP32 vs FP64, batched vs plain) at stated L1 error"
UNIT = "MLUPS"
N = 4096
LAM, S_RATE, A_REST = 8.0, 1.8, 0.05
BYTES_PER_LUP = {"f32": 104.0, "f64": 208.0}  # 13 populations read + 13 written
WORKLOAD = ("2D circular dam-break 4096x4096 periodic, D2Q5Q4Q4 (13 populations), "
            "lambda=8 s=1.8 a=0.05 g=1, h=2 for r<0.2 else 1 plus U[-1e-3,1e-3]")
JOB_STEPS = 1000  # steps of the workload as one job (the end-to-end unit)
REF_SAMPLE = 512   # side of the periodic window the CPU oracle advances per reference step

# One-step kernels by (variant, dtype).
KERNEL_NAMES = {(2, "f32"): "step2d_vec<float>", (2, "f64"): "step2d_vec<double>"}


def temporal_kernel_name(k: int, cells: int = 4096 * 4096) -> str:
    """The periodic temporal kernel the library launches for an even-width grid."""
    if k % 2:
        return f"step2d_temporal_periodic<{k}, 192>"
    if k == 6:
        return f"step2d_temporal_periodic_x2<6, {128 if cells < 2 ** 23 else 256}, 1, 0, 1>"
    return f"step2d_temporal_periodic_x2<{k}, 256, 2>" if k <= 4 else f"step2d_temporal_periodic_x2<{k}, 192, 1>"


# DRAM traffic per launch of each timed kernel on the 4096^2 workload from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), keyed by kernel name, valid only for the
# kernel sources it was taken on.
NCU_TRAFFIC = {
    "step2d_temporal_periodic_x2<6, 256, 1, 0, 1>": {
        "src_sha256": "80e7ae7f74be93879b84e2497f4374045768ef0edce63502b5c6969ca2b8cb60",
        "sources": ("temporal.cu", "temporal.cuh", "temporal_pair.cuh", "scheme.cuh"), "bytes_per_launch": 1745.18e6,
        "case": "ncu dram__bytes_read.sum + dram__bytes_write.sum (1 pass) of the 5 launches of "
                "bench.py --quick --skip-cpu --steps 12 --warmup 3 (4096x4096): 921.25 MB read + 823.93 MB "
                "written per launch (mean)"},
}

def kernel_source_hash(sources=("kernels_2d.cu", "scheme.cuh", "internal.h")) -> str:
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, "paper_1401_0427_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (every 100 ms) of SM clock and throttle reasons."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.perf_counter(), line.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)

    def summary(self, t0: float, t1: float):
        rows = [s for (t, s) in self.samples if t0 - 0.15 <= t <= t1 + 0.15]
        if not rows:
            rows = [s for (_, s) in self.samples]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            parts = [p.strip() for p in r.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- distributed
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def _all_reduce(world, value: float, op: str) -> float:
    """value reduced over the ranks (op "max" or "sum"); on the process group's device (CUDA
    for NCCL, host memory for gloo)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(world, value: float) -> float:
    return _all_reduce(world, value, "max")


def sum_over_ranks(world, value: float) -> float:
    return _all_reduce(world, value, "sum")


def job_throughput(world, units: float, ms: float) -> tuple[float, float]:
    """Whole-job throughput of replicas: the units of every rank over the slowest rank's time.
    Returns (value in units per microsecond, max time in ms)."""
    slowest = max_over_ranks(world, ms)
    return sum_over_ranks(world, units) / (slowest * 1e-3) / 1e6, slowest


# ----------------------------------------------------------------- CPU oracle
def cpu_oracle_mlups(W0, target_seconds: float = 15.0, max_steps: int = 120):
    """The FP64 oracle as it stands, on all host cores, over the full 4096^2 grid for
    a bounded number of steps (about target_seconds of CPU work)."""
    import oracle

    cores = oracle.set_threads(0)
    p = oracle.params(N, N, lam=LAM, s=S_RATE, a=A_REST)
    F = oracle.equilibrium_2d(*W0, p)
    F = oracle.run_2d(F, 1, p)  # first step pays the page faults of the work arrays
    t = time.perf_counter()
    F = oracle.run_2d(F, 1, p)
    t1 = time.perf_counter() - t
    steps = int(max(1, min(max_steps, math.ceil(target_seconds / max(t1, 1e-3)))))
    t = time.perf_counter()
    F = oracle.run_2d(F, steps, p)
    dt = time.perf_counter() - t
    h = oracle.moments_2d(F, p)[0]
    return {"value": N * N * steps / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle, the full 4096x4096 grid of the workload for {steps} steps "
                      f"({dt:.1f} s, OpenMP over rows)"}, (steps + 2, h)


def fp32_error_against_oracle(W0, oracle_run, stream, lbm_sw, torch):
    """Relative L1 of h between the library's FP32 run (default kernel) and the FP64
    oracle's run of the same steps on the full grid (the oracle state timed for the CPU
    baseline)."""
    steps, oh = oracle_run
    with lbm_sw.Simulation(N, N, precision=lbm_sw.FP32, lam=LAM, s=S_RATE, a=A_REST, stream=stream.cuda_stream) as sim:
        sim.set_state(*W0)
        sim.step(steps)
        gh = sim.moments()[0]
    return {"relative_l1_h": float(np.abs(gh - oh).sum() / np.abs(oh).sum()), "steps": steps,
            "against": f"the FP64 oracle run of the same {steps} steps on the full 4096x4096 grid "
                       "(the state timed for cpu_baseline)", "bar": 1e-5}


def _time_oracle(fn, min_seconds: float = 0.5):
    """Run fn() until min_seconds have passed; return (calls, seconds)."""
    calls, t0 = 0, time.perf_counter()
    while True:
        fn()
        calls += 1
        dt = time.perf_counter() - t0
        if dt >= min_seconds:
            return calls, dt


def cpu_oracle_configs():
    """The FP64 oracle on the other workloads, each on a bounded sample, on one core and on
    every core (MLUPS = cells x steps / s of oracle time)."""
    import oracle
    from paper_1401_0427_gb300 import inputs

    out = {}
    all_cores = oracle.set_threads(0)
    cases = []
    # 1D shock tube: the whole 1000-cell, 500-step run
    p1 = oracle.params(1000, a=0.15, lam=LAM, s=S_RATE, bc=(oracle.WALL, oracle.WALL))
    h, q = inputs.dam_break_1d(1000)
    F1 = oracle.equilibrium_1d(h, q, p1)
    cases.append(("shock_tube_1d_1000", 1000 * 500, lambda: oracle.run_1d(F1, 500, p1),
                  "the whole run: 1000 cells x 500 steps"))
    # 2D shock reflection 512^2: 20 of its 2000 steps
    n = 512
    uL = inputs.shock_speed_state(2.0, 1.0)
    p2 = oracle.params(n, n, lam=LAM, s=S_RATE, a=A_REST, bc=(oracle.INFLOW, oracle.WALL, oracle.PERIODIC, oracle.PERIODIC),
                       inflow=[(2.0, 2.0 * uL, 0.0)] * 4)
    F2 = oracle.equilibrium_2d(*inputs.planar_shock_2d(n, n), p2)
    cases.append(("shock_reflection_512", n * n * 20, lambda: oracle.run_2d(F2, 20, p2),
                  "20 of the 2000 steps on the full 512x512 grid"))
    # batched ensemble: 8 of the 256 instances (every 32nd), 10 steps
    table = inputs.batched_instances(256)[::32]
    bstates = []
    for k, hin, r in table:
        pb = oracle.params(k, k, lam=LAM, s=S_RATE, a=A_REST)
        bstates.append((pb, oracle.equilibrium_2d(*inputs.circular_dam_break_2d(k, seed=None, h_in=hin, radius=r), pb)))
    bcells = sum(k * k for k, _, _ in table)
    cases.append(("batched_256", bcells * 10, lambda: [oracle.run_2d(F, 10, pb) for pb, F in bstates],
                  f"every 32nd of the 256 instances ({bcells} cells), 10 steps each"))
    for name, lups, fn, sample in cases:
        entry = {"sample": sample, "unit": UNIT, "kind": "oracle"}
        for label, threads in (("one_core", 1), ("all_cores", 0)):
            cores = oracle.set_threads(threads)
            calls, dt = _time_oracle(fn)
            entry[label] = {"MLUPS": lups * calls / dt / 1e6, "cores": cores}
        out[name] = entry
    oracle.set_threads(all_cores)
    out["adjoint_1024"] = {"sample": "none: the oracle has no adjoint; its complex-step derivative gives one "
                                     "directional derivative per run, not a gradient"}
    return out


def run_reference(args, world, rank):
    """The oracle on the host cores: each bench step advances a 512x512 periodic window
    of the workload's initial field by one step (a bounded sample of the workload)."""
    if rank != 0:
        return
    import oracle
    from paper_1401_0427_gb300 import inputs

    cores = oracle.set_threads(0)
    h, hu, hv = inputs.circular_dam_break_2d(N, seed=inputs.stream_seed(3))
    c0 = N // 2 - REF_SAMPLE // 2
    win = [np.ascontiguousarray(x[c0:c0 + REF_SAMPLE, c0:c0 + REF_SAMPLE]) for x in (h, hu, hv)]
    p = oracle.params(REF_SAMPLE, REF_SAMPLE, lam=LAM, s=S_RATE, a=A_REST)
    F = oracle.equilibrium_2d(*win, p)
    for _ in range(args.warmup):
        F = oracle.run_2d(F, 1, p)
    t = time.perf_counter()
    for _ in range(args.steps):
        F = oracle.run_2d(F, 1, p)
    dt = time.perf_counter() - t
    value = REF_SAMPLE * REF_SAMPLE * args.steps / dt / 1e6
    sample = (f"FP64 oracle on a {REF_SAMPLE}x{REF_SAMPLE} periodic window (centre) of the workload, "
              f"one step per bench step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ----------------------------------------------------------------- our arm
def run_split(args, world, rank, local):
    """N > 1: the one 4096^2 grid split into N bands of rows, one per GPU (strong scaling),
    6 ghost rows per cut refreshed over NCCL after every fused launch of 6 steps
    (paper_1401_0427_gb300/decomposition.py).  value = cells x steps of the whole grid over
    the slowest rank's time."""
    global N
    import torch
    import torch.distributed as dist

    N = args.side
    torch.cuda.set_device(local)
    dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1401_0427_gb300 import build as libbuild
    from paper_1401_0427_gb300 import decomposition as dc
    from paper_1401_0427_gb300 import inputs, lbm_sw

    if rank == 0:
        libbuild.build()
    dist.barrier()
    libbuild.build()
    stream = torch.cuda.current_stream()
    W0 = inputs.circular_dam_break_2d(N, seed=inputs.stream_seed(3))
    band = dc.Band(N, N, rank, world, halo=6, lam=LAM, s=S_RATE, a=A_REST, stream=stream.cuda_stream)
    strips = dc.DistributedStrips(band)
    band.set_state(*W0)
    unit = max(1, band.sim.info().steps_per_launch)
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    gpu_index = int(vis.split(",")[local]) if vis and vis.split(",")[local].strip().isdigit() else local
    clocks = ClockSampler(gpu_index)
    clocks.start()
    time.sleep(0.3)  # the sampler is running before the warm-up, so no idle gap precedes the timed region
    strips.step(max(args.warmup, 3) * unit)
    torch.cuda.synchronize()
    launches0 = band.sim.info().kernel_launches
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    e0.record(stream)
    strips.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.perf_counter()
    dist.barrier()
    time.sleep(0.2)
    clocks.stop()
    ms = e0.elapsed_time(e1)
    launches = band.sim.info().kernel_launches - launches0
    value, total_ms = job_throughput(world, N * N * args.steps / world, ms)
    diag = strips.diagnostics()
    peak, peak_kind = measured_peaks()
    local_cells = N * band.L.local_ny
    achieved = BYTES_PER_LUP["f32"] * local_cells * (args.steps / unit) / (ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "peak_kind": f"{peak_kind} (copy bandwidth)", "per": "rank (its band with ghost rows)",
                "kernel": temporal_kernel_name(unit, local_cells), "steps_per_launch": unit}
    # whole jobs through the public API: upload W0, JOB_STEPS steps, download h, hu, hv
    pinned = [torch.empty((band.L.local_ny, N), dtype=torch.float64, pin_memory=True) for _ in range(3)]
    rows = band.local_rows()
    for t, w in zip(pinned, W0):
        t.numpy()[...] = w[rows]
    out = [torch.empty((band.L.local_ny, N), dtype=torch.float64, pin_memory=True) for _ in range(3)]
    dist.barrier()
    torch.cuda.synchronize()
    t = time.perf_counter()
    jobs = 2
    for _ in range(jobs):
        band.sim.set_state(*[p.numpy() for p in pinned])
        strips.step(JOB_STEPS)
        band.sim.moments_into(*[o.numpy() for o in out])
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t) * 1e3
    e2e_value, _ = job_throughput(world, N * N * JOB_STEPS * jobs / world, e2e_ms)
    band.sim.close()
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": N, "ny": N, "cells": N * N, "precision": "FP32 populations",
                       "l2": "inputs larger than L2 (each band's two population buffers exceed the 129 MB L2)",
                       "parallelism": f"{world} bands of rows, 6 ghost rows per cut, NCCL exchange every 6 steps"},
            "roofline": roofline, "gpu_launches": int(launches), "clocks": clocks.summary(t_wall0, t_wall1),
            "conservation": {"sum_h": diag[0], "min_h": diag[3]},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 3 * N * N * 8,
                    "d2h_bytes_per_step": 3 * N * N * 8, "step": f"one job: upload W0, {JOB_STEPS} steps, download W"},
        }))
    dist.destroy_process_group()


def run_ours(args, world, rank, local):
    global N
    import torch

    N = args.side
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1401_0427_gb300 import build as libbuild
    from paper_1401_0427_gb300 import inputs, lbm_sw

    libbuild.build()
    stream = torch.cuda.current_stream()
    W0 = inputs.circular_dam_break_2d(N, seed=inputs.stream_seed(3))
    cells = N * N
    prec = lbm_sw.FP64 if args.precision == "fp64" else lbm_sw.FP32
    dt_name = "f64" if prec == lbm_sw.FP64 else "f32"

    kernel = {"auto": lbm_sw.KERNEL_AUTO, "vec": lbm_sw.KERNEL_VEC, "temporal": lbm_sw.KERNEL_TEMPORAL}[args.kernel]
    sim = lbm_sw.Simulation(N, N, precision=prec, lam=LAM, s=S_RATE, a=A_REST, stream=stream.cuda_stream,
                            kernel=kernel, temporal_steps=args.temporal_steps)
    sim.set_state(*W0)
    info = sim.info()
    unit = max(1, info.steps_per_launch)  # steps per launch of the step kernel
    kname = temporal_kernel_name(unit, cells) if unit > 1 else KERNEL_NAMES[(lbm_sw.KERNEL_VEC, dt_name)]
    # The timed region is exactly --steps time steps, launched as lbm_sw_step(steps) does
    # (lbm_sw_step_plan: launches of `unit` steps, the tail split into shorter fused
    # launches; bit-identical results).  Each planned launch is issued by its own call; an
    # event is recorded only where the launch size changes (an event between two launches
    # would keep the second from starting during the first one's tail), so the launches of
    # the dominant kernel are timed as one group.
    plan = sim.step_plan(args.steps)
    if any(sim.step_plan(k) != [k] for k in set(plan)):
        plan = [args.steps]  # a size that one call would split: time the whole call instead
    groups = []  # (launch size, count), in plan order
    for k in plan:
        if groups and groups[-1][0] == k:
            groups[-1][1] += 1
        else:
            groups.append([k, 1])
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    gpu_index = int(vis.split(",")[local]) if vis and vis.split(",")[local].strip().isdigit() else local
    clocks = ClockSampler(gpu_index)
    clocks.start()
    time.sleep(0.3)  # the sampler is running before the warm-up, so no idle gap precedes the timed region

    launches0 = sim.info().kernel_launches
    sim.step(max(args.warmup, 3) * unit)  # warm-up: at least 3 launches of the timed kernel,
    for k in sorted(set(plan) - {unit}):  # and one of each other launch size of the plan
        sim.step(k)
    sim.synchronize()
    warm_launches = sim.info().kernel_launches - launches0

    events = [torch.cuda.Event(enable_timing=True) for _ in range(len(groups) + 1)]
    barrier(world)
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    events[0].record(stream)
    for i, (k, count) in enumerate(groups):
        for _ in range(count):
            sim.step(k)
        events[i + 1].record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.perf_counter()
    barrier(world)
    time.sleep(0.2)
    clocks.stop()

    total_ms = events[0].elapsed_time(events[-1])
    per_launch = [events[i].elapsed_time(events[i + 1]) / count for i, (k, count) in enumerate(groups) if k == unit]
    if not per_launch:
        per_launch = [total_ms * unit / args.steps]
    launches = sim.info().kernel_launches - launches0 - warm_launches
    value, total_ms = job_throughput(world, cells * args.steps, total_ms)
    diag = sim.diagnostics()

    avg_launch_s = float(np.mean(per_launch)) * 1e-3
    peak, peak_kind = measured_peaks()
    achieved = BYTES_PER_LUP[dt_name] * cells / avg_launch_s / 1e9
    entry = NCU_TRAFFIC.get(kname) if N == 4096 else None
    traffic = entry["bytes_per_launch"] if entry and entry["src_sha256"] == kernel_source_hash(entry["sources"]) \
        else None
    per_step_ceiling = peak * 1e9 / BYTES_PER_LUP[dt_name] / 1e6
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_kind": f"{peak_kind} (copy bandwidth)",
                "frac_of_nominal_8tbs": achieved / 8000.0, "kernel": kname, "steps_per_launch": unit,
                "algorithmic_bytes_per_launch": BYTES_PER_LUP[dt_name] * cells,
                "algorithmic_bytes_per_update": BYTES_PER_LUP[dt_name] / unit,
                "mean_launch_ms": float(np.mean(per_launch)),
                "one_step_per_launch_ceiling_MLUPS": per_step_ceiling,
                "value_over_one_step_ceiling": value / world / per_step_ceiling,
                "timed_launches_by_steps": {str(k): plan.count(k) for k in sorted(set(plan), reverse=True)}}
    sim.close()

    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
              "scaling": "weak" if world > 1 else "strong", "vs_baseline": None, "dtype": dt_name,
              "data": "synthetic",
              "config": {"workload": WORKLOAD if N == 4096 else WORKLOAD.replace("4096x4096", f"{N}x{N}"),
                         "nx": N, "ny": N, "cells": cells, "precision": f"{args.precision.upper()} populations",
                         "l2": "inputs larger than L2 (two 872 MB population buffers, 129 MB L2)",
                         "parallelism": "replicas" if world > 1 else "single GPU"},
              "roofline": roofline, "gpu_launches": int(launches),
              "clocks": clocks.summary(t_wall0, t_wall1),
              "conservation": {"sum_h": diag[0], "min_h": diag[3]}}

    if not args.quick:
        result["e2e"] = end_to_end(W0, stream, lbm_sw, torch)  # right after the headline, as the same workload
        result["variants"] = variants(args, W0, stream, lbm_sw, torch)
        result["l1_error"] = result["variants"].pop("_l1")
    if rank == 0 and not args.quick and not args.skip_cpu:
        result["cpu_baseline"], oracle_run = cpu_oracle_mlups(W0)
        result["l1_error"] = {"vs_oracle": fp32_error_against_oracle(W0, oracle_run, stream, lbm_sw, torch),
                              "vs_fp64_gpu": result.get("l1_error")}
        import oracle

        threads = oracle.set_threads(1)
        p512 = oracle.params(512, 512, lam=LAM, s=S_RATE, a=A_REST)
        F1 = oracle.equilibrium_2d(*(np.ascontiguousarray(x[:512, :512]) for x in W0), p512)
        calls, dt = _time_oracle(lambda: oracle.run_2d(F1, 2, p512), 2.0)
        result["cpu_baseline"]["one_core"] = {"MLUPS": 512 * 512 * 2 * calls / dt / 1e6, "cores": threads,
                                              "sample": "a 512x512 periodic corner of the workload, 2 steps a call"}
        oracle.set_threads(0)
        result["cpu_baseline_configs"] = cpu_oracle_configs()
    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def variants(args, W0, stream, lbm_sw, torch):
    """FP64 throughput of the same workload, and the FP32 error against the FP64 run
    (the FP64 path matches the FP64 oracle to 1e-12 in the parity tests)."""
    out = {}
    steps64 = min(args.steps, 200)
    hs = {}
    peak, _ = measured_peaks()
    for name, prec, kernel in (("fp32", lbm_sw.FP32, lbm_sw.KERNEL_AUTO),
                               ("fp32_one_step", lbm_sw.FP32, lbm_sw.KERNEL_VEC),
                               ("fp64", lbm_sw.FP64, lbm_sw.KERNEL_AUTO)):
        sim = lbm_sw.Simulation(N, N, precision=prec, lam=LAM, s=S_RATE, a=A_REST, stream=stream.cuda_stream,
                                kernel=kernel)
        sim.set_state(*W0)
        info = sim.info()
        sim.step(12)
        sim.synchronize()
        n_t = steps64 - steps64 % max(1, info.steps_per_launch)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(n_t)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / n_t
        if name != "fp32_one_step":
            sim.step(JOB_STEPS - 12 - n_t)
            hs[name] = sim.moments()[0]
        sim.close()
        bpl = BYTES_PER_LUP["f64" if name == "fp64" else "f32"]
        spl = max(1, info.steps_per_launch)
        out[name] = {"MLUPS": N * N / (ms * 1e-3) / 1e6, "ms_per_step": ms, "steps_per_launch": spl,
                     "kernel": temporal_kernel_name(spl, N * N) if spl > 1
                     else KERNEL_NAMES[(lbm_sw.KERNEL_VEC, "f64" if name == "fp64" else "f32")],
                     "HBM_GB_per_s": bpl * N * N / spl / (ms * 1e-3) / 1e9,
                     "frac_of_hbm_peak": bpl * N * N / spl / (ms * 1e-3) / 1e9 / peak}
    out["_l1"] = {"relative_l1_h": float(np.abs(hs["fp32"] - hs["fp64"]).sum() / np.abs(hs["fp64"]).sum()),
                  "steps": JOB_STEPS, "against": "the library's FP64 run of the same 1000 steps, which equals the "
                                                 "FP64 oracle's whole run within 1e-12 (tests/test_gpu_configs.py::"
                                                 "test_dam_break_4096_whole_run_matches_oracle)"}
    out["fp32_temporal_k"] = temporal_sweep(W0, stream, lbm_sw, torch)
    out["fp32_closed_basin"] = bounded_variant(W0, stream, lbm_sw, torch)
    out["fp32_mrt"] = mrt_variant(W0, stream, lbm_sw, torch)
    out["fp32_obstacles"] = obstacle_variant(W0, stream, lbm_sw, torch)
    out["batched_256"] = batched_variant(stream, lbm_sw, torch)
    out["shock_reflection_512"] = shock_reflection_variant(stream, lbm_sw, torch)
    out["shock_tube_1d_1000"] = shock_tube_variant(stream, lbm_sw, torch)
    out["adjoint_1024"] = adjoint_variant(stream, lbm_sw, torch)
    return out


def _timed(stream, torch, fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e-3


def temporal_sweep(W0, stream, lbm_sw, torch, steps: int = 840):
    """The same workload at 2 .. 8 fused steps per launch (bit-identical results)."""
    out = {}
    for k in range(2, 9):
        with lbm_sw.Simulation(N, N, precision=lbm_sw.FP32, lam=LAM, s=S_RATE, a=A_REST, stream=stream.cuda_stream,
                               kernel=lbm_sw.KERNEL_TEMPORAL, temporal_steps=k) as sim:
            sim.set_state(*W0)
            sim.step(3 * k)
            n = steps - steps % k
            t = _timed(stream, torch, lambda: sim.step(n))
        out[str(k)] = {"MLUPS": N * N * n / t / 1e6,
                       "HBM_GB_per_s": BYTES_PER_LUP["f32"] * N * N * (n // k) / t / 1e9}
    return out


def bounded_variant(W0, stream, lbm_sw, torch, steps: int = 240):
    """The same dam-break with boundaries: walls on every side (a closed basin), and a channel
    (inflow at x-, outflow at x+, walls at y-+), FP32, the library's kernel choice (the
    two-column temporal kernel, whose edge lanes apply the side rules) against one step per
    launch."""
    W, O, I = lbm_sw.WALL, lbm_sw.OUTFLOW, lbm_sw.INFLOW
    out = {}
    for name, bc in (("walls", (W, W, W, W)), ("channel", (I, O, W, W))):
        for kname, kernel in (("auto", lbm_sw.KERNEL_AUTO), ("one_step", lbm_sw.KERNEL_VEC)):
            with lbm_sw.Simulation(N, N, precision=lbm_sw.FP32, lam=LAM, s=S_RATE, a=A_REST, bc=bc,
                                   inflow=[(1.0, 0.2, 0.0)] * 4, stream=stream.cuda_stream, kernel=kernel) as sim:
                sim.set_state(*W0)
                sim.step(12)
                spl = max(1, sim.info().steps_per_launch)
                t = _timed(stream, torch, lambda: sim.step(steps))
            out[f"{name}_{kname}"] = {"MLUPS": N * N * steps / t / 1e6, "steps_per_launch": spl}
    return out


# MRT rates of the 13 moments of section 3 (the conserved ones ignored): ten distinct values
MRT_RATES = [0.0, 1.1, 1.2, 1.3, 1.4, 0.0, 1.5, 1.6, 1.7, 0.0, 1.75, 1.65, 0.9]


def mrt_variant(W0, stream, lbm_sw, torch, steps: int = 240):
    """The same periodic dam-break with the MRT collision (each moment at its own rate),
    FP32, the library's kernel choice against one step per launch."""
    out = {"rates": MRT_RATES}
    for kname, kernel in (("auto", lbm_sw.KERNEL_AUTO), ("one_step", lbm_sw.KERNEL_VEC)):
        with lbm_sw.Simulation(N, N, precision=lbm_sw.FP32, lam=LAM, s=S_RATE, a=A_REST, stream=stream.cuda_stream,
                               kernel=kernel) as sim:
            sim.set_relaxation(MRT_RATES)
            sim.set_state(*W0)
            sim.step(12)
            spl = max(1, sim.info().steps_per_launch)
            t = _timed(stream, torch, lambda: sim.step(steps))
        out[kname] = {"MLUPS": N * N * steps / t / 1e6, "steps_per_launch": spl}
    return out


def obstacle_variant(W0, stream, lbm_sw, torch, steps: int = 120):
    """The same periodic dam-break with 64 square obstacles (32 x 32 cells each, 0.39 % of the
    grid): the vectorised obstacle kernel (the library's choice) against one thread per cell
    (SIMPLE), one step per launch both."""
    solid = np.zeros((N, N), dtype=np.uint8)
    for i in range(8):
        for j in range(8):
            y, x = 256 + 512 * i - 16, 256 + 512 * j - 16
            solid[y:y + 32, x:x + 32] = 1
    out = {"solid_fraction": float(solid.mean())}
    for kname, kernel in (("auto", lbm_sw.KERNEL_AUTO), ("one_thread_per_cell", lbm_sw.KERNEL_SIMPLE)):
        with lbm_sw.Simulation(N, N, precision=lbm_sw.FP32, lam=LAM, s=S_RATE, a=A_REST, stream=stream.cuda_stream,
                               kernel=kernel) as sim:
            sim.set_obstacle(solid)
            sim.set_state(*W0)
            sim.step(4)
            t = _timed(stream, torch, lambda: sim.step(steps))
        out[kname] = {"MLUPS": N * N * steps / t / 1e6}
    return out


def batched_variant(stream, lbm_sw, torch, steps: int = 500):
    """256 dam-break instances (sides 64..1024, depth U[1.5, 4], radius U[0.1, 0.3]) for 500
    steps in FP32: one batch (autotuned: tile shape and schedule of the one-step tile-list
    kernel, and temporal blocking at K = 4, 6 or 8 steps per launch of a balanced work list)
    against a plain loop over 256 single handles (each with its own default kernel)."""
    from paper_1401_0427_gb300 import inputs

    table = inputs.batched_instances(256)
    sizes = [(n, n) for n, _, _ in table]
    cells = sum(n * n for n, _ in sizes)
    states = [inputs.circular_dam_break_2d(n, seed=None, h_in=hin, radius=r) for n, hin, r in table]
    out = {"instances": 256, "cells": cells, "steps": steps}
    for name, temporal in (("batched", 0), ("batched_one_step", 1)):
        with lbm_sw.Batch(sizes, lam=LAM, s=S_RATE, a=A_REST, stream=stream.cuda_stream, temporal_steps=temporal) as b:
            for i, W0 in enumerate(states):
                b.set_state(i, *W0)
            tune = b.autotune(3)
            b.step(12)
            t = _timed(stream, torch, lambda: b.step(steps))
        k = max(1, tune.temporal_steps)
        gbs = BYTES_PER_LUP["f32"] * cells * steps / k / t / 1e9
        peak, _ = measured_peaks()
        out[name] = {"MLUPS": cells * steps / t / 1e6, "ms_per_step": t / steps * 1e3, "steps_per_launch": k,
                     "HBM_GB_per_s": gbs, "frac_of_hbm_peak": gbs / peak, "tile_rows": tune.tile_rows,
                     "ctas_per_sm": tune.ctas_per_sm, "autotune_candidates": tune.candidates}
    sims = []
    for (n, _), W0 in zip(sizes, states):
        sim = lbm_sw.Simulation(n, n, lam=LAM, s=S_RATE, a=A_REST, stream=stream.cuda_stream)
        sim.set_state(*W0)
        sim.step(2)
        sims.append(sim)
    t_plain = _timed(stream, torch, lambda: [sim.step(steps) for sim in sims])
    for sim in sims:
        sim.close()
    out["plain_loop"] = {"MLUPS": cells * steps / t_plain / 1e6, "ms_per_step": t_plain / steps * 1e3}
    out["speedup_batched_over_plain"] = out["batched"]["MLUPS"] / out["plain_loop"]["MLUPS"]
    return out


def shock_reflection_variant(stream, lbm_sw, torch, steps: int = 2000):
    """512 x 512 planar shock reflected by a wall, 2000 steps, FP32 and FP64 (the state fits
    in L2: this measures L2-resident throughput)."""
    from paper_1401_0427_gb300 import inputs

    n = 512
    uL = inputs.shock_speed_state(2.0, 1.0)
    W0 = inputs.planar_shock_2d(n, n)
    out = {}
    for name, prec in (("fp32", lbm_sw.FP32), ("fp64", lbm_sw.FP64)):
        with lbm_sw.Simulation(n, n, precision=prec, lam=LAM, s=S_RATE, a=A_REST,
                               bc=(lbm_sw.INFLOW, lbm_sw.WALL, lbm_sw.PERIODIC, lbm_sw.PERIODIC),
                               inflow=[(2.0, 2.0 * uL, 0.0)] * 4, stream=stream.cuda_stream) as sim:
            sim.set_state(*W0)
            sim.step(4)
            t = _timed(stream, torch, lambda: sim.step(steps))
        out[name] = {"MLUPS": n * n * steps / t / 1e6, "ms_per_step": t / steps * 1e3}
    return out


def adjoint_variant(stream, lbm_sw, torch, steps: int = 200):
    """Inverse-problem workload: 1024 x 1024 periodic, 8 Gaussian bumps on depth 1, T = 200,
    FP32 states with FP64 checkpoints every ceil(sqrt(T)) steps.  One gradient = recorded
    forward run + adjoint (segment replays + adjoint steps), against 2T plain steps.  Also
    timed: the other end of the tape's memory / time trade-off, one checkpoint interval of
    T steps, where the recorded forward run keeps the moments of every step (T + K slots of
    3 planes) and the backward pass replays nothing."""
    from paper_1401_0427_gb300 import inputs

    n = 1024
    h0 = inputs.gaussian_bumps_2d(n, seed=inputs.stream_seed(5, 5))[0]
    z = np.zeros((n, n))
    with lbm_sw.Simulation(n, n, lam=LAM, s=S_RATE, a=A_REST, stream=stream.cuda_stream) as sim:
        sim.set_state(h0, z, z)
        sim.step(4)
        t_plain = _timed(stream, torch, lambda: sim.step(2 * steps))
        g = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        g += 1e-3
        res = {}
        for interval in (0, steps):
            times = []
            for _ in range(2):
                sim.set_state(h0, z, z)
                tape = lbm_sw.Tape(sim, steps, interval)

                def gradient():
                    tape.record()
                    tape.adjoint(g)

                times.append(_timed(stream, torch, gradient))
                info = tape.info()
                tape.close()
            res[interval] = (min(times), info)
    t_grad, info = res[0]
    t_all, info_all = res[steps]
    return {"cells": n * n, "steps": steps, "interval": info.interval, "checkpoints": info.checkpoints,
            "checkpoint_bytes": info.checkpoint_bytes, "moment_bytes": info.replay_bytes,
            "ms_per_gradient": t_grad * 1e3, "ms_2T_plain_steps": t_plain * 1e3,
            "gradient_over_2T_plain": t_grad / t_plain,
            "interval_T": {"interval": info_all.interval, "checkpoints": info_all.checkpoints,
                           "checkpoint_bytes": info_all.checkpoint_bytes, "moment_bytes": info_all.replay_bytes,
                           "ms_per_gradient": t_all * 1e3, "gradient_over_2T_plain": t_all / t_plain}}


def shock_tube_variant(stream, lbm_sw, torch, steps: int = 500):
    """1D dam-break shock tube, 1000 cells, 500 steps, FP64, walls (latency-bound)."""
    from paper_1401_0427_gb300 import inputs

    n = 1000
    h, q = inputs.dam_break_1d(n)
    with lbm_sw.Simulation(n, 1, dim=1, precision=lbm_sw.FP64, lam=LAM, s=S_RATE, a=0.15,
                           bc=(lbm_sw.WALL, lbm_sw.WALL), stream=stream.cuda_stream) as sim:
        sim.set_state(h, q)
        sim.step(4)
        t = _timed(stream, torch, lambda: sim.step(steps))
    return {"MLUPS": n * steps / t / 1e6, "ms_per_run": t * 1e3, "steps": steps}


def end_to_end(W0, stream, lbm_sw, torch, jobs: int = 4):
    """Whole jobs through the public API with pinned host buffers: upload W0
    (lbm_sw_set_state from host), 1000 steps, download (h, hu, hv) (lbm_sw_get_moments
    to host).  One e2e step = one job."""
    pinned = [torch.empty((N, N), dtype=torch.float64, pin_memory=True) for _ in range(6)]
    src = [p.numpy() for p in pinned[:3]]
    dst = [p.numpy() for p in pinned[3:]]
    for s, w in zip(src, W0):
        s[...] = w
    sim = lbm_sw.Simulation(N, N, precision=lbm_sw.FP32, lam=LAM, s=S_RATE, a=A_REST, stream=stream.cuda_stream)
    # one untimed job first: it captures the handle's CUDA graphs of the step chunks
    sim.set_state(*src)
    sim.step(JOB_STEPS)
    sim.moments_into(*dst)
    torch.cuda.synchronize()
    t = time.perf_counter()
    per_job = []
    for _ in range(jobs):
        tj = time.perf_counter()
        sim.set_state(*src)
        sim.step(JOB_STEPS)
        sim.moments_into(*dst)  # host arrays: returns once the moments are in host memory
        per_job.append((time.perf_counter() - tj) * 1e3)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    # one more job, untimed above, with a synchronize after each phase: where a job's time goes
    phases = {}
    for name, fn in (("upload_ms", lambda: sim.set_state(*src)), ("steps_ms", lambda: sim.step(JOB_STEPS)),
                     ("download_ms", lambda: sim.moments_into(*dst))):
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        phases[name] = (time.perf_counter() - t0) * 1e3
    sim.close()
    nbytes = 3 * N * N * 8
    return {"value": N * N * JOB_STEPS * jobs / dt / 1e6, "unit": UNIT, "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes, "step": f"one job: upload W0, {JOB_STEPS} steps, download W",
            "lb_steps_per_step": JOB_STEPS, "jobs": jobs, "seconds": dt, "per_job_ms": per_job,
            "phases_of_one_more_job": phases}


def profile_case(args, local):
    """Run one kernel family for --warmup + --steps iterations so that a profiler can
    capture it (prints a short JSON summary, not the benchmark line)."""
    import torch

    torch.cuda.set_device(local)
    from paper_1401_0427_gb300 import build as libbuild
    from paper_1401_0427_gb300 import inputs, lbm_sw

    libbuild.build()
    stream = torch.cuda.current_stream()
    n = args.side
    out = {"case": args.case, "side": n, "steps": args.steps, "warmup": args.warmup}
    if args.case == "batched":
        table = inputs.batched_instances(256)[:args.count]
        sizes = [(k, k) for k, _, _ in table]
        with lbm_sw.Batch(sizes, lam=LAM, s=S_RATE, a=A_REST, stream=stream.cuda_stream, tile_rows=1,
                          ctas_per_sm=0, graph_chunk=-1, temporal_steps=args.temporal_steps or 1) as b:
            for i, (k, hin, r) in enumerate(table):
                b.set_state(i, *inputs.circular_dam_break_2d(k, seed=None, h_in=hin, radius=r))
            b.step(args.warmup)
            t = _timed(stream, torch, lambda: b.step(args.steps))
            out["cells"] = sum(k * k for k, _ in sizes)
    elif args.case == "adjoint":
        h0 = inputs.gaussian_bumps_2d(n, seed=inputs.stream_seed(5, 5))[0]
        z = np.zeros((n, n))
        prec = lbm_sw.FP64 if args.precision == "fp64" else lbm_sw.FP32
        with lbm_sw.Simulation(n, n, precision=prec, lam=LAM, s=S_RATE, a=A_REST, stream=stream.cuda_stream) as sim:
            sim.set_state(h0, z, z)
            with lbm_sw.Tape(sim, args.steps) as tape:
                tape.record()
                g = torch.full((n, n), 1e-3, dtype=torch.float64, device="cuda")
                t = _timed(stream, torch, lambda: tape.adjoint(g))
        out["cells"] = n * n
    elif args.case == "reflection":
        n = 512
        uL = inputs.shock_speed_state(2.0, 1.0)
        prec = lbm_sw.FP64 if args.precision == "fp64" else lbm_sw.FP32
        with lbm_sw.Simulation(n, n, precision=prec, lam=LAM, s=S_RATE, a=A_REST,
                               bc=(lbm_sw.INFLOW, lbm_sw.WALL, lbm_sw.PERIODIC, lbm_sw.PERIODIC),
                               inflow=[(2.0, 2.0 * uL, 0.0)] * 4, stream=stream.cuda_stream, graph_chunk=-1) as sim:
            sim.set_state(*inputs.planar_shock_2d(n, n))
            sim.step(args.warmup)
            t = _timed(stream, torch, lambda: sim.step(args.steps))
        out["cells"] = n * n
    elif args.case == "basin":
        W = lbm_sw.WALL
        with lbm_sw.Simulation(n, n, lam=LAM, s=S_RATE, a=A_REST, bc=(W, W, W, W), stream=stream.cuda_stream,
                               graph_chunk=-1) as sim:
            sim.set_state(*inputs.circular_dam_break_2d(n, seed=inputs.stream_seed(3)))
            sim.step(args.warmup)
            t = _timed(stream, torch, lambda: sim.step(args.steps))
            out["steps_per_launch"] = sim.info().steps_per_launch
        out["cells"] = n * n
    elif args.case == "mrt":
        with lbm_sw.Simulation(n, n, lam=LAM, s=S_RATE, a=A_REST, stream=stream.cuda_stream, graph_chunk=-1) as sim:
            sim.set_relaxation(MRT_RATES)
            sim.set_state(*inputs.circular_dam_break_2d(n, seed=inputs.stream_seed(3)))
            sim.step(args.warmup)
            t = _timed(stream, torch, lambda: sim.step(args.steps))
            out["steps_per_launch"] = sim.info().steps_per_launch
        out["cells"] = n * n
    elif args.case == "shock_tube":
        h, q = inputs.dam_break_1d(1000)
        with lbm_sw.Simulation(1000, 1, dim=1, precision=lbm_sw.FP64, lam=LAM, s=S_RATE, a=0.15,
                               bc=(lbm_sw.WALL, lbm_sw.WALL), stream=stream.cuda_stream, graph_chunk=-1) as sim:
            sim.set_state(h, q)
            sim.step(args.warmup)
            t = _timed(stream, torch, lambda: sim.step(args.steps))
        out["cells"] = 1000
    else:  # diag
        W0 = inputs.circular_dam_break_2d(n, seed=inputs.stream_seed(3))
        with lbm_sw.Simulation(n, n, lam=LAM, s=S_RATE, a=A_REST, stream=stream.cuda_stream) as sim:
            sim.set_state(*W0)
            for _ in range(args.warmup):
                sim.diagnostics()
            t = _timed(stream, torch, lambda: [sim.diagnostics() for _ in range(args.steps)])
        out["cells"] = n * n
    out["seconds"] = t
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--quick", action="store_true", help="timed loop only (no variants, e2e, CPU baseline)")
    ap.add_argument("--skip-cpu", action="store_true", help="omit the CPU oracle baseline")
    ap.add_argument("--side", type=int, default=4096, help="grid side (profiling of smaller cases only)")
    ap.add_argument("--count", type=int, default=256, help="instances of the batched profiling case")
    ap.add_argument("--kernel", choices=["auto", "vec", "temporal"], default="auto",
                    help="step kernel of the timed loop (auto: the library's choice, temporal blocking on this "
                         "workload; vec: one step per launch)")
    ap.add_argument("--temporal-steps", type=int, default=0,
                    help="steps per launch of the temporal kernel (0: the library default, 6 here; for "
                         "--case batched: 0 or 1 = one step per launch)")
    ap.add_argument("--case", choices=["step", "batched", "adjoint", "reflection", "basin", "mrt", "shock_tube", "diag"],
                    default="step",
                    help="kernel to run for profiling (only 'step' prints the benchmark line; basin: the "
                         "dam-break with walls on every side; mrt: the dam-break with the MRT collision)")
    ap.add_argument("--replicas", action="store_true",
                    help="with N > 1 GPUs, run N independent replicas of the grid instead of splitting it")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32",
                    help="population precision of the timed loop (fp32 is the workload)")
    args = ap.parse_args()
    if args.warmup < 3 and args.case == "step":
        ap.error("--warmup must be >= 3")
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.case != "step":
        profile_case(args, local)
    elif world > 1 and not args.replicas:
        run_split(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
