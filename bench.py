"""Benchmark of the fused wave-propagation step on GB300.

Default workload: 2D shallow water (Roe + Harten-Hyman entropy fix), radial
dam break on a 4096 x 4096 grid, FP32, reflecting walls, MC limiter,
transverse splits, CFL 0.9 with the device-side variable dt rule.  One bench
"step" is one time step of that problem (ghost fill + fused step + dt rule),
all of them launched as CUDA graphs by one mc_advance call; the timed region
is exactly K steps.  Each state array is 201 MB, larger than the 129 MB L2, so
every step streams its input from HBM.

Printed (rank 0): one JSON line with the metric (cell-updates/s), the kernel
roofline of the fused step (algorithmic bytes / CUDA-event duration against
the measured HBM copy bandwidth), the end-to-end rate through the host-buffer
C-ABI call, the FP64 CPU oracle timed on this machine's cores as a baseline,
and SM clocks sampled during the timed region.

``--impl reference`` times the oracle itself (the only reference there is:
the paper publishes no code), on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
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

WORKLOADS = {
    "swe32": dict(solver="swe", dtype="f32", n=4096, cfl=0.9, bc="wall",
                  desc="shallow-water Roe+HH dam break 4096x4096 fp32, walls, MC, CFL 0.9"),
    "swe64": dict(solver="swe", dtype="f64", n=4096, cfl=0.9, bc="wall",
                  desc="shallow-water Roe+HH dam break 4096x4096 fp64, walls, MC, CFL 0.9"),
    "euler32": dict(solver="euler", dtype="f32", n=4096, cfl=0.8, bc="extrap",
                    desc="Euler Roe+HH four-quadrant 4096x4096 fp32, extrapolation, MC, CFL 0.8"),
    # the small case: 10 steps of dt = 0.9 dx / c, the state (0.4 MB) L2-resident
    # within a run, so each 10-step run starts after an L2 flush
    "acoustics": dict(solver="acoustics", dtype="f64", n=128, cfl=0.9, bc="periodic",
                      fixed_dt=0.9 * (1.0 / 128) / 2.0, iter_steps=10,
                      desc="acoustics Gaussian pulse 128x128 fp64, periodic, MC, dt = 0.9 dx / c, "
                           "runs of 10 steps"),
    # further solvers and options of the step (advection on 8192^2 so that a
    # state, 268 MB, exceeds the L2 like the others)
    "adv32": dict(solver="advection", dtype="f32", n=8192, cfl=0.9, bc="periodic",
                  desc="advection (u, v) = (1, 0.6) Gaussian 8192x8192 fp32, periodic, MC, CFL 0.9"),
    "acvar32": dict(solver="acoustics_var", dtype="f32", n=4096, cfl=0.9, bc="extrap",
                    desc="variable-coefficient acoustics, layered medium 4096x4096 fp32, "
                         "extrapolation, MC, CFL 0.9"),
    "eulg32": dict(solver="euler_godunov", dtype="f32", n=4096, cfl=0.8, bc="extrap",
                   desc="Euler with the exact-solution (Godunov) normal solve, four-quadrant "
                        "4096x4096 fp32, extrapolation, MC, CFL 0.8"),
    "swe32t2": dict(solver="swe", dtype="f32", n=4096, cfl=0.9, bc="wall", limiter=3, transverse=2,
                    desc="shallow-water Roe+HH dam break 4096x4096 fp32, walls, van Leer, "
                         "transverse option 2, CFL 0.9"),
}
G, GAMMA = 9.81, 1.4
# GB300 FP64 (non-tensor) nominal rate, TFLOP/s
FP64_NOMINAL_TFLOPS = 1.25


class L2Flush:
    """Writes a device buffer of twice the L2 size, so that the next timed
    iteration finds none of its inputs in the L2."""

    def __init__(self, torch):
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        self.l2_bytes = int(getattr(props, "L2_cache_size", 0) or (129 << 20))
        self.buf = torch.empty(2 * self.l2_bytes, dtype=torch.uint8, device="cuda")
        self.k = 0

    def __call__(self):
        self.k += 1
        self.buf.fill_(self.k & 0xFF)


def dist_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(ms: float, world: int, device: str) -> float:
    """The timed region's duration as the slowest rank saw it (all ranks
    return the same value).  Each rank runs an independent replica of the
    workload, so this is the only exchange between ranks."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def replica_throughput(ms: float, world: int, units_per_step: int, steps: int) -> float:
    """Whole-job rate: the units every rank processed over the max-over-ranks time."""
    return world * units_per_step * steps / (ms * 1e-3)


def make_problem(mc, wl, mx=None, my=None, window=None):
    """The workload's problem on an mx x my grid (n x n by default) and its
    initial state, only the cells of `window` (i0, j0, nx, ny) if given."""
    from paper_1308_1464_gb300 import workloads
    mx = mx or wl["n"]
    my = my or wl["n"]
    if wl["solver"] == "swe":
        g = workloads.swe_dambreak(mx, my, window=window)
        sid, param, bc = mc.SWE_ROE, (G, 0, 0, 0), mc.BC_WALL
    elif wl["solver"] in ("euler", "euler_godunov"):
        g = workloads.euler_quadrants(mx, my, window=window)
        sid = mc.EULER_ROE if wl["solver"] == "euler" else mc.EULER_GODUNOV
        param, bc = (GAMMA, 0, 0, 0), mc.BC_EXTRAP
    elif wl["solver"] == "advection":
        g = workloads.advection_pulse(mx, my, window=window)
        sid, param, bc = mc.ADVECTION, (1.0, 0.6, 0, 0), mc.BC_PERIODIC
    elif wl["solver"] == "acoustics_var":
        g = workloads.acoustics_layered(mx, my, window=window)
        sid, param, bc = mc.ACOUSTICS_VAR, (0, 0, 0, 0), mc.BC_EXTRAP
    else:
        g = workloads.acoustics_pulse(mx, my, window=window)
        sid, param, bc = mc.ACOUSTICS, (1.0, 4.0, 0, 0), mc.BC_PERIODIC
    dtype = mc.F64 if wl["dtype"] == "f64" else mc.F32
    p = mc.Problem.make(sid, mx, my, g.dx, g.dy, dtype=dtype, bc=(bc,) * 4, param=param,
                        limiter=wl.get("limiter", mc.LIM_MC), transverse=wl.get("transverse", 1))
    return p, g


def sweep_kernels(mc, p) -> int:
    """Kernels one fused-step call launches: the step kernel, plus the FP64
    guard kernel of an FP32 Roe solver (shallow water, Euler) with the guard
    on (param[3] >= 0)."""
    guarded = (p.dtype == mc.F32 and p.solver in (mc.SWE_ROE, mc.EULER_ROE)
               and float(p.param[3]) >= 0.0)
    return 2 if guarded else 1


def block_shape(world: int, spec: str = ""):
    """px x py blocks: from spec "PXxPY", else the most nearly square
    factorisation of world with px >= py."""
    if spec:
        px, py = (int(v) for v in spec.lower().split("x"))
        return px, py
    py = max(d for d in range(1, int(world ** 0.5) + 1) if world % d == 0)
    return world // py, py


class ClockSampler:
    """nvidia-smi clock/throttle sampling while a region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def __enter__(self):
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.tmp.flush()
        with open(self.tmp.name) as f:
            rows = [r.strip().split(", ") for r in f if r.strip()]
        os.unlink(self.tmp.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [s for s in sm if s > 0.5 * max(sm)]
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d["hbm_gbs"], "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def measured_unit_peaks():
    """The execution-unit rates of profiles/peaks_gb300.json (bench.py --peaks
    on a GB300 of this pool), or None."""
    try:
        with open(os.path.join(ROOT, "profiles", "peaks_gb300.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


def fp64_peak():
    """(TFLOP/s, source) of the FP64 fused multiply-add: measured if on record."""
    pk = measured_unit_peaks()
    if pk and "dfma" in pk:
        return pk["dfma"]["value"], "measured DFMA rate (profiles/peaks_gb300.json)"
    return FP64_NOMINAL_TFLOPS, "nominal GB300 FP64 rate"


def sweep_source_hash():
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_1308_1464_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.startswith("mc_sweep") or name in ("mc_riemann.cuh", "mc_device.cuh", "mc_tile.h"):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode())
                h.update(f.read())
    return h.hexdigest()[:16]


def batch_source_hash():
    """Sources of the batched kernel: its own files and the fused step's."""
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_1308_1464_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if (name.startswith("mc_sweep") or name.startswith("mc_batch")
                or name in ("mc_riemann.cuh", "mc_device.cuh", "mc_tile.h")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode())
                h.update(f.read())
    return h.hexdigest()[:16]


def exact_source_hash():
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_1308_1464_gb300", "csrc")
    for name in ("mc_exact.cu", "mc_seednet.cuh", "mc_mma.cuh"):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_exact():
    """FP64 instruction counts of the exact-solver kernel from the committed
    ncu summary, if it was taken on the current sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_exact.json")) as f:
            d = json.load(f)
        if d.get("source_hash") == exact_source_hash():
            return d
    except (OSError, ValueError):
        pass
    return None


def ncu_fp64(workload: str):
    """FP64 counts of the fused step of an FP64 workload from the committed
    ncu summary, if taken on the current kernel sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_fp64.json")) as f:
            d = json.load(f)
        e = d.get(workload)
        if e and e.get("source_hash") == sweep_source_hash():
            return e
    except (OSError, ValueError):
        pass
    return None


def ncu_traffic(workload: str):
    """DRAM bytes per launch of the fused step from the committed ncu summary,
    if it was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d.get(workload)
        if e and e.get("source_hash") == sweep_source_hash():
            return e["dram_bytes_per_launch"]
    except (OSError, ValueError):
        pass
    return None


def ncu_batch():
    """DRAM bytes of one persistent launch of the batched kernel (20 steps
    over the 2000 patches) from the committed ncu summary, if it was taken
    on the current sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            d = json.load(f)
        e = d.get("batch2000")
        if e and e.get("source_hash") == batch_source_hash():
            return e
    except (OSError, ValueError):
        pass
    return None


def oracle_problem(wl, n):
    """The oracle's problem and seeded input for workload wl on an n x n grid."""
    import oracle
    from paper_1308_1464_gb300 import workloads
    opts = dict(limiter=wl.get("limiter", oracle.LIM_MC), transverse=wl.get("transverse", 1))
    if wl["solver"] == "swe":
        g = workloads.swe_dambreak(n, n)
        op = oracle.Problem(oracle.SWE, n, n, g.dx, g.dy, bc=(oracle.BC_WALL,) * 4,
                            param=(G, 0, 0, 0), **opts)
    elif wl["solver"] in ("euler", "euler_godunov"):
        g = workloads.euler_quadrants(n, n)
        sid = oracle.EULER if wl["solver"] == "euler" else oracle.EULER_GODUNOV
        op = oracle.Problem(sid, n, n, g.dx, g.dy, bc=(oracle.BC_EXTRAP,) * 4,
                            param=(GAMMA, 0, 0, 0), **opts)
    elif wl["solver"] == "advection":
        g = workloads.advection_pulse(n, n)
        op = oracle.Problem(oracle.ADVECTION, n, n, g.dx, g.dy, param=(1.0, 0.6, 0, 0), **opts)
    elif wl["solver"] == "acoustics_var":
        g = workloads.acoustics_layered(n, n)
        op = oracle.Problem(oracle.ACOUSTICS_VAR, n, n, g.dx, g.dy, bc=(oracle.BC_EXTRAP,) * 4,
                            param=(0, 0, 0, 0), **opts)
    else:
        g = workloads.acoustics_pulse(n, n)
        op = oracle.Problem(oracle.ACOUSTICS, n, n, g.dx, g.dy, param=(1.0, 4.0, 0, 0), **opts)
    return op, g


def cpu_baseline(wl, budget_s=12.0):
    """The FP64 oracle, as it stands, timed on this machine's cores on a bounded
    sample of the workload: steps of the same problem on an n x n grid."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    n = 1024 if wl["solver"] != "acoustics" else 128
    op, g = oracle_problem(wl, n)
    q = np.zeros(op.shape)
    q[:, 2:-2, 2:-2] = g.q
    dt = wl["cfl"] / oracle.max_cell_speed(op, oracle.bc_fill(op, q))
    oracle.step(op, q, dt, nthreads=cores)   # warm-up
    steps, t0 = 0, time.perf_counter()
    while True:
        q, smax, _ = oracle.step(op, q, dt, nthreads=cores)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or steps >= (200 if n >= 1024 else 10000):
            break
    rec = {"value": n * n * steps / el, "unit": "cell-updates/s", "cores": cores,
           "kind": "oracle",
           "sample": f"{steps} FP64 oracle steps of the same problem on a {n}x{n} grid "
                     f"(OpenMP over rows, {cores} threads), {el:.1f} s"}
    # the plain oracle on one core, a shorter sample of the same grid
    q1 = np.zeros(op.shape)
    q1[:, 2:-2, 2:-2] = g.q
    s1, t1 = 0, time.perf_counter()
    while True:
        q1, _, _ = oracle.step(op, q1, dt, nthreads=1)
        s1 += 1
        e1 = time.perf_counter() - t1
        if e1 >= budget_s / 3 or s1 >= 50:
            break
    rec["single_thread"] = {"value": n * n * s1 / e1, "unit": "cell-updates/s", "cores": 1,
                            "sample": f"{s1} FP64 oracle steps on the {n}x{n} grid, one thread, "
                                      f"{e1:.1f} s"}
    return rec


def run_reference(args, wl):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0))
    # size each step's sample so that warmup + steps fit in about two minutes
    per_step_budget = 120.0 / max(1, args.steps + args.warmup)
    probe = cpu_baseline(wl, budget_s=1.0)
    rate = probe["value"]
    n = int(max(16, min(wl["n"], (rate * per_step_budget) ** 0.5)))
    op, g = oracle_problem(wl, n)
    q = np.zeros(op.shape)
    q[:, 2:-2, 2:-2] = g.q
    dt = wl["cfl"] / oracle.max_cell_speed(op, oracle.bc_fill(op, q))
    for _ in range(args.warmup):
        q, smax, _ = oracle.step(op, q, dt, nthreads=cores)
        dt = wl["cfl"] / smax
    t0 = time.perf_counter()
    for _ in range(args.steps):
        q, smax, _ = oracle.step(op, q, dt, nthreads=cores)
        dt = wl["cfl"] / smax
    el = time.perf_counter() - t0
    value = n * n * args.steps / el
    sample = f"each step: one FP64 oracle step on a {n}x{n} grid of the same problem"
    print(json.dumps({
        "impl": "reference", "metric": "cell-updates/s", "value": value, "unit": "cell-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["desc"], "sample_grid": n},
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


def bench_batch(args, rank, world):
    """2000 uneven shallow-water patches (sides log-uniform in [16, 256]) per
    GPU, FP32, walls, per-patch dt at CFL 0.9: K steps in one persistent
    launch inside a CUDA graph with autotuned work splits, against one launch
    per patch per step on the same GPU.  With N ranks the 2000 N patches of
    the seeded set are shared by greedy longest-processing-time on cell
    count; the patches are independent, so the ranks exchange nothing but
    the slowest rank's time."""
    import torch
    import paper_1308_1464_gb300 as mc
    from paper_1308_1464_gb300 import autotune, workloads
    from paper_1308_1464_gb300.blocks import lpt_shards
    from paper_1308_1464_gb300.state import PatchSet
    nall = 2000 * world
    sizes_all = workloads.swe_patches(nall, with_state=False)
    cells_all = sum(q.nx * q.ny for q in sizes_all)
    mine = lpt_shards([q.nx * q.ny for q in sizes_all], world)[rank]
    pats_w = workloads.swe_patches(nall, only=mine)
    pats = [(p.nx, p.ny, p.grid.dx, p.grid.dy, p.grid.q) for p in pats_w]
    cells = sum(p[0] * p[1] for p in pats)
    proto = mc.Problem.make(mc.SWE_ROE, 16, 16, 1 / 128, 1 / 128, dtype=mc.F32,
                            bc=(mc.BC_WALL,) * 4, param=(G, 0, 0, 0))
    ps = PatchSet(proto, pats)
    b = mc.Batch(proto, ps.pointers())
    sizes = [(p[0], p[1]) for p in pats]
    cache = os.path.join(tempfile.gettempdir(), "manyclaw_batch_tune%s.json" % (f"_r{rank}" if world > 1 else ""))
    policy, tune_ms = autotune.tune_batch(b, sizes, ps.reset, nsteps=4, cache_path=cache)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    # the configuration's 20 steps per persistent launch; K steps are timed as
    # K / 20 such launches, each continuing from the previous state
    per_launch = 20
    launches = max(1, args.steps // per_launch)
    K = launches * per_launch
    for _ in range(args.warmup):
        ps.reset()
        b.advance(per_launch, 0.9, stream=sh)
    ps.reset()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        e0.record(stream)
        for _ in range(launches):
            b.advance(per_launch, 0.9, stream=sh)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    # one launch per step over all patches (the same kernel, one step per
    # launch, the launches of a call in one graph): the step-synchronous form
    ps.reset()
    b.advance_steps(per_launch, 0.9, stream=sh)   # builds its graph
    ps.reset()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(launches):
        b.advance_steps(per_launch, 0.9, stream=sh)
    s1.record(stream)
    torch.cuda.synchronize()
    ms_steps = max_over_ranks(s0.elapsed_time(s1), world, "cuda")
    ps.reset()
    b.advance_plain(2, 0.9, stream=sh)       # warm the per-patch path
    ps.reset()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    b.advance_plain(per_launch, 0.9, stream=sh)
    p1.record(stream)
    torch.cuda.synchronize()
    ms_plain = max_over_ranks(p0.elapsed_time(p1), world, "cuda") * K / per_launch
    value = cells_all * K / (ms * 1e-3)
    alg = 2 * cells * 3 * 4 * K     # this rank's bytes (the roofline is per GPU)
    peak, kind = measured_peaks()
    nb = ncu_batch() if world == 1 else None
    b.close()
    return {
        "metric": "cell-updates/s", "value": value, "unit": "cell-updates/s", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "2000 uneven shallow-water patches (16..256 per side) per GPU, fp32, "
                               "walls, per-patch dt CFL 0.9, 20 steps per persistent launch in a "
                               "CUDA graph",
                   "cells": cells_all, "patches": nall, "tune_policy": policy, "tune_ms": tune_ms,
                   "tuned_over_as_created": round(tune_ms["as_created"] / min(tune_ms.values()), 4),
                   "parallelism": ("patches shared by LPT on cell count, %d ranks" % world
                                   if world > 1 else "single"),
                   "l2": "inputs larger than L2 (%.0f MB per state)" % (ps.nbytes / 1e6)},
        "per_step_launch": {"value": cells_all * K / (ms_steps * 1e-3), "ms_per_step": ms_steps / K,
                            "launches_per_step": 1,
                            "note": "the same kernel, one launch per step over all patches, "
                                    "a call's launches in one CUDA graph"},
        "plain": {"value": cells_all * K / (ms_plain * 1e-3), "ms_per_step": ms_plain / K,
                  "launches_per_step": 3 * len(pats), "timed_steps": per_launch},
        "batched_over_per_step_launch": ms_steps / ms,
        "batched_over_plain": ms_plain / ms,
        "roofline": {"bound": "hbm", "achieved": round(alg / (ms * 1e-3) / 1e9, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(alg / (ms * 1e-3) / 1e9 / peak, 4),
                     "traffic": nb["dram_bytes_per_launch"] if nb else None,
                     "kernel": "batch_sweep_kernel",
                     "algorithmic_bytes_per_launch": 2 * cells * 3 * 4 * per_launch,
                     "timed": "each persistent launch with its initial speed scan",
                     "peak_source": f"{kind} HBM copy"},
        # per persistent launch: the per-patch initial speed scan and the sweep
        "gpu_launches": 2 * launches, "clocks": clk.summary(),
    }


def bench_amr(args, rank, world):
    """Shallow-water dam break on a 4096^2 coarse grid (FP32, walls) with
    ratio-2 patches of 128^2 coarse cells over the ring 0.3 <= r <= 0.7 that
    the waves cross: K coarse steps of mc_amr_advance (two fine steps per
    patch each, conservative coupling by refluxing), against a uniformly fine
    8192^2 grid advanced over the same simulated time with the fused step
    alone.  The coarse state and the patch states together exceed the L2."""
    import torch
    import paper_1308_1464_gb300 as mc
    from paper_1308_1464_gb300 import workloads
    from paper_1308_1464_gb300.state import DeviceState
    nc, r, blk = 4096, 2, 128
    g = workloads.swe_dambreak(nc, nc)
    p = mc.Problem.make(mc.SWE_ROE, nc, nc, g.dx, g.dy, dtype=mc.F32, bc=(mc.BC_WALL,) * 4,
                        param=(G, 0, 0, 0))
    ctx = mc.Context(p)
    qa, qb = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
    q0 = np.ascontiguousarray(g.q.astype(np.float32))
    qa.upload(q0)
    patches, fine = [], []
    for bj in range(nc // blk):
        for bi in range(nc // blk):
            xc = g.x_lo + (bi + 0.5) * blk * g.dx
            yc = g.y_lo + (bj + 0.5) * blk * g.dy
            if 0.3 <= (xc * xc + yc * yc) ** 0.5 <= 0.7:
                fp = mc.amr_fine_problem(p, r, bi * blk, bj * blk, blk, blk)
                lay = mc.layout_of(fp)
                a = torch.zeros(int(lay.bytes), dtype=torch.uint8, device="cuda")
                b = torch.zeros_like(a)
                # fine initial data: each coarse value on its r x r fine cells
                sub = q0[:, bj * blk:(bj + 1) * blk, bi * blk:(bi + 1) * blk]
                v = a.view(torch.float32)[: lay.meqn * lay.ld_field].view(int(lay.meqn), fp.my + 4, int(lay.ld_x))
                x0 = int(lay.x_offset)
                v[:, 2:-2, x0: x0 + fp.mx] = torch.from_numpy(np.repeat(np.repeat(sub, r, 1), r, 2)).cuda()
                patches.append((bi * blk, bj * blk, blk, blk, a.data_ptr(), b.data_ptr()))
                fine.append((a, b))
    amr = mc.Amr(p, r, patches, reflux=True)
    smax = ctx.max_cell_speed(qa.ptr)
    dt = 0.8 / smax
    K = args.steps
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    for _ in range(args.warmup):
        amr.advance(qa.ptr, qb.ptr, 2, dt, sh)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        e0.record(stream)
        amr.advance(qa.ptr, qb.ptr, K, dt, sh)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    fine_cells = len(patches) * (r * blk) ** 2
    updates = K * (nc * nc + r * fine_cells)
    # the same simulated time on a uniformly fine grid: r K fused steps of dt / r
    gf = workloads.swe_dambreak(r * nc, r * nc)
    pf = mc.Problem.make(mc.SWE_ROE, r * nc, r * nc, gf.dx, gf.dy, dtype=mc.F32, bc=(mc.BC_WALL,) * 4,
                         param=(G, 0, 0, 0))
    cf = mc.Context(pf)
    fa, fb = DeviceState(cf).zero_(), DeviceState(cf).zero_()
    fa.upload(np.ascontiguousarray(gf.q.astype(np.float32)))
    cf.bc_fill(fa.ptr, sh)
    for _ in range(3):
        cf.sweep(fa.ptr, fb.ptr, dt / r, sh)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for k in range(r * K):
        src, dst = (fa, fb) if k % 2 == 0 else (fb, fa)
        cf.step(src.ptr, dst.ptr, dt / r, want_smax=False, stream=sh)
    f1.record(stream)
    torch.cuda.synchronize()
    fms = max_over_ranks(f0.elapsed_time(f1), world, "cuda")
    amr.close()
    return {
        "metric": "cell-updates/s", "value": world * updates / (ms * 1e-3), "unit": "cell-updates/s",
        "n_gpus": world, "steps": K, "warmup": args.warmup, "ms_per_step": ms / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "shallow-water dam break, 4096^2 coarse fp32 walls, ratio-2 patches "
                               "of 128^2 coarse cells over the ring 0.3 <= r <= 0.7, refluxing, CFL 0.8",
                   "patches": len(patches), "fine_cells": fine_cells,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (%d MB coarse state, %d MB of patch states)"
                         % (int(ctx.layout.bytes) // 10**6,
                            sum(int(a.numel()) for a, _ in fine) // 10**6)},
        "uniform_fine": {"grid": f"{r * nc}x{r * nc}", "ms_for_same_time": fms,
                         "amr_ms": ms, "amr_speedup": fms / ms},
        # per coarse step: ghost fill + fused step (coarse), ghost fill of the
        # new coarse state, the coarse boundary fluxes, ratio x (patch ghosts +
        # fine boundary fluxes + one multi-patch fused step), average down, the
        # flux correction (one launch per edge class) and a last ghost fill
        "gpu_launches": K * (2 + 1 + 1 + 3 * r + 1 + 4 + 1),
        "clocks": clk.summary(),
    }


TRAIN_OFFSET, TRAIN_ROWS = 1 << 26, 1 << 22   # the seed network's training draws


def exact_offset(rank: int, n: int) -> int:
    """First draw of rank r's n interfaces: blocks disjoint across ranks and
    from the training draws [TRAIN_OFFSET, TRAIN_OFFSET + TRAIN_ROWS)."""
    if (rank + 1) * n <= TRAIN_OFFSET:
        return rank * n
    return 2 * TRAIN_OFFSET + rank * n


def bench_exact(args, rank, world):
    """2^24 exact Euler Riemann problems (rho in [0.01, 10], p in [0.01, 100]
    log-uniform, |u| <= 5), FP64 Newton to |dp|/p < 1e-8: the plain adaptive
    seed against the 10-64-64-1 network seed.  The network is trained here,
    on the GPU, on 2^22 separate interfaces whose star pressures come from the
    same exact solver run to 1e-12."""
    import torch
    import paper_1308_1464_gb300 as mc
    from paper_1308_1464_gb300 import workloads
    GAM = 1.4

    def dev_states(n, offset):
        st = workloads.riemann_states(n, seed=1308, offset=offset)
        return [torch.from_numpy(a.astype(np.float32)).cuda() for a in st]

    def solve(states, mode, net, tol=1e-8):
        n = states[0].numel()
        ps = torch.empty(n, dtype=torch.float32, device="cuda")
        us = torch.empty_like(ps)
        it = torch.empty(n, dtype=torch.uint8, device="cuda")
        fl = torch.empty_like(it)
        stats = torch.zeros(8, dtype=torch.int64, device="cuda")
        mc.riemann_exact(n, GAM, [s.data_ptr() for s in states], ps.data_ptr(), us.data_ptr(),
                         it.data_ptr(), fl.data_ptr(), mode, net, tol, 30, stats.data_ptr())
        return ps, it, fl, stats, us

    from paper_1308_1464_gb300.seednet import train_seed_net
    ntrain, epochs = TRAIN_ROWS, 12
    net, losses, train_s = train_seed_net(ntrain=ntrain, epochs=epochs, gamma=GAM,
                                          offset=TRAIN_OFFSET)

    n = 1 << 24
    off = exact_offset(rank, n)
    test = dev_states(n, offset=off)
    stream = torch.cuda.current_stream()
    out = {}
    clk = ClockSampler(torch.cuda.current_device())
    clk.__enter__()
    arms = (("plain", mc.SEED_ADAPTIVE, None), ("learned", mc.SEED_MLP, net),
            ("plain_mixed", mc.SEED_ADAPTIVE | mc.NEWTON_MIXED, None),
            ("learned_mixed", mc.SEED_MLP | mc.NEWTON_MIXED, net))
    for name, mode, nn in arms:
        for _ in range(args.warmup):
            solve(test, mode, nn)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        reps = max(1, args.steps)
        for _ in range(reps):
            ps, it, fl, stats, _ = solve(test, mode, nn)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda") / reps
        st = stats.cpu().numpy()
        nonvac = st[0] - st[1]
        out[name] = {"solves_per_s": world * n / (ms * 1e-3), "ms": ms,
                     "mean_newton_updates": float(st[4] / max(nonvac, 1)),
                     "fallback_rate": float(st[2] / max(nonvac, 1)), "vacuum": int(st[1]),
                     "not_converged": int(st[3])}
        if mode & mc.NEWTON_MIXED:
            out[name]["mean_fp32_updates"] = float(st[6] / max(nonvac, 1))
            out[name]["mean_fp64_updates"] = float(st[7] / max(nonvac, 1))
        if name == "plain":
            ps_plain = ps.clone()
        else:
            ok = fl.cpu().numpy() & 1 == 0
            a, c = ps.cpu().numpy()[ok], ps_plain.cpu().numpy()[ok]
            out[name]["max_rel_diff_vs_plain"] = float(np.max(np.abs(a - c) / np.abs(c)))
    clk.__exit__(None, None, None)
    e2e = None
    if not getattr(args, "light", False):
        e2e = exact_e2e(n, off, world, solve, net, mc)
    return exact_record(args, out, e2e, world, n, ntrain, epochs, train_s, losses, clk)


def exact_e2e(n, off, world, solve, net, mc):
    """End to end through the public call: the six state arrays from pinned
    host memory, the learned-seed solve, p* and u* back to pinned host memory."""
    import torch
    from paper_1308_1464_gb300 import workloads
    host = [torch.from_numpy(a.astype(np.float32)).pin_memory()
            for a in workloads.riemann_states(n, seed=1308, offset=off)]
    h_ps = torch.empty(n, dtype=torch.float32).pin_memory()
    h_us = torch.empty_like(h_ps).pin_memory()
    dev = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(6)]
    reps_e2e = 3
    for rep in range(reps_e2e + 1):
        if rep == 1:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
        for d, h in zip(dev, host):
            d.copy_(h, non_blocking=True)
        ps, _, _, _, us = solve(dev, mc.SEED_MLP | mc.NEWTON_MIXED, net)
        h_ps.copy_(ps, non_blocking=True)
        h_us.copy_(us, non_blocking=True)
        torch.cuda.synchronize()
    el = max_over_ranks((time.perf_counter() - t0) * 1e3, world, "cuda") * 1e-3
    return {"value": world * n * reps_e2e / el, "unit": "solves/s",
            "h2d_bytes_per_step": 6 * 4 * n, "d2h_bytes_per_step": 2 * 4 * n,
            "note": "six FP32 state arrays from pinned host memory, mc_riemann_exact with the "
                    "learned seed, p* and u* back to pinned host memory; one step = 2^24 solves"}


def exact_record(args, out, e2e, world, n, ntrain, epochs, train_s, losses, clk):
    peak, kind = measured_peaks()
    # the headline arm: the learned seed, FP32 Newton stage and FP64 finish (the same
    # |dp|/p < 1e-8 test in FP64)
    ms = out["learned_mixed"]["ms"]
    cnt = ncu_exact()
    if cnt is not None and "learned_mixed" in cnt:
        # FP64-pipe bound: flops counted by ncu on these sources over the live time
        c = cnt["learned_mixed"]
        achieved = c["fp64_flops_per_launch"] / (ms * 1e-3) / 1e12
        pk64, pk64_src = fp64_peak()
        roofline = {"bound": "alu", "achieved": round(achieved, 4), "peak": pk64,
                    "unit": "TFLOP/s", "frac": round(achieved / pk64, 4),
                    "traffic": c["dram_bytes_per_launch"], "kernel": "exact_kernel<1, 1>",
                    "fp64_pipe_active_pct": c["fp64_pipe_active_pct"],
                    "fp32_flops_per_launch": c["fp32_flops_per_launch"],
                    "peak_source": pk64_src,
                    "flops_source": "FP64 thread instructions of one launch counted by ncu on "
                                    "these sources (FMA = 2 flops, add and multiply = 1)"}
    else:
        roofline = {"bound": "hbm", "achieved": round(34 * n / (ms * 1e-3) / 1e9, 1),
                    "peak": peak, "unit": "GB/s",
                    "frac": round(34 * n / (ms * 1e-3) / 1e9 / peak, 4), "traffic": None,
                    "kernel": "exact_kernel<1, 1>", "note": "FP64-ALU bound; bytes not binding"}
    return {
        "metric": "Riemann solves/s", "value": out["learned_mixed"]["solves_per_s"],
        "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 then f64 Newton, f32 io, bf16 network", "data": "synthetic",
        "config": {"workload": "2^24 exact Euler Riemann problems, gamma 1.4, tol 1e-8",
                   "train_rows": ntrain, "train_epochs": epochs, "train_s": round(train_s, 2),
                   "train_loss": [float(x) for x in losses]},
        "plain": out["plain"], "learned": out["learned"],
        "plain_mixed": out["plain_mixed"], "learned_mixed": out["learned_mixed"],
        "roofline": roofline, "e2e": e2e,
        "gpu_launches": 1, "clocks": clk.summary(),
    }


PEAK_KINDS = [("ffma", 0, "TFLOP/s", 1e12), ("ffma2", 1, "TFLOP/s", 1e12), ("dfma", 2, "TFLOP/s", 1e12),
              ("rsqrt", 3, "Gresults/s", 1e9), ("rcp", 4, "Gresults/s", 1e9),
              ("iadd", 5, "T thread-inst/s", 1e12), ("issue", 6, "T thread-inst/s", 1e12)]


def bench_peaks(args):
    """Throughput of the execution units on all SMs (mc_peak_run), each kind
    timed by CUDA events over 5 launches of about 25 ms, clocks sampled."""
    import torch
    import paper_1308_1464_gb300 as mc
    from paper_1308_1464_gb300 import _build
    torch.cuda.set_device(0)
    _build.build()
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    sink = torch.zeros(1, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"sms": sms, "device": props.name, "blocks_per_sm": 8, "threads_per_block": 256}
    with ClockSampler(0) as clk:
        for name, kind, unit, scale in PEAK_KINDS:
            iters = 64
            for _ in range(8):   # grow until one launch takes about 25 ms
                mc.peak_run(kind, 8, iters, sink.data_ptr(), sh)
                e0.record(stream)
                mc.peak_run(kind, 8, iters, sink.data_ptr(), sh)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                if ms > 15.0:
                    break
                iters = int(iters * min(16.0, 25.0 / max(ms, 1e-3)))
            e0.record(stream)
            ops = 0.0
            for _ in range(5):
                ops += mc.peak_run(kind, 8, iters, sink.data_ptr(), sh)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            out[name] = {"value": round(ops / (ms * 1e-3) / scale, 3), "unit": unit,
                         "ms_per_launch": round(ms / 5, 3), "iters": iters}
            if ms / 5 < 1.0:   # the loop did not take the time its count implies
                out[name]["value"] = None
                out[name]["note"] = "launch too short to be the counted work; not a rate"
    out["clocks"] = clk.summary()
    mhz = out["clocks"].get("sm_mhz") or 0
    if mhz:
        # warp instructions issued per cycle per SM (4 schedulers: at most 4)
        out["issue"]["warp_inst_per_clk_per_sm"] = round(
            out["issue"]["value"] * 1e12 / 32 / sms / (mhz * 1e6), 3)
    line = {"metric": "peak throughput", "peaks": out}
    if args.peaks_out:
        with open(args.peaks_out, "w") as f:
            json.dump(out, f, indent=1)
    print(json.dumps(line))


def time_large_grid(args, wl, ctx, a, b, q0, dt0, stream, sh, world):
    """A state larger than the L2: the K steps run as one timed region
    (graph-captured attempts of mc_advance, the time-step rule on the device),
    and the fused step alone is timed over 50 back-to-back launches."""
    import torch
    # warm-up (also builds the cached step graphs)
    t_sim, dt, inb, _ = ctx.advance(a.ptr, b.ptr, args.warmup, wl["cfl"], 1.0, 0.0, dt0, sh)
    qa, qb = (b, a) if inb else (a, b)
    ctx.advance(qa.ptr, qb.ptr, min(args.steps, 50), wl["cfl"], 1.0, t_sim, dt, sh)  # graph build
    a.upload(q0)
    qa, qb = a, b
    t_sim, dt, inb, _ = ctx.advance(qa.ptr, qb.ptr, args.warmup, wl["cfl"], 1.0, 0.0, dt0, sh)
    if inb:
        qa, qb = qb, qa
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        ev0.record(stream)
        t_sim2, dt2, inb2, nrej = ctx.advance(qa.ptr, qb.ptr, args.steps, wl["cfl"], 1.0, t_sim,
                                              dt, sh)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    # the fused step alone, CUDA events on its stream
    if inb2:
        qa, qb = qb, qa
    ctx.bc_fill(qa.ptr, sh)
    reps = 50
    for _ in range(3):
        ctx.sweep(qa.ptr, qb.ptr, dt2, sh)
    torch.cuda.synchronize()
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    for _ in range(reps):
        ctx.sweep(qa.ptr, qb.ptr, dt2, sh)
    k1.record(stream)
    torch.cuda.synchronize()
    return ms, nrej, clk.summary(), k0.elapsed_time(k1) / reps


def time_small_grid(args, wl, ctx, a, b, q0, l2, stream, sh, world, dt0):
    """A state smaller than the L2 (the small fixed-dt case, or a grid
    workload run at a small --size with half its initial dt held fixed, so
    that the Courant number stays below one as the waves speed up): runs of
    iter_steps steps (ghost fill + fused step each, mc_step without a
    read-back), each run timed by CUDA events after an L2 flush; the fused
    step alone is timed the same way, one flushed launch at a time.  The
    host enqueues while the flush runs, so the events see GPU time only."""
    import torch
    dt = wl.get("fixed_dt", 0.5 * dt0)
    it_steps = wl.get("iter_steps", 10)
    assert args.steps % it_steps == 0, f"steps must be a multiple of {it_steps}"
    qa, qb = a, b
    for _ in range(args.warmup):
        ctx.step(qa.ptr, qb.ptr, dt, want_smax=False, stream=sh)
        qa, qb = qb, qa
    a.upload(q0)
    qa, qb = a, b
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total = 0.0
    with ClockSampler(torch.cuda.current_device()) as clk:
        for _ in range(args.steps // it_steps):
            l2()
            ev0.record(stream)
            for _ in range(it_steps):
                ctx.step(qa.ptr, qb.ptr, dt, want_smax=False, stream=sh)
                qa, qb = qb, qa
            ev1.record(stream)
            ev1.synchronize()
            total += ev0.elapsed_time(ev1)
    reps, kms = 20, 0.0
    ctx.bc_fill(qa.ptr, sh)
    for _ in range(reps):
        l2()
        ev0.record(stream)
        ctx.sweep(qa.ptr, qb.ptr, dt, sh)
        ev1.record(stream)
        ev1.synchronize()
        kms += ev0.elapsed_time(ev1)
    note = ("state %.2f MB, smaller than the %.0f MB L2: runs of %d steps, L2 flushed "
            "(a %.0f MB write) before each" % (ctx.layout.bytes / 1e6, l2.l2_bytes / 1e6, it_steps,
                                                 2 * l2.l2_bytes / 1e6))
    return total, 0, clk.summary(), kms / reps, note


def bench_grid(args, wl, rank, world, sub=False, key=None):
    """One grid workload: K time steps in one timed region (graph-captured
    mc_advance) or runs of a few steps after an L2 flush for a state smaller
    than the L2, plus the fused step alone; with sub, the record of a further
    configuration (no end-to-end or CPU-baseline legs)."""
    import torch
    import paper_1308_1464_gb300 as mc
    from paper_1308_1464_gb300.state import DeviceState

    key = key or args.workload      # the workload's name in WORKLOADS (its ncu records)
    # the committed ncu counts were taken at the workload's own size
    same_size = key in WORKLOADS and WORKLOADS[key]["n"] == wl["n"]
    p, g = make_problem(mc, wl)
    n_cells = p.mx * p.my
    ctx = mc.Context(p)
    lay = ctx.layout
    a, b = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
    npdt = np.float64 if p.dtype == mc.F64 else np.float32
    q0 = np.ascontiguousarray(g.q.astype(npdt))
    a.upload(q0)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    smax0 = ctx.max_cell_speed(a.ptr, sh)
    dt0 = wl["cfl"] / smax0
    if args.kernel_only:
        for _ in range(args.kernel_only):
            ctx.step(a.ptr, b.ptr, dt0, want_smax=False, stream=sh)
        torch.cuda.synchronize()
        print(json.dumps({"kernel_only": args.kernel_only, "workload": wl["desc"]}))
        ctx.close()
        return None

    l2 = L2Flush(torch)
    if lay.bytes < l2.l2_bytes:
        ms, nrej, clocks, kms, l2_note = time_small_grid(args, wl, ctx, a, b, q0, l2, stream, sh,
                                                         world, dt0)
        launches = (1 + sweep_kernels(mc, p)) * args.steps
    else:
        ms, nrej, clocks, kms = time_large_grid(args, wl, ctx, a, b, q0, dt0, stream, sh, world)
        l2_note = "inputs larger than L2 (%.0f MB per state, %.0f MB L2)" % (lay.bytes / 1e6,
                                                                           l2.l2_bytes / 1e6)
        # per attempt: the ghost fill, the step kernel, and either the FP64
        # guard's kernel (which then applies the dt rule) or the dt rule
        launches = 3 * (args.steps + nrej)
    del l2
    ms = max_over_ranks(ms, world, "cuda")
    value = replica_throughput(ms, world, n_cells, args.steps)
    solves = world * ((p.mx + 1) * p.my + p.mx * (p.my + 1)) * args.steps / (ms * 1e-3)
    alg_bytes = 2 * n_cells * p.meqn * lay.elem_bytes
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / (kms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4),
                "traffic": ncu_traffic(key) if same_size else None,
                "kernel": "ctu_sweep_kernel", "kernel_ms": round(kms, 4),
                "algorithmic_bytes_per_launch": alg_bytes, "peak_source": f"{peak_kind} HBM copy"}
    f64 = ncu_fp64(key) if p.dtype == mc.F64 and same_size else None
    if f64 is not None:
        # an FP64 step is bound by the FP64 pipe: counted FP64 flops over the
        # live kernel time, against the nominal FP64 rate
        tf = f64["fp64_flops_per_launch"] / (kms * 1e-3) / 1e12
        pk64, pk64_src = fp64_peak()
        roofline = {"bound": "alu", "achieved": round(tf, 4), "peak": pk64,
                    "unit": "TFLOP/s", "frac": round(tf / pk64, 4),
                    "traffic": f64["dram_bytes_per_launch"], "kernel": "ctu_sweep_kernel",
                    "kernel_ms": round(kms, 4), "fp64_pipe_active_pct": f64["fp64_pipe_active_pct"],
                    "hbm_frac": round(achieved / peak, 4),
                    "peak_source": pk64_src,
                    "flops_source": "FP64 thread instructions of one launch counted by ncu on these "
                                    "sources (FMA = 2 flops, add and multiply = 1)"}
    # end to end through the host-buffer C-ABI call (pinned host memory)
    e2e = None
    if not args.no_e2e and not sub:
        host0 = torch.from_numpy(q0).pin_memory()
        hostq = torch.empty_like(host0).pin_memory()
        nsteps_e2e = 100
        ctx.advance_host(host0.data_ptr(), hostq.data_ptr(), a.ptr, b.ptr, nsteps_e2e,
                         wl["cfl"], 1.0, 0.0, dt0, sh)
        reps_e2e = 3
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps_e2e):
            ctx.advance_host(host0.data_ptr(), hostq.data_ptr(), a.ptr, b.ptr, nsteps_e2e,
                             wl["cfl"], 1.0, 0.0, dt0, sh)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        nbytes = host0.numel() * host0.element_size()
        e2e = {"value": world * n_cells * nsteps_e2e * reps_e2e / el, "unit": "cell-updates/s",
               "h2d_bytes_per_step": nbytes / nsteps_e2e, "d2h_bytes_per_step": nbytes / nsteps_e2e,
               "steps_per_call": nsteps_e2e,
               "note": "mc_advance_host: dense host state in, 100 steps, dense host state out"}

    # the exact-solution solver: the same timed steps with the learned
    # pressure seed, and Newton updates per normal solve with either seed
    seeds = None
    if wl["solver"] == "euler_godunov":
        from paper_1308_1464_gb300.seednet import train_seed_net
        net, losses, train_s = train_seed_net(ntrain=1 << 22, epochs=12, gamma=GAMMA)
        seeds = {"train_rows": 1 << 22, "train_epochs": 12, "train_s": round(train_s, 2)}
        for name, nn in (("plain", None), ("learned", net)):
            ctx.set_seed_net(nn)
            a.upload(q0)
            t1, d1, i1, _ = ctx.advance(a.ptr, b.ptr, args.warmup, wl["cfl"], 1.0, 0.0, dt0, sh)
            x, y = (b, a) if i1 else (a, b)
            ctx.newton_stats(reset=True, stream=sh)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.advance(x.ptr, y.ptr, args.steps, wl["cfl"], 1.0, t1, d1, sh)
            e1.record(stream)
            torch.cuda.synchronize()
            sms = e0.elapsed_time(e1)
            upd, nsolve = ctx.newton_stats(reset=True, stream=sh)
            seeds[name] = {"value": n_cells * args.steps / (sms * 1e-3), "ms_per_step": sms / args.steps,
                           "newton_updates_per_solve": upd / max(nsolve, 1)}
        ctx.set_seed_net(None)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not sub:
        cpu = cpu_baseline(wl)

    if rank == 0:
        line = {
            "metric": "cell-updates/s", "value": value, "unit": "cell-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": wl["dtype"], "data": "synthetic",
            "config": {"workload": wl["desc"], "mx": p.mx, "my": p.my,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": l2_note, "rejected_steps": nrej},
            "riemann_solves_per_s": solves,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clocks,
        }
        if seeds is not None:
            line["pressure_seed"] = seeds
    ctx.close()
    return line if rank == 0 else None




def bench_blocks(args, wl, rank, world):
    """A decomposed grid: px x py blocks of n x n cells each (the workload's
    n, so the work per block stays fixed as blocks are added: weak scaling),
    one block per rank under torchrun, or all of them held by this process
    with --blocks on one rank.  Each attempt of a step exchanges the two
    ghost layers of every shared side (NCCL point-to-point of device strips,
    or device copies within the process), runs the fused step with the
    device dt, max-reduces the speed maximum on the device and applies the
    dt rule on the device; the host reads the time-step state once per
    advance call.  The timed region is K accepted steps of one call."""
    import torch
    import paper_1308_1464_gb300 as mc
    from paper_1308_1464_gb300.blocks import (Block, Decomposition, DeviceBlockOps, DeviceStepper,
                                              DistTransport)
    from paper_1308_1464_gb300.state import DeviceState

    px, py = block_shape(world, args.blocks)
    if world > 1 and px * py != world:
        raise SystemExit(f"--blocks {px}x{py} needs {px * py} ranks, not {world}")
    n = wl["n"]
    mx, my = px * n, py * n
    glob, _ = make_problem(mc, wl, mx, my, window=(0, 0, 1, 1))
    decomp = Decomposition(glob, px, py)
    mine = [rank] if world > 1 else list(range(px * py))
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    blocks, qas, qbs, q0s, keep = [], [], [], [], []
    for r in mine:
        e = decomp.extent(r)
        _, g = make_problem(mc, wl, mx, my, window=(e.i0, e.j0, e.mx, e.my))
        ctx = mc.Context(decomp.local_problem(r))
        b = Block(decomp, r, DeviceBlockOps(ctx, sh))
        a, bb = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
        npdt = np.float64 if glob.dtype == mc.F64 else np.float32
        q0 = np.ascontiguousarray(g.q.astype(npdt))
        a.upload(q0)
        blocks.append(b)
        qas.append(a.ptr)
        qbs.append(bb.ptr)
        q0s.append(q0)
        keep.append((ctx, a, bb))
    transport = DistTransport() if world > 1 else None
    stepper = DeviceStepper(blocks, transport)
    dt0 = wl["cfl"] / stepper.max_cell_speed(qas)

    # warm-up, then the timed K steps from the warmed-up state
    t_sim, dt, inb, _ = stepper.advance(qas, qbs, args.warmup, wl["cfl"], 1.0, 0.0, dt0)
    cur_a, cur_b = (qbs, qas) if inb else (qas, qbs)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        ev0.record(stream)
        t2, dt2, inb2, nrej = stepper.advance(cur_a, cur_b, args.steps, wl["cfl"], 1.0, t_sim, dt)
        ev1.record(stream)
        torch.cuda.synchronize()
    rdev = "cpu" if world > 1 and torch.distributed.get_backend() == "gloo" else "cuda"
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, rdev)
    ncells = n * n * len(mine)
    value = world * ncells * args.steps / (ms * 1e-3)

    # kernel launches of one attempt on this process: per direction the
    # packs, unpacks and the directional fill; the step's kernels; the dt rule
    per_attempt = 0
    for b in blocks:
        for d in (0, 1):
            sends, recvs = decomp.messages(b.rank, d)
            per_attempt += len(sends) + len(recvs) + 1
        per_attempt += sweep_kernels(mc, b.problem) + 1

    # the fused step of the first held block alone (CUDA events on its stream)
    ctx0 = keep[0][0]
    q_in, q_out = (cur_b[0], cur_a[0]) if inb2 else (cur_a[0], cur_b[0])
    ctx0.bc_fill(q_in, sh)
    for _ in range(3):
        ctx0.sweep(q_in, q_out, dt2, sh)
    torch.cuda.synchronize()
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 50
    k0.record(stream)
    for _ in range(reps):
        ctx0.sweep(q_in, q_out, dt2, sh)
    k1.record(stream)
    torch.cuda.synchronize()
    kms = k0.elapsed_time(k1) / reps
    lay = ctx0.layout
    alg_bytes = 2 * n * n * glob.meqn * lay.elem_bytes
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / (kms * 1e-3) / 1e9
    # a block runs the single grid's kernel at the same size: its counters apply
    same_size = args.workload in WORKLOADS and WORKLOADS[args.workload]["n"] == n
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4),
                "traffic": ncu_traffic(args.workload) if same_size else None,
                "kernel": "ctu_sweep_kernel", "kernel_ms": round(kms, 4),
                "algorithmic_bytes_per_launch": alg_bytes, "peak_source": f"{peak_kind} HBM copy"}

    # end to end: each block's state from pinned host memory, 100 steps,
    # each block's state back to pinned host memory
    e2e = None
    if not args.no_e2e:
        hosts = [torch.from_numpy(q0).pin_memory() for q0 in q0s]
        backs = [torch.empty_like(h).pin_memory() for h in hosts]
        nsteps_e2e = 100

        def dense_view(state, h):
            return state.buf[:h.numel() * h.element_size()].view(h.dtype)

        def e2e_once():
            # one contiguous copy per block each way, staged in the spare
            # buffer and repacked on the device (mc_repack)
            for (ctx, a, bb), h in zip(keep, hosts):
                dense_view(bb, h).copy_(h.view(-1), non_blocking=True)
                ctx.repack(bb.ptr, a.ptr, True, sh)
            _, _, ib, _ = stepper.advance(qas, qbs, nsteps_e2e, wl["cfl"], 1.0, 0.0, dt0)
            for (ctx, a, bb), h in zip(keep, backs):
                res, spare = (bb, a) if ib else (a, bb)
                ctx.repack(res.ptr, spare.ptr, False, sh)
                h.view(-1).copy_(dense_view(spare, h), non_blocking=True)
            torch.cuda.synchronize()

        e2e_once()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        e2e_once()
        el = max_over_ranks((time.perf_counter() - t0) * 1e3, world, rdev) * 1e-3
        nbytes = sum(h.numel() * h.element_size() for h in hosts)
        e2e = {"value": world * ncells * nsteps_e2e / el,
               "unit": "cell-updates/s", "h2d_bytes_per_step": nbytes / nsteps_e2e,
               "d2h_bytes_per_step": nbytes / nsteps_e2e, "steps_per_call": nsteps_e2e,
               "note": "per block: dense host state in (one copy, mc_repack), 100 decomposed "
                       "steps (DeviceStepper), dense host state out (mc_repack, one copy)"}

    line = None
    if rank == 0:
        line = {
            "metric": "cell-updates/s", "value": value, "unit": "cell-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": wl["dtype"], "data": "synthetic",
            "config": {"workload": wl["desc"].replace(f"{n}x{n}", f"{mx}x{my}")
                       + f", {px}x{py} blocks of {n}x{n}",
                       "mx": mx, "my": my, "blocks": [px, py],
                       "parallelism": "blocks" if world > 1 else f"blocks ({px * py} on one GPU)",
                       "transport": (DistTransport.__name__ + " " + torch.distributed.get_backend()
                                     if world > 1 else "device copies"),
                       "l2": "inputs larger than L2 (%.0f MB per block state)" % (lay.bytes / 1e6),
                       "rejected_steps": nrej},
            "roofline": roofline, "cpu_baseline": None, "e2e": e2e,
            "gpu_launches": per_attempt * (args.steps + nrej), "clocks": clk.summary(),
        }
    for ctx, _, _ in keep:
        ctx.close()
    return line


def compact(line, keep=("metric", "value", "unit", "ms_per_step", "steps", "warmup", "dtype",
                         "riemann_solves_per_s", "roofline", "clocks", "gpu_launches")):
    out = {k: line[k] for k in keep if k in line}
    out["workload"] = line.get("config", {}).get("workload")
    return out


def bench_configs(args):
    """The further configurations of the benchmark (acoustics 128^2 FP64, the
    dam break in FP64, Euler four quadrants in FP32, 2000 batched patches,
    2^24 exact Riemann problems), each timed briefly on this GPU with CUDA
    events and its own clock record, as sub-records of the one JSON line."""
    import copy
    sub = copy.copy(args)
    sub.steps, sub.warmup, sub.light = 20, 5, True
    out = {}
    for key, name in (("acoustics_128_fp64", "acoustics"), ("swe_4096_fp64", "swe64"),
                      ("euler_4096_fp32", "euler32")):
        t0 = time.perf_counter()
        out[key] = compact(bench_grid(sub, WORKLOADS[name], 0, 1, sub=True, key=name))
        out[key]["wall_s"] = round(time.perf_counter() - t0, 1)
    t0 = time.perf_counter()
    bsub = copy.copy(sub)
    bsub.blocks, bsub.no_e2e = "2x1", True
    rec = compact(bench_blocks(bsub, WORKLOADS["swe32"], 0, 1))
    rec["parallelism"] = ("2x1 blocks of 4096x4096 on one GPU, halo strips by device copies, "
                          "each attempt replayed from a CUDA graph")
    rec["wall_s"] = round(time.perf_counter() - t0, 1)
    out["swe_blocks_2x1_fp32"] = rec
    t0 = time.perf_counter()
    bl = bench_batch(sub, 0, 1)
    rec = compact(bl)
    for k in ("per_step_launch", "plain", "batched_over_per_step_launch", "batched_over_plain"):
        rec[k] = bl[k]
    rec["tune_policy"] = bl["config"].get("tune_policy")
    rec["tuned_over_as_created"] = bl["config"].get("tuned_over_as_created")
    rec["wall_s"] = round(time.perf_counter() - t0, 1)
    out["batch_2000_fp32"] = rec
    t0 = time.perf_counter()
    ex = bench_exact(sub, 0, 1)
    rec = compact(ex)
    for k in ("plain", "learned", "plain_mixed", "learned_mixed"):
        rec[k] = ex[k]
    rec["train_s"] = ex["config"].get("train_s")
    rec["wall_s"] = round(time.perf_counter() - t0, 1)
    out["exact_2p24"] = rec
    return out


def bench_next_rows(args):
    """The step's further forms, each timed briefly on this GPU like the
    further configurations: the van Leer limiter with transverse option 2
    (f1), advection and variable-coefficient acoustics (f2), Euler with the
    exact-solution normal solve and the learned pressure seed (f3), and
    refined patches with refluxing against the uniformly fine grid (f4)."""
    import copy
    sub = copy.copy(args)
    sub.steps, sub.warmup, sub.light = 20, 5, True
    out = {}
    for key, name in (("f1_swe_vanleer_trans2_4096_fp32", "swe32t2"),
                      ("f2_advection_8192_fp32", "adv32"),
                      ("f2_acoustics_var_4096_fp32", "acvar32"),
                      ("f3_euler_godunov_4096_fp32", "eulg32")):
        t0 = time.perf_counter()
        line = bench_grid(sub, WORKLOADS[name], 0, 1, sub=True, key=name)
        rec = compact(line)
        if "pressure_seed" in line:
            rec["pressure_seed"] = line["pressure_seed"]
        rec["wall_s"] = round(time.perf_counter() - t0, 1)
        out[key] = rec
    t0 = time.perf_counter()
    am = bench_amr(sub, 0, 1)
    rec = compact(am)
    rec["uniform_fine"] = am["uniform_fine"]
    rec["wall_s"] = round(time.perf_counter() - t0, 1)
    out["f4_amr_dambreak_4096_fp32"] = rec
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="swe32", choices=sorted(WORKLOADS) + ["batch", "exact", "amr"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the records of the further configurations and forms in the default run")
    ap.add_argument("--peaks", action="store_true",
                    help="time the execution-unit microbenchmarks (FFMA, FFMA2, DFMA, MUFU, issue) and exit")
    ap.add_argument("--peaks-out", default="", help="with --peaks: also write the JSON to this file")
    ap.add_argument("--kernel-only", type=int, default=0, metavar="K",
                    help="profiling aid: run K stand-alone fused steps (mc_step) and exit")
    ap.add_argument("--size", type=int, default=0,
                    help="a grid of n x n cells (per block with --blocks) in place of the workload's")
    ap.add_argument("--blocks", default="",
                    help="PXxPY: a grid workload decomposed into PX x PY blocks of n x n cells "
                         "(under torchrun one block per rank, PX * PY = ranks; on one rank all "
                         "blocks on this GPU); with several ranks the default is the most nearly "
                         "square shape")
    ap.add_argument("--dist-backend", default="nccl", choices=["nccl", "gloo"],
                    help="torch.distributed backend of a multi-rank run")
    args = ap.parse_args()
    if args.peaks:
        return bench_peaks(args)
    if args.workload in ("batch", "exact", "amr"):
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle baseline is timed "
                              "for the grid workloads only"}))
            return
        import torch
        from paper_1308_1464_gb300 import _build
        rank, world, local = dist_info()
        torch.cuda.set_device(local)
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl")
        _build.build()
        line = {"batch": bench_batch, "exact": bench_exact, "amr": bench_amr}[args.workload](args, rank, world)
        if rank == 0:
            print(json.dumps(line))
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl)
    assert args.warmup >= 3, "at least 3 warm-up steps"

    import torch
    from paper_1308_1464_gb300 import _build

    rank, world, local = dist_info()
    # gloo ranks (a test of the multi-rank path) may share one GPU; NCCL ranks never do
    torch.cuda.set_device(local if args.dist_backend == "nccl"
                          else local % max(1, torch.cuda.device_count()))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(args.dist_backend)
    _build.build()
    if args.size:
        wl = dict(wl, n=args.size, desc=wl["desc"].replace("%dx%d" % (wl["n"], wl["n"]),
                                                           "%dx%d" % (args.size, args.size)))
    if (world > 1 or args.blocks) and not args.kernel_only:
        line = bench_blocks(args, wl, rank, world)
    else:
        line = bench_grid(args, wl, rank, world)
    if (line is not None and args.workload == "swe32" and world == 1 and not args.no_configs
            and not args.blocks):
        line["configs"] = bench_configs(args)
        blk = line["configs"]["swe_blocks_2x1_fp32"]
        blk["over_single_grid"] = round(blk["value"] / line["value"], 4)
        line["next_rows"] = bench_next_rows(args)
    if rank == 0 and line is not None:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
