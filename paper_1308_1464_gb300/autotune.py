"""Autotuner for the batched step's per-patch work split.

The batched kernel cuts every patch into warp tasks of 29 columns by
`rows` rows; the split decides how many tasks a patch has (parallelism and
load balance across the persistent grid) against the two halo rows each task
re-reads.  Candidate policies map a patch size to its rows; each is timed
through mc_batch_advance with CUDA events and the fastest is applied and, if
a cache path is given, remembered under a key of the patch sizes and the GPU
name.  Results never depend on the split (the kernels are bitwise invariant
to it), only the time does.
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics


def _pow2_clamp(v: float, lo: int, hi: int) -> int:
    r = lo
    while r < hi and r * 2 <= v:
        r *= 2
    return r


POLICIES = {
    "rows8": lambda mx, my: 8,
    "rows16": lambda mx, my: 16,
    "rows32": lambda mx, my: 32,
    "rows64": lambda mx, my: 64,
    "half": lambda mx, my: _pow2_clamp(my / 2, 8, 128),
    "quarter": lambda mx, my: _pow2_clamp(my / 4, 8, 128),
    "whole": lambda mx, my: max(8, my),
}


def cache_key(sizes, device_name: str) -> str:
    h = hashlib.sha1(repr(sorted(sizes)).encode()).hexdigest()[:16]
    return f"{device_name}|{len(sizes)}|{h}"


def tune_batch(batch, sizes, reset, nsteps: int = 4, cfl: float = 0.9, repeats: int = 3,
               cache_path: str | None = None, policies=None):
    """Pick the fastest policy for `batch` (a paper_1308_1464_gb300.Batch).

    sizes: (mx, my) per patch; reset: callable restoring the initial state
    between trials.  Returns (policy name, {policy: median ms}).
    """
    import torch
    policies = policies or POLICIES
    key = cache_key(sizes, torch.cuda.get_device_name())
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache and cache[key]["policy"] in policies:
            name = cache[key]["policy"]
            batch.set_tile_rows([policies[name](mx, my) for mx, my in sizes])
            return name, cache[key]["timings"]
    timings = {}
    stream = torch.cuda.current_stream()
    for name, f in policies.items():
        batch.set_tile_rows([f(mx, my) for mx, my in sizes])
        reset()
        batch.advance(nsteps, cfl, stream=stream.cuda_stream)   # builds the graph
        ts = []
        for _ in range(repeats):
            reset()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            batch.advance(nsteps, cfl, stream=stream.cuda_stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        timings[name] = statistics.median(ts)
    best = min(timings, key=timings.get)
    batch.set_tile_rows([policies[best](mx, my) for mx, my in sizes])
    reset()
    if cache_path:
        cache = {}
        if os.path.exists(cache_path):
            with open(cache_path) as f:
                cache = json.load(f)
        cache[key] = {"policy": best, "timings": timings}
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return best, timings
