"""Autotuner for the batched step's per-patch work split.

The batched kernel cuts every patch into warp tasks of 29 columns by `rows`
rows; the split decides how many tasks a patch has (parallelism and load
balance across the persistent grid) against the halo rows each task re-reads
(three per task).  The tuner first times a few global policies (a patch size
to its rows), then refines the best one per size class: patches are grouped
by height, and the rows of each class are chosen in turn (coordinate descent,
largest total work first) among powers of two, every candidate timed through
mc_batch_advance with CUDA events (median of a few runs).  The faster of the
best policy and the refined plan is applied to the batch and, if a cache
path is given, remembered (rows per patch) under a key of the patch sizes,
the GPU name and the tuner version.  Results never depend on the split (the kernels are bitwise
invariant to it), only the time does.
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics

TUNER_VERSION = 2


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

# height classes [lo, hi) of the per-class refinement, and the rows tried
CLASSES = ((0, 24), (24, 48), (48, 96), (96, 192), (192, 1 << 30))
ROW_CHOICES = (8, 16, 32, 64, 128, 256)


def class_of(my: int) -> int:
    for k, (lo, hi) in enumerate(CLASSES):
        if lo <= my < hi:
            return k
    return len(CLASSES) - 1


def rows_from_plan(plan, sizes):
    """Rows per patch of a per-class plan (a list of rows per class); a task
    never needs more rows than its patch has (at least 8)."""
    return [min(int(plan[class_of(my)]), max(8, int(my))) for _, my in sizes]


def plan_from_policy(policy, sizes):
    """The per-class plan closest to a global policy: each class takes the
    rows the policy gives its most common patch height (the class's middle
    for an empty class)."""
    plan = []
    for k, (lo, hi) in enumerate(CLASSES):
        mys = [my for _, my in sizes if class_of(my) == k]
        if mys:
            my = statistics.median_low(mys)
            mx = next(m for m, y in sizes if y == my)
        else:
            my, mx = min(max(lo, 16), 256), 64
        plan.append(int(policy(mx, my)))
    return plan


def refinement_trials(plan, sizes):
    """(class, rows) candidates of the refinement, classes by decreasing
    total cells; rows from ROW_CHOICES up to the first one that covers the
    class's tallest patch (larger ones split the same way)."""
    work = [0] * len(CLASSES)
    tallest = [0] * len(CLASSES)
    for mx, my in sizes:
        k = class_of(my)
        work[k] += mx * my
        tallest[k] = max(tallest[k], my)
    out = []
    for k in sorted(range(len(CLASSES)), key=lambda k: (-work[k], k)):
        if work[k] == 0:
            continue
        for r in ROW_CHOICES:
            out.append((k, r))
            if r >= tallest[k]:
                break
    return out


def cache_key(sizes, device_name: str) -> str:
    h = hashlib.sha1(repr(sorted(sizes)).encode()).hexdigest()[:16]
    return f"{device_name}|{len(sizes)}|{h}|v{TUNER_VERSION}"


def _time(batch, rows, reset, nsteps, cfl, repeats):
    import torch
    if rows is not None:
        batch.set_tile_rows(rows)
    stream = torch.cuda.current_stream()
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
    return statistics.median(ts)


def tune_batch(batch, sizes, reset, nsteps: int = 4, cfl: float = 0.9, repeats: int = 3,
               cache_path: str | None = None, policies=None, refine: bool = True,
               device_name: str | None = None):
    """Pick a work split for `batch` (a paper_1308_1464_gb300.Batch).

    sizes: (mx, my) per patch; reset: callable restoring the initial state
    between trials.  Returns (description, {candidate: median ms}); the
    description names the best global policy and the per-class rows.
    """
    policies = policies or POLICIES
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name()
    key = cache_key(sizes, device_name)
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache and len(cache[key].get("rows", ())) == len(sizes):
            batch.set_tile_rows(cache[key]["rows"])
            return cache[key]["desc"], cache[key]["timings"]
    # the split the batch was created with, for the record
    timings = {"as_created": _time(batch, None, reset, nsteps, cfl, repeats)}
    for name, f in policies.items():
        timings[name] = _time(batch, [f(mx, my) for mx, my in sizes], reset, nsteps, cfl, repeats)
    best = min(policies, key=timings.get)
    rows = [policies[best](mx, my) for mx, my in sizes]
    best_ms = timings[best]
    desc = best
    if refine:
        plan = plan_from_policy(policies[best], sizes)
        plan_ms = _time(batch, rows_from_plan(plan, sizes), reset, nsteps, cfl, repeats)
        timings["plan:" + best] = plan_ms
        for k, r in refinement_trials(plan, sizes):
            if r == plan[k]:
                continue
            trial = list(plan)
            trial[k] = r
            ms = _time(batch, rows_from_plan(trial, sizes), reset, nsteps, cfl, repeats)
            timings[f"class{k}:rows{r}"] = ms
            if ms < plan_ms:
                plan_ms, plan = ms, trial
        if plan_ms < best_ms:
            best_ms, rows = plan_ms, rows_from_plan(plan, sizes)
            desc = f"{best} refined per height class: rows {plan}"
    batch.set_tile_rows(rows)
    reset()
    if cache_path:
        cache = {}
        if os.path.exists(cache_path):
            with open(cache_path) as f:
                cache = json.load(f)
        cache[key] = {"desc": desc, "rows": rows, "timings": timings}
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return desc, timings
