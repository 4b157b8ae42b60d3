"""Autotuner of the fused schedule.

The fused schedule has two free parameters: the time-tile width W and the
shared memory a block may use (which sets the cone sizes and how many blocks
share an SM).  For each candidate pair the planner picks the level grouping
with its cost model (fdmt_plan_ex); the autotuner then times every candidate
plan, and the plain schedule, on the device with CUDA events and keeps the
fastest.  Results are cached per (shape, dtype, band, GPU) in a JSON file
(``$FDMT_AUTOTUNE_CACHE`` or ``~/.cache/paper_1411_5373_gb300/autotune.json``).
"""
from __future__ import annotations

import json
import os

from .plan import Plan
from ._native import FdmtError

TILES = (0, 128, 256, 512)  # 0 = tile chosen per level group by the planner
BUDGETS_KIB = (40, 56, 72, 96, 112, 150, 200)


def _cache_path():
    return os.environ.get("FDMT_AUTOTUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "paper_1411_5373_gb300", "autotune.json")


def _key(f_min, f_max, nf, nt, nd, dtype):
    import torch
    prop = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{prop.name}/{prop.multi_processor_count}sm/{nf}x{nt}x{nd}/{dtype}/{f_min:g}-{f_max:g}"


def _time_plan(plan, x, out, reps):
    import torch
    ws = plan.workspace(x.device)
    for _ in range(2):
        plan.execute(x, out=out, workspace=ws)
    s = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        plan.execute(x, out=out, workspace=ws)
    e1.record(s)
    torch.cuda.synchronize()
    plan.device_status()
    return e0.elapsed_time(e1) / reps


def autotune(f_min, f_max, nf, nt, nd, dtype="f32", reps=10, use_cache=True, verbose=False):
    """Return the fastest schedule for this shape as a dict
    {"schedule": "plain"|"fused", "tile", "smem_budget", "bounds", "ms", "trials"}."""
    import torch
    key = _key(f_min, f_max, nf, nt, nd, dtype)
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as fh:
                cache = json.load(fh)
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return cache[key]
    dev = torch.device("cuda", torch.cuda.current_device())
    in_dtype = torch.uint8 if dtype == "u8" else torch.float32
    out_dtype = torch.int32 if dtype == "u8" else torch.float32
    if dtype == "u8":
        x = torch.randint(0, 256, (nf, nt), dtype=torch.uint8, device=dev)
    else:
        x = torch.randn((nf, nt), dtype=torch.float32, device=dev)
    assert x.dtype == in_dtype
    out = torch.empty((nd, nt), dtype=out_dtype, device=dev)
    trials = []
    plain = Plan(f_min, f_max, nf, nt, nd, dtype, schedule="plain")
    trials.append({"schedule": "plain", "tile": 0, "smem_budget": 0, "bounds": [],
                   "ms": _time_plan(plain, x, out, reps)})
    plain.close()
    seen = set()
    for tile in TILES:
        for kib in BUDGETS_KIB:
            try:
                p = Plan(f_min, f_max, nf, nt, nd, dtype, schedule="fused", tile=tile,
                         smem_budget=kib * 1024)
            except FdmtError:
                continue
            w, bounds = p.schedule_info()
            sig = (w, tuple(bounds), len(p.fused_table(1)), kib)
            if sig in seen:
                p.close()
                continue
            seen.add(sig)
            try:
                ms = _time_plan(p, x, out, reps)
            except (FdmtError, RuntimeError):
                p.close()
                continue
            trials.append({"schedule": "fused", "tile": w, "smem_budget": kib * 1024,
                           "bounds": bounds, "ms": ms})
            if verbose:
                print(f"autotune {key}: tile {w} budget {kib} KiB bounds {bounds}: {ms:.4f} ms")
            p.close()
    best = dict(min(trials, key=lambda t: t["ms"]))
    best["trials"] = sorted(trials, key=lambda t: t["ms"])
    cache[key] = best
    if use_cache:
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path, "w") as fh:
                json.dump(cache, fh, indent=1)
        except OSError:
            pass
    return best


def tuned_plan(f_min, f_max, nf, nt, nd, dtype="f32", **kw):
    """A Plan with the autotuned schedule for this shape."""
    best = autotune(f_min, f_max, nf, nt, nd, dtype, **kw)
    if best["schedule"] == "plain":
        return Plan(f_min, f_max, nf, nt, nd, dtype, schedule="plain"), best
    return Plan(f_min, f_max, nf, nt, nd, dtype, schedule="fused", tile=best["tile"],
                smem_budget=best["smem_budget"], bounds=best["bounds"]), best
