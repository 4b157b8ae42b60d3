"""Autotuner of the fused schedule.

The fused schedule has three free choices: the level grouping (which merge
levels share a launch), and per launch the time-tile width W and the shared
memory a block may use (which sets the cone sizes and how many blocks share
an SM).  Phase 1 times whole plans: for each (W, budget) candidate the
planner's cost model picks the grouping (fdmt_plan_ex), and the plain
schedule is timed too.  Phase 2 keeps the best groupings and, since the
launches of a grouping are independent, times every (W, budget) for every
launch at once with the library's per-launch profiler and combines the best
choice per launch.  All timing is on the device (CUDA events).  Results are
cached per (shape, dtype, band, GPU, kernel sources) in a JSON file
(``$FDMT_AUTOTUNE_CACHE`` or ``~/.cache/paper_1411_5373_gb300/autotune.json``);
a table shipped with the package (``tuned_schedules.json``, schedules tuned on
a GB300 for the benchmark shapes) is consulted after it, read only.  Entries
are keyed by a hash of the fused-schedule sources, so a changed kernel or
planner is tuned afresh.
"""
from __future__ import annotations

import hashlib
import json
import os

from .plan import Plan
from ._native import FdmtError

TILES = (0, 256, 448, 512, 960)  # 0 = tile chosen per level group by the planner
BUDGETS_KIB = (56, 64, 72, 80, 96, 112, 150)
GROUP_TILES = (256, 384, 448, 512, 960)
PHASE2_GROUPINGS = 3
SHAPES = (  # the benchmark shapes the shipped table covers: (f_min, f_max, nf, nt, nd, dtype)
    (1200.0, 1600.0, 1024, 65536, 1024, "f32"),
    (1200.0, 1600.0, 1024, 65536, 1024, "u8"),
    (1200.0, 1600.0, 1024, 65536, 1024, "f16state"),
    (1100.0, 1700.0, 4096, 1 << 20, 4096, "f32"),
    (1100.0, 1700.0, 4096, 1 << 20, 4096, "f16state"),
)


SHIPPED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_schedules.json")
_SOURCES = ("fdmt_fused.cu", "fdmt_fused_f32.cu", "fdmt_fused_u8.cu", "fdmt_fused_launch.cuh", "fdmt_fused_dev.cuh",
            "fdmt_fused.h", "fdmt_fused_plan.cpp", "fdmt_common.cuh", "fdmt_tma.h")


def _cache_path():
    return os.environ.get("FDMT_AUTOTUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "paper_1411_5373_gb300", "autotune.json")


def sources_hash():
    """Hash of the fused-schedule sources (kernel and planner)."""
    h = hashlib.sha256()
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc")
    for fn in _SOURCES:
        with open(os.path.join(csrc, fn), "rb") as fh:
            h.update(fn.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def _key(f_min, f_max, nf, nt, nd, dtype):
    import torch
    prop = torch.cuda.get_device_properties(torch.cuda.current_device())
    return (f"{prop.name}/{prop.multi_processor_count}sm/{nf}x{nt}x{nd}/{dtype}/{f_min:g}-{f_max:g}"
            f"/src={sources_hash()}")


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


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
    cache = _load(path) if use_cache else {}
    if use_cache:
        if key in cache:
            return cache[key]
        shipped = _load(SHIPPED)
        if key in shipped:
            return shipped[key]
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
    # Phase 2: per-launch tuning of the best groupings, and of a few regular
    # ones the cost model may rank too low.
    groupings = []
    for t in sorted(trials, key=lambda t: t["ms"]):
        if t["schedule"] == "fused" and t["bounds"] not in groupings:
            groupings.append(t["bounds"])
        if len(groupings) == PHASE2_GROUPINGS:
            break
    for b in _regular_groupings(None, nf):
        if b not in groupings:
            groupings.append(b)
    for bounds in groupings:
        ng = len(bounds) - 1
        codes = [bounds[i] * 100 + bounds[i + 1] for i in range(ng)]
        best_g = [None] * ng
        for tile in GROUP_TILES:
            for kib in BUDGETS_KIB:
                try:
                    p = Plan(f_min, f_max, nf, nt, nd, dtype, schedule="fused", tile=tile,
                             smem_budget=kib * 1024, bounds=bounds)
                except FdmtError:
                    continue
                try:
                    per = _time_groups(p, x, out, reps, codes)
                except (FdmtError, RuntimeError):
                    p.close()
                    continue
                p.close()
                for g in range(ng):
                    if per[g] is not None and (best_g[g] is None or per[g] < best_g[g][0]):
                        best_g[g] = (per[g], tile, kib * 1024)
        if any(b is None for b in best_g):
            continue
        tiles = [b[1] for b in best_g]
        budgets = [b[2] for b in best_g]
        try:
            p = Plan(f_min, f_max, nf, nt, nd, dtype, schedule="fused", bounds=bounds,
                     group_tiles=tiles, group_budgets=budgets, smem_budget=max(budgets))
            ms = _time_plan(p, x, out, reps)
            p.close()
        except (FdmtError, RuntimeError):
            continue
        trials.append({"schedule": "fused", "tile": tiles[0], "smem_budget": max(budgets),
                       "bounds": bounds, "group_tiles": tiles, "group_budgets": budgets, "ms": ms})
        if verbose:
            print(f"autotune {key}: per-launch {bounds} tiles {tiles} budgets {budgets}: {ms:.4f} ms")
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


def _regular_groupings(levels, nf):
    """Level groupings with a first launch of 2 or 3 levels from the input
    and then launches of 2, 3 or 4 levels (the last one takes the rest)."""
    L = levels if levels else max(1, (nf - 1).bit_length())
    out = []
    for first, step in ((3, 3), (3, 2), (2, 2), (3, 4)):
        if L <= first:
            continue
        b = [0, first]
        while b[-1] < L:
            b.append(min(L, b[-1] + step))
        if len(b) >= 4 and b[-1] - b[-2] == 1:
            b.pop(-2)  # no one-level tail: the last launch takes it
        if b not in out:
            out.append(b)
    return out


def ship(path=SHIPPED, reps=10, verbose=True):
    """Tune the benchmark shapes on this GPU and write the shipped table."""
    table = {}
    for f_min, f_max, nf, nt, nd, dtype in SHAPES:
        best = autotune(f_min, f_max, nf, nt, nd, dtype, reps=reps, use_cache=False, verbose=verbose)
        table[_key(f_min, f_max, nf, nt, nd, dtype)] = best
        if verbose:
            print(f"shipped {nf}x{nt}x{nd} {dtype}: {best['schedule']} {best.get('bounds')} {best['ms']:.4f} ms",
                  flush=True)
    with open(path, "w") as fh:
        json.dump(table, fh, indent=1)
    return table


def _time_groups(plan, x, out, reps, codes):
    """Mean device time of each launch of a fused plan, by level code."""
    import torch
    ws = plan.workspace(x.device)
    for _ in range(2):
        plan.execute(x, out=out, workspace=ws)
    torch.cuda.synchronize()
    plan.profile_enable(reps * (len(codes) + 1))
    for _ in range(reps):
        plan.execute(x, out=out, workspace=ws)
    _, rows = plan.profile_read()
    plan.profile_enable(0)
    plan.device_status()
    per = []
    for c in codes:
        ms = [r[2] for r in rows if r[1] == c]
        per.append(sum(ms) / len(ms) if ms else None)
    return per


def tuned_plan(f_min, f_max, nf, nt, nd, dtype="f32", d_min=0, descending=False, **kw):
    """A Plan with the autotuned schedule for this shape (the schedule is
    tuned without an input mapping; d_min / descending only add the mapping
    pass in front of it)."""
    best = autotune(f_min, f_max, nf, nt, nd, dtype, **kw)
    m = dict(d_min=d_min, descending=descending)
    if best["schedule"] == "plain":
        return Plan(f_min, f_max, nf, nt, nd, dtype, schedule="plain", **m), best
    return Plan(f_min, f_max, nf, nt, nd, dtype, schedule="fused", tile=best["tile"],
                smem_budget=best["smem_budget"], bounds=best["bounds"],
                group_tiles=best.get("group_tiles"), group_budgets=best.get("group_budgets"), **m), best


if __name__ == "__main__":
    # python -m paper_1411_5373_gb300.autotune [output.json]: tune the
    # benchmark shapes on the current GPU and write the table
    import sys
    ship(sys.argv[1] if len(sys.argv) > 1 else SHIPPED)
