#!/usr/bin/env python
"""FDMT throughput on GB300: (t,DM) cells/s and the HBM roofline fraction.

One step = one whole transform (initialisation + all merge levels) of one
seeded synthetic filterbank that is already resident in HBM.  The default
workload is the single beam Nf=1024, Nt=65536, Nd=1024 in float32 (input and
output 256 MiB each, both larger than the 129 MB L2, so no flush is needed
between steps).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--schedule plain|fused] [--impl ours|reference]

Multi-GPU runs (torchrun, one rank per GPU) process one independent beam per
rank with no data-path collective (weak scaling); the barrier and the
max-over-ranks reduction of the timed interval are the only collectives.
``--impl reference`` times the CPU oracle (the plain Algorithm 1 of the
paper) on a bounded column sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import filterbank_synth as fs  # noqa: E402

WORKLOADS = {
    "single-1k-f32": (fs.SINGLE_1K, "f32"),
    "single-1k-u8": (fs.SINGLE_1K, "u8"),
    "single-1k-f16state": (fs.SINGLE_1K, "f16state"),
    "large-4k-f32": (fs.LARGE_4K, "f32"),
    "large-4k-f16state": (fs.LARGE_4K, "f16state"),
    "small-64-f32": (fs.SINGLE_SMALL, "f32"),
    # forward with per-channel weights plus the adjoint (input and weight
    # gradients) of a seeded output gradient: one training step's FDMT work
    "diff-1k-f32": (fs.DIFF_1K, "f32"),
    # the transform followed by the boxcar search of section 4.2 (widths
    # 1 .. 128): peak value and first time per (row, width)
    "search-1k-u8": (fs.SINGLE_1K, "u8"),
    "search-1k-f32": (fs.SINGLE_1K, "f32"),
    "filterbank-1k-f32": (fs.SINGLE_1K, "f32"),
    # FFT-FDMT (section 5, Algorithm 2): the same transform computed per
    # Fourier bin between a forward and an inverse FFT of the time axis
    "fft-1k-f32": (fs.SINGLE_1K, "f32"),
    "fft-1k-u8": (fs.SINGLE_1K, "u8"),
}
FFT_WORKLOADS = {"fft-1k-f32", "fft-1k-u8"}
DIFFERENTIABLE = {"diff-1k-f32"}
# complex voltages -> STFT filterbank (section 2) -> transform: the input is
# Nf Nt complex64 samples (seeded complex Gaussian noise)
FRONT_END = {"filterbank-1k-f32"}
SEARCH_WIDTHS = {"search-1k-u8": 8, "search-1k-f32": 8}
IN_BYTES = {"f32": 4, "u8": 1, "f16state": 4}
STATE_BYTES = {"f32": 4, "u8": 4, "f16state": 2}
OUT_BYTES = 4
DTYPE_NAME = {"f32": "f32", "u8": "u8->i32", "f16state": "f32 (fp16 state)"}
METRIC = "FDMT (t,DM) cells/s"
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--workload", default="single-1k-f32", choices=sorted(WORKLOADS) + ["batch-64-u8"])
    ap.add_argument("--schedule", default="auto", choices=["auto", "plain", "fused"],
                    help="auto = autotuned (tile, shared-memory budget, level grouping)")
    ap.add_argument("--tile", type=int, default=0, help="fused: time tile (0 = planner)")
    ap.add_argument("--smem-budget", type=int, default=0, help="fused: bytes per block (0 = planner)")
    ap.add_argument("--bounds", default="", help="fused: level boundaries, e.g. 0,2,4,6,8,10 (empty = planner)")
    ap.add_argument("--group-tiles", default="", help="fused, with --bounds: tile per launch")
    ap.add_argument("--group-budgets", default="", help="fused, with --bounds: bytes per block per launch")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--d-min", type=int, default=0,
                    help="single-beam workloads: delay of output row 0 (input pre-shift)")
    ap.add_argument("--descending", action="store_true",
                    help="single-beam workloads: input rows in descending frequency")
    ap.add_argument("--widths", type=int, default=0,
                    help="search workloads: number of boxcar widths K (1..13; default 8)")
    ap.add_argument("--fft-block", type=int, default=0, help="fft workloads: FFT length (0 = planner)")
    ap.add_argument("--fft-bins", type=int, default=0, help="fft workloads: Fourier bins per merge block (0 = planner)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-schedule comparison")
    ap.add_argument("--nt", type=int, default=0,
                    help="profiling: the workload scaled down to this many samples, with the full-size shape's "
                         "schedule (the line says so in config)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# helpers

def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            v = float(json.load(fh)["hbm_gbs"])
        return v, "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def source_hash(files):
    """Hash of the kernel source files a traffic record was taken on."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1411_5373_gb300", "csrc")
    for fn in sorted(files):
        with open(os.path.join(csrc, fn), "rb") as fh:
            h.update(fn.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def schedule_key(plan):
    """The fused schedule as "bounds:tiles", e.g. "0-2-4-6-8-10:512-1024-512-512-512"
    (level boundaries and the time tile of each launch)."""
    g = plan.fused_table(0).reshape(len(plan.schedule_info()[1]) - 1, -1)
    bounds = [int(g[0, 0])] + [int(v) for v in g[:, 1]]
    return "-".join(map(str, bounds)) + ":" + "-".join(str(int(v)) for v in g[:, 7])


def batch_key(cfg):
    """The batch work schedule as a traffic-record key, e.g. "fused:0:57344"."""
    if cfg.get("schedule") == "fused":
        return f"fused:{cfg.get('fused_tile', 0)}:{cfg.get('smem_budget', 0)}"
    if cfg.get("schedule") == "launches":
        return "launches"
    return f"levels:{cfg.get('rows_per_item', 0)}:{cfg.get('tile', 0)}"


def recorded_traffic(kernel, workload, schedule=None):
    """DRAM bytes per launch of `kernel` on `workload` (and, for the fused
    kernels, the schedule "tile:bounds") from a committed ncu summary, if it
    was taken on the kernel's current sources (else None)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        kv = dict(p.split("=", 1) for p in line.split() if "=" in p)
        if kv.get("kernel") != kernel or kv.get("workload") != workload:
            continue
        if "schedule" in kv and kv["schedule"] != schedule:
            continue
        try:
            if source_hash(kv["files"].split(",")) == kv.get("src"):
                return float(kv["bytes_per_launch"])
        except (KeyError, OSError):
            return None
    return None


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(self.REASONS, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "power_w_max": float(max(power)) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def gpu_identifier(torch, dev):
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(dev).uuid).replace("GPU-", "")
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            return vis.split(",")[dev]
        return str(dev)


def algorithmic_bytes(kernel, level, rows, nf, nt, dtype, sizes=None):
    """Bytes a launch must move: every row it reads and writes, once.
    rows[l] = total rows of level l; level L is the output.  sizes maps a
    fused launch (lb, lt) to its (staged, written) bytes per sample."""
    L = len(rows) - 1
    s_in, s_st, s_out = IN_BYTES[dtype], STATE_BYTES[dtype], OUT_BYTES
    if sizes is not None and kernel in ("fused_local", "fused_cone"):
        lo, hi = (0, level) if kernel == "fused_local" else (level // 100, level % 100)
        b_in, b_out = sizes[(lo, hi)]
        return nt * ((nf if lo == 0 else rows[lo]) * b_in + rows[hi] * b_out)
    if kernel == "init":
        return nt * (nf * s_in + rows[0] * s_st)
    if kernel == "merge":
        return nt * (rows[level - 1] * s_st + rows[level] * (s_out if level == L else s_st))
    if kernel == "fused_local":
        return nt * (nf * s_in + rows[level] * (s_out if level == L else s_st))
    if kernel == "fused_cone":
        lo, hi = level // 100, level % 100
        return nt * (rows[lo] * s_st + rows[hi] * (s_out if hi == L else s_st))
    if kernel == "adjoint_merge":  # gradient of level `level` in, level - 1 out (float32)
        return nt * (rows[level] + rows[level - 1]) * 4
    if kernel == "adjoint_merge2":  # two transposed levels: level `level` in, level - 2 out
        return nt * (rows[level] + rows[level - 2]) * 4
    if kernel == "adjoint_init":
        return nt * (rows[0] + nf) * 4
    if kernel == "adjoint_cone":  # fused adjoint launch lt -> lb (level = 100 lb + lt); lb = 0 writes the input gradient
        lo, hi = level // 100, level % 100
        return nt * (rows[hi] + (nf if lo == 0 else rows[lo])) * 4
    if kernel == "adjoint_weights_finalize":  # the weight gradient from the init launch's partials
        return 0
    if kernel == "weights_epilogue":  # input, gradient in; gradient rescaled in place
        return nt * nf * (s_in + 4 + 4)
    if kernel == "map_input":  # raw input in, mapped input out
        return nt * nf * 2 * s_in
    if kernel == "unmap_grad":
        return nt * nf * 2 * 4
    return None


# ---------------------------------------------------------------------------
# CPU oracle baseline (the reference arm and the cpu_baseline key)

def oracle_sample_cells_per_s(w, dtype, seconds_budget, nt_cap=None, adjoint=False, search=0, front=False):
    """Time the oracle (as it stands) on a column sample of the workload:
    all Nf channels and all Nd rows, the first nt_s samples (with `adjoint`,
    the forward transform plus the adjoint of an output gradient; with
    `search` = K, the transform plus the boxcar search of K widths).
    Returns (cells/s, sample description, runs)."""
    import oracle
    T = oracle.build_tables(w.f_min, w.f_max, w.nf, w.nd)
    nt_s = w.nt if nt_cap is None else max(16, min(w.nt, (nt_cap // 16) * 16))
    x = fs.filterbank_u8(w, 0, nt_s) if dtype == "u8" else fs.filterbank_f32(w, 0, nt_s)
    mode = {"f32": "f32", "u8": "i64", "f16state": "f16state"}[dtype]
    g = fs.random_f32(w.seed + 7, w.nd, nt_s).astype(np.float64) if adjoint else None
    if front:
        rng = np.random.Generator(np.random.PCG64([w.seed, 61]))
        v = (rng.standard_normal(w.nf * nt_s) + 1j * rng.standard_normal(w.nf * nt_s)).astype(np.complex64)
    runs, elapsed = 0, 0.0
    while True:
        t0 = time.perf_counter()
        A = oracle.fdmt(oracle.stft_filterbank(v, w.nf) if front else x, T, mode)
        if adjoint:
            oracle.fdmt_adjoint(g, T)
        if search:
            oracle.boxcar_search(A, search)
        elapsed += time.perf_counter() - t0
        runs += 1
        if elapsed >= seconds_budget or runs >= 5:
            break
    cells = float(w.nd) * nt_s * runs
    extra = " + adjoint" if adjoint else (f" + boxcar search of {search} widths" if search else "")
    if front:
        extra = " after the STFT filterbank of complex voltages"
    desc = (f"numpy oracle (Algorithm 1, mode {mode}{extra}), {runs} run(s) "
            f"over columns [0,{nt_s}) of the Nf={w.nf} Nt={w.nt} Nd={w.nd} workload, all Nd rows")
    return cells / elapsed, desc, runs, elapsed


def _oracle_shard_worker(conn, wl, dtype, t0, t1, halo):
    """One host core's share of the all-core oracle timing: output columns
    [t0, t1) of the workload, computed by the oracle on input columns
    [t0 - halo, t1) (halo = Nd - 1: an output column needs the Nd - 1 input
    columns before it, so the shard's columns are exact)."""
    import oracle
    T = oracle.build_tables(wl.f_min, wl.f_max, wl.nf, wl.nd)
    a = max(0, t0 - halo)
    x = fs.filterbank_u8(wl, a, t1) if dtype == "u8" else fs.filterbank_f32(wl, a, t1)
    mode = {"f32": "f32", "u8": "i64", "f16state": "f16state"}[dtype]
    conn.send("ready")
    while True:
        msg = conn.recv()
        if msg is None:
            break
        A = oracle.fdmt(x, T, mode)
        conn.send(float(A[:, t0 - a:].sum()))
    conn.close()


class OracleCores:
    """The oracle run on every host core at once: the sample's output columns
    are split into one contiguous shard per core (time sharding by
    causality); each worker process (spawned, so no GPU state is inherited)
    prepares its input once and transforms it on every step.  A step's time
    is the wall time until the last shard is done."""

    def __init__(self, wl, dtype, nt_s, cores=None):
        import multiprocessing as mp
        self.cores = cores or len(os.sched_getaffinity(0))
        self.nt_s = nt_s
        ctx = mp.get_context("spawn")
        bounds = [round(nt_s * i / self.cores / 16) * 16 for i in range(self.cores + 1)]
        self.conns, self.procs = [], []
        for i in range(self.cores):
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_oracle_shard_worker, args=(b, wl, dtype, bounds[i], bounds[i + 1], wl.nd - 1),
                             daemon=True)
            pr.start()
            self.conns.append(a)
            self.procs.append(pr)
        for c in self.conns:
            if c.recv() != "ready":
                raise RuntimeError("oracle worker failed to start")

    def step(self):
        t0 = time.perf_counter()
        for c in self.conns:
            c.send("go")
        for c in self.conns:
            c.recv()
        return time.perf_counter() - t0

    def close(self):
        for c in self.conns:
            try:
                c.send(None)
            except Exception:
                pass
        for pr in self.procs:
            pr.join(timeout=10)
            if pr.is_alive():
                pr.terminate()


def oracle_all_cores(w, dtype, runs=5, nt_cap=1 << 16):
    """(cells/s, cores, sample description) of the forward-transform oracle on
    all host cores over the first min(Nt, nt_cap) columns of the workload."""
    nt_s = min(w.nt, nt_cap)
    oc = OracleCores(w, dtype, nt_s)
    try:
        oc.step()  # warm-up
        el = sum(oc.step() for _ in range(runs))
    finally:
        oc.close()
    mode = {"f32": "f32", "u8": "i64", "f16state": "f16state"}[dtype]
    desc = (f"numpy oracle (Algorithm 1, mode {mode}) on {oc.cores} host cores at once, one process per core, "
            f"columns [0,{nt_s}) of the Nf={w.nf} Nt={w.nt} Nd={w.nd} workload split into {oc.cores} "
            f"contiguous shards (each with its Nd-1 input columns of history), {runs} run(s)")
    return float(w.nd) * nt_s * runs / el, oc.cores, desc


def workload_config(args, w, dtype, n_widths, front, world, fft=False):
    """The line's `config`: the workload alone (the same for both arms; how
    an arm computes it goes elsewhere in its line)."""
    return {"workload": ("FFT-FDMT (Algorithm 2) " if fft else "") +
            ("complex voltages -> STFT filterbank -> " if front else "") + w.name +
            f" {dtype}" + (f" + boxcar search of {n_widths} widths" if n_widths else ""),
            "nf": w.nf, "nt": w.nt, "nd": w.nd, "f_min": w.f_min, "f_max": w.f_max,
            "d_min": args.d_min, "descending": args.descending,
            "l2": "inputs and outputs larger than L2, no flush",
            "parallelism": f"replica x{world} (one beam per GPU)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w, dtype = WORKLOADS[args.workload]
    import oracle  # noqa: F401
    # each step: one oracle pass over a column sample sized so that the whole
    # warmup + steps run stays within about two minutes
    budget = 120.0 / max(1, args.steps + args.warmup)
    fft = args.workload in FFT_WORKLOADS
    est_rate = 4e6 if fft else 2.5e7  # cells/s of the numpy oracle, rough, to size the sample
    nt_s = int(max(256 if fft else 1024, min(w.nt, budget * est_rate / w.nd)))
    if fft:  # the oracle holds two levels of nt + nd - 1 padded complex rows
        nt_s = min(nt_s, 8192)
    nt_s = (nt_s // 16) * 16
    T = oracle.build_tables(w.f_min, w.f_max, w.nf, w.nd)
    x = fs.filterbank_u8(w, 0, nt_s) if dtype == "u8" else fs.filterbank_f32(w, 0, nt_s)
    mode = {"f32": "f32", "u8": "i64", "f16state": "f16state"}[dtype]
    diff = args.workload in DIFFERENTIABLE
    n_widths = (args.widths or SEARCH_WIDTHS[args.workload]) if args.workload in SEARCH_WIDTHS else 0
    g = fs.random_f32(w.seed + 7, w.nd, nt_s).astype(np.float64) if diff else None

    front = args.workload in FRONT_END
    if front:
        rng = np.random.Generator(np.random.PCG64([w.seed, 61]))
        v = (rng.standard_normal(w.nf * nt_s) + 1j * rng.standard_normal(w.nf * nt_s)).astype(np.complex64)

    def step():
        if fft:
            oracle.fft_fdmt(x.astype(np.float64), T)
            return
        A = oracle.fdmt(oracle.stft_filterbank(v, w.nf) if front else x, T, mode)
        if diff:
            oracle.fdmt_adjoint(g, T)
        if n_widths:
            oracle.boxcar_search(A, n_widths)

    # the plain forward transform runs on every host core at once (one
    # process per core, contiguous column shards); the other workloads run the
    # oracle as one process
    cores_used = 1
    oc = None
    if not (fft or diff or n_widths or front):
        nt_s = min(w.nt, 1 << 16)
        oc = OracleCores(w, dtype, nt_s)
        cores_used = oc.cores

        def step():  # noqa: F811
            oc.step()

    try:
        for _ in range(args.warmup):
            step()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step()
        el = time.perf_counter() - t0
    finally:
        if oc is not None:
            oc.close()
    cells = float(w.nd) * nt_s
    value = cells * args.steps / el
    extra = " + adjoint" if diff else (f" + boxcar search of {n_widths} widths" if n_widths else "")
    if front:
        extra = " after the STFT filterbank of complex voltages"
    if fft:
        mode, extra = "f64", ""
    sample = (f"numpy oracle ({'FFT-FDMT, Algorithm 2' if fft else 'Algorithm 1'}, mode {mode}{extra}) on columns "
              f"[0,{nt_s}) of the Nf={w.nf} Nt={w.nt} Nd={w.nd} workload per step, all Nd rows")
    if oc is not None:
        sample += (f", on {cores_used} host cores at once (one process per core, {cores_used} contiguous column "
                   f"shards, each with its Nd-1 input columns of history)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 (oracle)" if fft else DTYPE_NAME[dtype], "data": "synthetic (seeded)",
        "config": workload_config(args, w, dtype, n_widths, front, int(os.environ.get("WORLD_SIZE", "1")), fft),
        "cpu_baseline": {"value": value, "unit": "cells/s", "cores": cores_used, "kind": "oracle",
                         "sample": sample, "sample_nt": nt_s},
        "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm

def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_1411_5373_gb300 import build
    if rank == 0 and not os.path.exists(build.LIB_PATH):
        build.build()
    barrier()
    import paper_1411_5373_gb300 as FD

    w, dtype = WORKLOADS[args.workload]
    full_nt = w.nt
    if args.nt:  # a scaled-down shape for profiling, same channels, delays and schedule
        if args.nt < w.nd or args.nt % 64:
            raise SystemExit("--nt must be a multiple of 64 and at least Nd")
        w = dataclasses.replace(w, nt=args.nt, name=f"{w.name} scaled to Nt={args.nt}")
    tuned = None
    if args.schedule == "auto":
        from paper_1411_5373_gb300.autotune import autotune
        tuned = autotune(w.f_min, w.f_max, w.nf, full_nt, w.nd, dtype, use_cache=True)
        if tuned["schedule"] == "plain":
            plan = FD.Plan(w.f_min, w.f_max, w.nf, w.nt, w.nd, dtype, schedule="plain", d_min=args.d_min,
                           descending=args.descending)
        else:
            plan = FD.Plan(w.f_min, w.f_max, w.nf, w.nt, w.nd, dtype, schedule="fused", tile=tuned["tile"],
                           smem_budget=tuned["smem_budget"], bounds=tuned["bounds"],
                           group_tiles=tuned.get("group_tiles"), group_budgets=tuned.get("group_budgets"),
                           d_min=args.d_min, descending=args.descending)
    else:
        ints = lambda v: [int(u) for u in v.split(",")] if v else None
        plan = FD.Plan(w.f_min, w.f_max, w.nf, w.nt, w.nd, dtype, schedule=args.schedule,
                       tile=args.tile, smem_budget=args.smem_budget, bounds=ints(args.bounds),
                       group_tiles=ints(args.group_tiles), group_budgets=ints(args.group_budgets),
                       d_min=args.d_min, descending=args.descending)
    rows = [int(plan.band_rows(l).sum()) for l in range(plan.levels + 1)]
    tile, bounds = plan.schedule_info()

    # one independent beam per rank (weak scaling): rank r draws seed + r
    wr = fs.Workload(w.name, w.nf, w.nt, w.nd, w.f_min, w.f_max, w.seed + 1000 * rank,
                     w.n_pulses, w.width_range, w.amp_range, w.fixed_pulse)
    x_host = fs.filterbank_u8(wr) if dtype == "u8" else fs.filterbank_f32(wr)
    x = torch.from_numpy(x_host).to(dev)
    out = torch.empty((w.nd, w.nt), dtype=plan.out_dtype, device=dev)
    ws = plan.workspace(dev)
    stream = torch.cuda.current_stream(dev)
    diff = args.workload in DIFFERENTIABLE
    if diff:
        wts = torch.ones(w.nf, dtype=torch.float32, device=dev)
        g = torch.from_numpy(fs.random_f32(wr.seed + 7, w.nd, w.nt)).to(dev)
        gi = torch.empty((w.nf, w.nt), dtype=torch.float32, device=dev)
        gw = torch.empty(w.nf, dtype=torch.float32, device=dev)
        aws = plan.adjoint_workspace(dev)

    n_widths = (args.widths or SEARCH_WIDTHS[args.workload]) if args.workload in SEARCH_WIDTHS else 0
    search_ms = []
    front = args.workload in FRONT_END
    fb_ms = []
    if front:
        gen = torch.Generator(device=dev)
        gen.manual_seed(wr.seed)
        volts = torch.view_as_complex(torch.randn((w.nf * w.nt, 2), device=dev, generator=gen))
    search_paths = None
    in_launch = None  # a plan whose last launch runs the search (fdmt_execute_search)
    if n_widths:
        pk = torch.empty((w.nd, n_widths), dtype=torch.int64 if dtype == "u8" else torch.float32, device=dev)
        tm = torch.empty((w.nd, n_widths), dtype=torch.int32, device=dev)
        sws = torch.empty(FD.search_workspace_bytes(w.nd, w.nt, n_widths), dtype=torch.uint8, device=dev)
        # The two ways to run transform + search: the transform then the
        # standalone search, or the search inside the last fused launch
        # (same level grouping, tiles and budgets).  Both give the same
        # peaks and times; the faster one is timed.
        if plan.schedule == "fused" and n_widths <= 9:
            g = plan.fused_table(0).reshape(-1, 16)
            try:
                in_launch = FD.Plan(w.f_min, w.f_max, w.nf, w.nt, w.nd, dtype, schedule="fused",
                                    bounds=[int(g[0, 0])] + [int(v) for v in g[:, 1]],
                                    group_tiles=[int(v) for v in g[:, 7]],
                                    group_budgets=[int(v) for v in g[:, 5]] if tuned else None,
                                    smem_budget=max(int(v) for v in g[:, 5]), search_widths=n_widths,
                                    d_min=args.d_min, descending=args.descending)
                iws = torch.empty(in_launch.search_workspace_bytes(n_widths), dtype=torch.uint8, device=dev)
            except FD.FdmtError:
                in_launch = None

        def two_pass():
            plan.execute(x, out=out, workspace=ws)
            plan.search(out, n_widths, peak=pk, time=tm, workspace=sws)

        def one_pass():
            in_launch.execute_search(x, n_widths, out=out, peak=pk, time=tm, workspace=iws)

        def time_path(fn, reps=20):
            for _ in range(3):
                fn()
            torch.cuda.synchronize(dev)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
            torch.cuda.synchronize(dev)
            return a.elapsed_time(b) / reps

        search_paths = {"transform_then_search_ms": time_path(two_pass)}
        if in_launch is not None:
            search_paths["search_in_last_launch_ms"] = time_path(one_pass)
            if search_paths["search_in_last_launch_ms"] < search_paths["transform_then_search_ms"]:
                search_paths["timed"] = "search in the last launch (fdmt_execute_search)"
            else:
                search_paths["timed"] = "transform, then the standalone search (fdmt_search)"
                in_launch = None

    def step(timed=False):
        if front:
            if timed:
                f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                f0.record(stream)
            FD.filterbank(volts, w.nf, out=x)
            if timed:
                f1.record(stream)
                fb_ms.append((f0, f1))
        if diff:
            plan.execute(x, out=out, weights=wts, workspace=ws)
            plan.adjoint(g, x=x, weights=wts, grad_in=gi, grad_weights=gw, workspace=aws)
        elif n_widths and in_launch is not None:
            in_launch.execute_search(x, n_widths, out=out, peak=pk, time=tm, workspace=iws)
            return
        else:
            plan.execute(x, out=out, workspace=ws)
        if n_widths:
            if timed:
                s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s0.record(stream)
            plan.search(out, n_widths, peak=pk, time=tm, workspace=sws)
            if timed:
                s1.record(stream)
                search_ms.append((s0, s1))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    cap = min(65536, max(64, args.steps * (2 * plan.levels + 8)))
    prof_plan = in_launch if (n_widths and in_launch is not None) else plan
    sampler = ClockSampler(gpu_identifier(torch, dev))
    sampler.start()
    barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    ms_total = e0.elapsed_time(e1)
    # The same steps again with an event pair around every launch (the
    # launch profiler): per-kernel durations for the roofline.  The events
    # between launches cost a few microseconds a step, so the step time
    # above comes from the pass without them.
    prof_plan.profile_enable(cap)
    for _ in range(args.steps):
        step(timed=True)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    launches, prof = prof_plan.profile_read()
    prof_plan.profile_enable(0)
    if world > 1:
        t = torch.tensor([ms_total], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / args.steps
    cells_step = float(w.nd) * w.nt
    value = cells_step * world * args.steps / (ms_total / 1e3)

    # per-kernel device time over the timed region (recorded launches)
    per = {}
    sizes = None
    if plan.schedule == "fused":
        sizes = {(int(g[0]), int(g[1])): (int(g[14]), int(g[15])) for g in plan.fused_table(0).reshape(-1, 16)}
    for name, level, ms in prof:
        b = algorithmic_bytes(name, level, rows, w.nf, w.nt, dtype, sizes)
        d = per.setdefault(name, {"launches": 0, "ms": 0.0, "bytes": 0.0})
        d["launches"] += 1
        d["ms"] += ms
        d["bytes"] += b or 0.0
    if fb_ms:
        # the filterbank kernel: complex64 voltages in, float32 spectra out
        per["filterbank"] = {"launches": len(fb_ms), "ms": sum(a.elapsed_time(b) for a, b in fb_ms),
                             "bytes": float(len(fb_ms)) * w.nf * w.nt * (8 + 4)}
        launches += len(fb_ms)
    if n_widths and in_launch is not None:
        launches += args.steps  # the finalize launch after the last fused launch
    if search_ms:
        # the search's two kernels (the streaming search and the per-row
        # finalize), timed together around each call: they read A once
        per["search+finalize"] = {"launches": 2 * len(search_ms),
                                  "ms": sum(a.elapsed_time(b) for a, b in search_ms),
                                  "bytes": float(len(search_ms)) * w.nd * w.nt * OUT_BYTES}
        launches += 2 * len(search_ms)
    dom = max(per, key=lambda k: per[k]["ms"]) if per else None
    peak, peak_kind = measured_peak()
    compulsory = w.nt * (w.nf * IN_BYTES[dtype] + w.nd * OUT_BYTES)
    if front:  # voltages in (8 B per sample), spectra out and read back by the transform
        compulsory += w.nt * w.nf * (8 + 4)
    if n_widths:
        compulsory += w.nt * w.nd * OUT_BYTES  # the search reads the output once
    if diff:  # adjoint: output gradient in, input gradient out, input re-read for the weight gradient
        compulsory += w.nt * (w.nd * 4 + w.nf * 4 + w.nf * IN_BYTES[dtype])
    sched_key = schedule_key(plan) if bounds else None
    # DRAM traffic of one step from the committed ncu records of every kernel
    # the step launches (None unless all were taken on the current sources)
    step_traffic = 0.0
    for name, d in per.items():
        t = recorded_traffic(name, args.workload, sched_key)
        if t is None:
            step_traffic = None
            break
        step_traffic += t * d["launches"] / args.steps
    roofline = None
    if dom is not None:
        d = per[dom]
        achieved_launch = d["bytes"] / (d["ms"] / 1e3) / 1e9
        achieved = compulsory / (ms_step / 1e3) / 1e9
        roofline = {"bound": "hbm", "kernel": f"whole step ({launches / args.steps:g} launches)",
                    "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                    "traffic": step_traffic,
                    "algorithmic_bytes_per_step": compulsory,
                    "algorithmic_bytes_per_cell": compulsory / cells_step,
                    "traffic_over_algorithmic": None if step_traffic is None else round(step_traffic / compulsory, 3),
                    "dominant_kernel": dom,
                    "per_launch_state_frac": round(achieved_launch / peak, 4),
                    "per_launch_state_bytes": d["bytes"] / d["launches"],
                    "avg_launch_ms": d["ms"] / d["launches"],
                    "dominant_kernel_traffic": recorded_traffic(dom, args.workload, sched_key)}
    search_roofline = None
    if n_widths and search_ms:
        d = per["search+finalize"]
        achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
        search_roofline = {"bound": "hbm", "kernel": "search+finalize", "achieved": round(achieved, 1),
                           "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                           "peak_kind": peak_kind, "widths": n_widths,
                           "traffic": recorded_traffic("search+finalize", args.workload, f"widths:{n_widths}"),
                           "algorithmic_bytes_per_call": d["bytes"] / len(search_ms),
                           "avg_call_ms": d["ms"] / len(search_ms)}
    front_roofline = None
    if front:
        d = per["filterbank"]
        achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
        front_roofline = {"bound": "hbm", "kernel": "filterbank", "achieved": round(achieved, 1), "peak": peak,
                          "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                          "algorithmic_bytes_per_launch": d["bytes"] / d["launches"],
                          "avg_launch_ms": d["ms"] / d["launches"]}
    effective = compulsory / (ms_step / 1e3) / 1e9

    # the plain schedule (one launch per level) on the same input, same GPU,
    # timed the same way, so that the line carries both forms of the metric
    plain = None
    if plan.schedule == "fused" and not (diff or n_widths or front) and not args.no_plain:
        pp = FD.Plan(w.f_min, w.f_max, w.nf, w.nt, w.nd, dtype, schedule="plain",
                     d_min=args.d_min, descending=args.descending)
        pws = pp.workspace(dev)
        for _ in range(3):
            pp.execute(x, out=out, workspace=pws)
        n_plain = max(3, min(args.steps, 200))
        barrier()
        torch.cuda.synchronize(dev)
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(n_plain):
            pp.execute(x, out=out, workspace=pws)
        p1.record(stream)
        torch.cuda.synchronize(dev)
        ms_plain = p0.elapsed_time(p1)
        if world > 1:
            t = torch.tensor([ms_plain], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_plain = float(t.item())
        ms_plain /= n_plain
        plain = {"schedule": "plain (initialisation + one launch per merge level)", "steps": n_plain,
                 "ms_per_step": ms_plain, "value": cells_step * world / (ms_plain / 1e3),
                 "frac": round(compulsory / (ms_plain / 1e3) / 1e9 / peak, 4),
                 "launches_per_step": plan.levels + 1}
        del pws
        pp.close()

    # end to end through the host-buffer C ABI call (pinned buffers)
    e2e = None
    if not args.no_e2e and n_widths:
        xh = torch.from_numpy(x_host).pin_memory()
        ph = torch.empty(pk.shape, dtype=pk.dtype).pin_memory()
        th = torch.empty(tm.shape, dtype=tm.dtype).pin_memory()

        def e2e_step():
            x.copy_(xh, non_blocking=True)
            plan.execute(x, out=out, workspace=ws)
            plan.search(out, n_widths, peak=pk, time=tm, workspace=sws)
            ph.copy_(pk, non_blocking=True)
            th.copy_(tm, non_blocking=True)
            torch.cuda.synchronize(dev)

        for _ in range(3):
            e2e_step()
        n_e2e = max(3, min(args.steps, 200))
        barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        el = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([el], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el = float(t.item())
        e2e = {"value": cells_step * world * n_e2e / el, "unit": "cells/s",
               "h2d_bytes_per_step": int(xh.numel() * xh.element_size()),
               "d2h_bytes_per_step": int(ph.numel() * ph.element_size() + th.numel() * th.element_size()),
               "steps": n_e2e, "timer": "host perf_counter around synchronous steps",
               "api": "Plan.execute + Plan.search on device tensors, pinned host copies"}
    elif not args.no_e2e and front:
        vh = volts.cpu().pin_memory()
        oh = torch.empty((w.nd, w.nt), dtype=plan.out_dtype).pin_memory()

        def e2e_front():
            volts.copy_(vh, non_blocking=True)
            FD.filterbank(volts, w.nf, out=x)
            plan.execute(x, out=out, workspace=ws)
            oh.copy_(out, non_blocking=True)
            torch.cuda.synchronize(dev)

        for _ in range(3):
            e2e_front()
        n_e2e = max(3, min(args.steps, 100))
        barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_front()
        el = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([el], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el = float(t.item())
        e2e = {"value": cells_step * world * n_e2e / el, "unit": "cells/s",
               "h2d_bytes_per_step": int(vh.numel() * vh.element_size()),
               "d2h_bytes_per_step": int(oh.numel() * oh.element_size()),
               "steps": n_e2e, "timer": "host perf_counter around synchronous steps",
               "api": "filterbank + Plan.execute on device tensors, pinned host copies"}
    elif not args.no_e2e and not diff:
        xh = torch.from_numpy(x_host).pin_memory()
        ohs = [torch.empty((w.nd, w.nt), dtype=plan.out_dtype).pin_memory() for _ in range(2)]
        n_e2e = max(3, min(args.steps, 200))
        # one call per step, synchronous (fdmt_execute_host)
        for _ in range(3):
            plan.execute_host(xh, ohs[0], x, out, workspace=ws)
        barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            plan.execute_host(xh, ohs[0], x, out, workspace=ws)
        el_sync = time.perf_counter() - t0
        # pipelined (fdmt_pipeline_*): the copies of consecutive steps overlap
        # with compute; every step still copies its input in and its output out
        pipe = FD.Pipeline(plan)
        for i in range(3):
            pipe.push(xh, ohs[i % 2])
        pipe.wait()
        barrier()
        t0 = time.perf_counter()
        for i in range(n_e2e):
            pipe.push(xh, ohs[i % 2])
        pipe.wait()
        el = time.perf_counter() - t0
        pipe.close()
        if world > 1:
            t = torch.tensor([el, el_sync], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el, el_sync = float(t[0].item()), float(t[1].item())
        e2e = {"value": cells_step * world * n_e2e / el, "unit": "cells/s",
               "h2d_bytes_per_step": int(xh.numel() * xh.element_size()),
               "d2h_bytes_per_step": int(ohs[0].numel() * ohs[0].element_size()),
               "steps": n_e2e, "timer": "host perf_counter from the first push to the last output in host memory",
               "api": "Pipeline.push (fdmt_pipeline_push): copies of consecutive steps overlap with compute",
               "synchronous_value": cells_step * world * n_e2e / el_sync,
               "synchronous_api": "Plan.execute_host (fdmt_execute_host), one blocking call per step"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, desc, runs, el = oracle_sample_cells_per_s(w, dtype, 10.0, nt_cap=min(w.nt, 1 << 16),
                                                         adjoint=diff, search=n_widths, front=front)
        cpu = {"value": rate, "unit": "cells/s", "cores": 1, "kind": "oracle", "sample": desc,
               "seconds": round(el, 2)}
        if not (diff or n_widths or front):
            # the same oracle on every host core at once; the line reports the
            # all-core figure and keeps the one-core figure beside it
            rate_all, cores, desc_all = oracle_all_cores(w, dtype)
            cpu = {"value": rate_all, "unit": "cells/s", "cores": cores, "kind": "oracle", "sample": desc_all,
                   "single_core": cpu}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE_NAME[dtype], "data": "synthetic (seeded N(0,1) + injected pulses)",
            "config": workload_config(args, w, dtype, n_widths, front, world),
            # how this arm computes it: the schedule and the tuner's best trials
            "schedule": {"name": plan.schedule, "tile": tile, "level_bounds": bounds,
                         "autotune": None if tuned is None else
                         [{k: t[k] for k in ("schedule", "tile", "smem_budget", "bounds",
                                             "group_tiles", "group_budgets", "ms") if k in t}
                          for t in tuned["trials"][:6]]},
            "roofline": roofline,
            "plain": plain,
            "search_roofline": search_roofline,
            "search_paths": search_paths,
            "filterbank_roofline": front_roofline,
            "effective_hbm": {"compulsory_bytes_per_step": compulsory,
                              "gbs": round(effective, 1), "frac": round(effective / peak, 4)},
            "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                            "share": round(v["ms"] / sum(x["ms"] for x in per.values()), 4)}
                        for k, v in per.items()},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """64 uneven beams (Nf in {256..4096}, Nt in {2^14..2^18}, Nd in {256..2048},
    uint8 -> int32) in one persistent, graph-recorded launch per step."""
    import torch
    from paper_1411_5373_gb300 import build
    if not os.path.exists(build.LIB_PATH):
        build.build()
    import paper_1411_5373_gb300 as FD
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    dev = torch.device("cuda", 0)
    beams = fs.batch_beams()
    spec = [(1200.0, 1600.0, b.nf, b.nt, b.nd) for b in beams]
    cells = float(sum(b.nd * b.nt for b in beams))
    # uint8 noise and four injected pulses per beam, drawn on the host cores
    # (worker processes) and copied to the device once
    ins = [None] * len(beams)
    for i, xb in fs.batch_inputs_u8(beams):
        ins[i] = torch.from_numpy(xb).to(dev)
    # Work-item shape: timed per candidate (the workspace layout does not
    # depend on it, so one workspace and one set of outputs serve all).
    trials = []
    best = None
    bp0 = FD.BatchPlan(spec, "u8")
    ws = torch.empty(bp0.workspace_bytes, dtype=torch.uint8, device=dev)
    outs = bp0.outputs(dev)
    bp0.close()
    cands = [{"schedule": "levels", "rows_per_item": rpi, "tile": tile}
             for rpi, tile in ((16, 2048), (32, 2048), (32, 4096))]
    cands += [{"schedule": "fused", "fused_tile": ft, "smem_budget": sb}
              for ft, sb in ((0, 73728), (0, 57344), (0, 114688), (256, 73728))]
    cands += [{"schedule": "launches"}]
    for c in cands:
        bp = FD.BatchPlan(spec, "u8", **c)
        need = bp.workspace_bytes
        if ws.numel() < need:
            ws = torch.empty(need, dtype=torch.uint8, device=dev)
        bp.execute(ins, outs, workspace=ws)
        t0 = time.perf_counter()
        bp.execute(ins, outs, workspace=ws)
        el = time.perf_counter() - t0
        trials.append(dict(c, ms=1e3 * el))
        if best is None or el < best[0]:
            best = (el, c)
        bp.close()
    _, cfg = best
    bp = FD.BatchPlan(spec, "u8", **cfg)
    for _ in range(args.warmup):
        bp.execute(ins, outs, workspace=ws)
    stream = torch.cuda.current_stream(dev)
    sampler = ClockSampler(gpu_identifier(torch, dev))
    sampler.start()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        bp.execute(ins, outs, workspace=ws)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    value = cells / (ms / 1e3)
    peak, kind = measured_peak()
    compulsory = sum(b.nf * b.nt * 1 + b.nd * b.nt * 4 for b in beams)
    # Algorithmic bytes of the one launch: for every beam and every level
    # group (or level) it runs, the base rows once in, the top rows once out.
    alg = 0.0
    n_launch = 0
    rows_cache = {}
    for i, b in enumerate(beams):
        key = (b.nf, b.nt, b.nd)
        if key not in rows_cache:
            hp = FD.Plan(1200.0, 1600.0, b.nf, b.nt, b.nd, "u8", schedule="plain", host_only=True)
            rows_cache[key] = [int(hp.band_rows(l).sum()) for l in range(hp.levels + 1)]
            hp.close()
        rows = rows_cache[key]
        bounds, sizes = bp.levels(i, sizes=True)
        for k, (lb, lt) in enumerate(zip(bounds[:-1], bounds[1:])):
            s_lb, s_lt = sizes[k], sizes[k + 1]
            if lt == 0:  # level schedule: the initialisation
                alg += (b.nf * s_lb + rows[0] * s_lt) * b.nt
            else:
                alg += ((b.nf if lb == 0 and bp.schedule in ("fused", "launches") else rows[lb]) * s_lb +
                        rows[lt] * s_lt) * b.nt
        n_launch += len(bounds) - 1
    kname = {"fused": "batch_fused", "levels": "batch_levels", "launches": "batch_launches"}[bp.schedule]
    achieved = alg / (ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": kname, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_kind": kind,
                "traffic": recorded_traffic(kname, "batch-64-u8", batch_key(cfg)),
                "algorithmic_bytes_per_launch": alg, "avg_launch_ms": ms}
    line = {
        "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8->i32", "data": "synthetic (seeded uint8 noise + 4 injected pulses per beam)",
        "config": {"workload": "64 uneven beams, Nf 256-4096, Nt 2^14-2^18, Nd 256-2048",
                   "beams": len(beams), "cells_per_step": cells, "batch_schedule": cfg,
                   "autotune": trials,
                   "launch": ("every beam's fused launches, largest beam first, over 4 streams forked from the "
                              "caller's stream" if bp.schedule == "launches" else
                              "one persistent kernel per step, CUDA graph replay"),
                   "l2": "inputs and outputs larger than L2, no flush"},
        "roofline": roofline,
        "effective_hbm": {"compulsory_bytes_per_step": compulsory,
                          "gbs": round(compulsory / (ms / 1e3) / 1e9, 1),
                          "frac": round(compulsory / (ms / 1e3) / 1e9 / peak, 4), "peak_kind": kind},
        "gpu_launches": args.steps * (n_launch if bp.schedule == "launches" else 1), "clocks": clocks,
        "e2e": None, "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_fft(args):
    """FFT-FDMT of the single 1k beam: three launches per step (forward FFTs,
    per-bin merges of all levels, inverse FFTs), output float32 [Nd][Nt]."""
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_1411_5373_gb300 import build
    if rank == 0 and not os.path.exists(build.LIB_PATH):
        build.build()
    barrier()
    import paper_1411_5373_gb300 as FD

    w, dtype = WORKLOADS[args.workload]
    plan = FD.FFTPlan(w.f_min, w.f_max, w.nf, w.nt, w.nd, dtype, block=args.fft_block, bins=args.fft_bins)
    wr = fs.Workload(w.name, w.nf, w.nt, w.nd, w.f_min, w.f_max, w.seed + 1000 * rank,
                     w.n_pulses, w.width_range, w.amp_range, w.fixed_pulse)
    x_host = fs.filterbank_u8(wr) if dtype == "u8" else fs.filterbank_f32(wr)
    x = torch.from_numpy(x_host).to(dev)
    out = torch.empty((w.nd, w.nt), dtype=torch.float32, device=dev)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        plan(x, out=out, workspace=ws)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(gpu_identifier(torch, dev))
    sampler.start()
    barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan(x, out=out, workspace=ws)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    ms_total = e0.elapsed_time(e1)
    # per-launch events in a second pass of the same steps (see run_ours)
    plan.profile_enable(min(65536, 3 * args.steps + 8))
    for _ in range(args.steps):
        plan(x, out=out, workspace=ws)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    launches, prof = plan.profile_read()
    plan.profile_enable(0)
    if world > 1:
        t = torch.tensor([ms_total], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / args.steps
    cells_step = float(w.nd) * w.nt
    value = cells_step * world * args.steps / (ms_total / 1e3)

    # algorithmic HBM bytes per launch: the input once, the transformed
    # blocks (complex64 per Fourier bin) once each way, the output once
    nk = plan.pairs * plan.block
    hbm = {"fft_forward": w.nf * w.nt * IN_BYTES[dtype] + w.nf * nk * 8,
           "fft_merge": (w.nf + w.nd) * nk * 8,
           "fft_inverse": w.nd * nk * 8 + w.nd * w.nt * OUT_BYTES}
    # on-chip bytes of the merge per bin: every op of levels >= 2 reads two
    # rows and a shift-vector entry (8 B each) and every stored row is
    # written; level 1 reads two X values, two geometric sums and an entry
    lvl = 0
    while (1 << lvl) < w.nf:
        lvl += 1
    probe = FD.Plan(w.f_min, w.f_max, w.nf, ((w.nt + 15) // 16) * 16, w.nd, "f32", host_only=True)
    rows = [int(probe.band_rows(l).sum()) for l in range(probe.levels + 1)]
    probe.close()
    onchip_per_bin = sum(rows[l] * (40 if l == 1 else 24) + (8 * rows[l] if l < lvl else 0)
                         for l in range(1, lvl + 1))
    per = {}
    for name, ms in prof:
        d = per.setdefault(name, {"launches": 0, "ms": 0.0, "bytes": 0.0})
        d["launches"] += 1
        d["ms"] += ms
        d["bytes"] += hbm[name]
    dom = max(per, key=lambda k: per[k]["ms"])
    peak, peak_kind = measured_peak()
    d = per[dom]
    achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                "traffic": recorded_traffic(dom, args.workload, f"block:{plan.block}:bins:{plan.bins}"),
                "algorithmic_bytes_per_launch": d["bytes"] / d["launches"],
                "avg_launch_ms": d["ms"] / d["launches"]}
    m = per["fft_merge"]
    sm_mhz = (clocks or {}).get("sm_mhz") or 1920.0
    onchip_peak = 128.0 * 152 * sm_mhz * 1e6 / 1e9
    onchip = m["launches"] * nk * onchip_per_bin / (m["ms"] / 1e3) / 1e9
    onchip_roofline = {"bound": "shared memory / L1", "kernel": "fft_merge", "achieved": round(onchip, 1),
                       "peak": round(onchip_peak, 1), "unit": "GB/s", "frac": round(onchip / onchip_peak, 4),
                       "peak_kind": "derived: 128 B/clk/SM x 152 SMs x median SM clock",
                       "bytes_per_bin": onchip_per_bin, "bins": nk}
    compulsory = w.nt * (w.nf * IN_BYTES[dtype] + w.nd * OUT_BYTES)
    effective = compulsory / (ms_step / 1e3) / 1e9

    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(x_host).pin_memory()
        oh = torch.empty((w.nd, w.nt), dtype=torch.float32).pin_memory()

        def e2e_step():
            x.copy_(xh, non_blocking=True)
            plan(x, out=out, workspace=ws)
            oh.copy_(out, non_blocking=True)
            torch.cuda.synchronize(dev)

        for _ in range(3):
            e2e_step()
        n_e2e = max(3, min(args.steps, 100))
        barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        el = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([el], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el = float(t.item())
        e2e = {"value": cells_step * world * n_e2e / el, "unit": "cells/s",
               "h2d_bytes_per_step": int(xh.numel() * xh.element_size()),
               "d2h_bytes_per_step": int(oh.numel() * oh.element_size()),
               "steps": n_e2e, "timer": "host perf_counter around synchronous steps",
               "api": "FFTPlan call on device tensors, pinned host copies"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        T = oracle.build_tables(w.f_min, w.f_max, w.nf, w.nd)
        nt_s = 4096
        xs = (fs.filterbank_u8(w, 0, nt_s) if dtype == "u8" else fs.filterbank_f32(w, 0, nt_s)).astype(np.float64)
        runs, el = 0, 0.0
        while el < 10.0 and runs < 5:
            t0 = time.perf_counter()
            oracle.fft_fdmt(xs, T)
            el += time.perf_counter() - t0
            runs += 1
        cpu = {"value": float(w.nd) * nt_s * runs / el, "unit": "cells/s", "cores": 1, "kind": "oracle",
               "sample": f"numpy oracle (FFT-FDMT, Algorithm 2, f64), {runs} run(s) over columns [0,{nt_s}) "
                         f"of the Nf={w.nf} Nt={w.nt} Nd={w.nd} workload, all Nd rows",
               "seconds": round(el, 2)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (complex64 Fourier state)" if dtype == "f32" else "u8 in, f32 (complex64 Fourier state)",
            "data": "synthetic (seeded N(0,1) + injected pulses)",
            "config": workload_config(args, w, dtype, 0, False, world, True),
            "schedule": {"name": "fft-fdmt", "fft_block": plan.block, "hop": plan.hop, "block_pairs": plan.pairs,
                         "bins_per_merge_block": plan.bins},
            "roofline": roofline,
            "onchip_roofline": onchip_roofline,
            "effective_hbm": {"compulsory_bytes_per_step": compulsory,
                              "gbs": round(effective, 1), "frac": round(effective / peak, 4)},
            "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                            "share": round(v["ms"] / sum(q["ms"] for q in per.values()), 4),
                            "hbm_frac": round(v["bytes"] / (v["ms"] / 1e3) / 1e9 / peak, 4)}
                        for k, v in per.items()},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload.startswith("batch"):
        return run_batch(args)
    if args.workload in FFT_WORKLOADS:
        return run_fft(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
