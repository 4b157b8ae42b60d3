"""The bench line's host-side pieces (no GPU): the workload config both
arms print, and the reference arm's line with the contract's keys."""
import argparse
import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_workload_config_names_the_workload_alone():
    b = _bench()
    args = argparse.Namespace(d_min=0, descending=False)
    w, dtype = b.WORKLOADS["single-1k-f32"]
    cfg = b.workload_config(args, w, dtype, 0, False, 1)
    assert cfg["nf"] == 1024 and cfg["nt"] == 65536 and cfg["nd"] == 1024
    assert (cfg["f_min"], cfg["f_max"]) == (1200.0, 1600.0) and "no flush" in cfg["l2"]
    # nothing about how an arm computes it
    assert not {"schedule", "tile", "level_bounds", "autotune", "sample_nt"} & set(cfg)


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "small-64-f32", "--steps", "1", "--warmup", "1"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "cells/s"
    assert line["higher_is_better"] is True and line["steps"] == 1 and line["warmup"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "cells/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    b = _bench()
    w, dtype = b.WORKLOADS["small-64-f32"]
    assert line["config"] == b.workload_config(argparse.Namespace(d_min=0, descending=False), w, dtype, 0,
                                               False, 1)
