"""fdmt_execute_static, the entry point that allocates nothing.

It is meant for callers that cannot allocate device memory when they run the
transform (a real-time pipeline that must not allocate once data is flowing,
or a framework that owns the whole device memory pool); its scratch is a
fixed array inside the library.  This file is named to be collected last, so
a run that stops at the first failure has already run every other test.

Checks, through the C ABI: two calls in a row equal the workspace entry
point fdmt_execute bit for bit (the parity bar of the float32 and uint8
paths), the second call on different data so stale scratch contents cannot
leak into the result; plans made with the fused schedule (which this entry
point runs on the plain schedule); two plans on one device, interleaved with
fdmt_execute; and a plan whose plain-schedule scratch exceeds the array is
refused.  The array's size is read from the header, and the sizes the cases
need are those of the plain schedule.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import filterbank_synth as fs
import paper_1411_5373_gb300 as FD
from paper_1411_5373_gb300 import _native as N
from paper_1411_5373_gb300 import build

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_limit():
    src = open(os.path.join(ROOT, "include", "fdmt.h")).read()
    m = re.search(r"#define\s+FDMT_STATIC_SCRATCH_BYTES\s+\((\d+)u\s*<<\s*(\d+)\)", src)
    assert m, "FDMT_STATIC_SCRATCH_BYTES not found in include/fdmt.h"
    return int(m.group(1)) << int(m.group(2))


LIMIT = _header_limit()


def _plain_scratch(nf, nt, nd, dtype):
    """Scratch the static entry point needs: the plain schedule's workspace."""
    return FD.Plan(1200.0, 1600.0, nf, nt, nd, dtype, schedule="plain", host_only=True).workspace_bytes


@pytest.fixture(scope="module")
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return N.load()


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _input(dtype, seed, nf, nt):
    xh = fs.random_u8(seed, nf, nt) if dtype == "u8" else fs.random_f32(seed, nf, nt)
    return torch.from_numpy(xh).cuda()


def _both(lib, plan, x):
    """(fdmt_execute, fdmt_execute_static) outputs of one input."""
    ws = plan.workspace()
    ref = torch.empty((plan.nd, plan.nt), dtype=plan.out_dtype, device="cuda")
    got = torch.full((plan.nd, plan.nt), 7, dtype=plan.out_dtype, device="cuda")
    st = lib.fdmt_execute(plan._h, _p(x), None, _p(ref), _p(ws), ws.numel(), _stream())
    assert st == N.OK, N.error_string(st)
    st = lib.fdmt_execute_static(plan._h, _p(x), None, _p(got), _stream())
    assert st == N.OK, N.error_string(st)
    return ref, got


@pytest.mark.parametrize("dtype,nf,nt,nd,schedule", [
    ("f32", 64, 1024, 64, "plain"), ("u8", 1024, 2048, 1024, "plain"), ("f16state", 256, 4096, 300, "plain"),
    ("f32", 128, 2048, 128, "fused"), ("u8", 256, 4096, 256, "fused")])
def test_static_matches_workspace_entry_point_twice(lib, dtype, nf, nt, nd, schedule):
    assert _plain_scratch(nf, nt, nd, dtype) <= LIMIT
    plan = FD.Plan(1200.0, 1600.0, nf, nt, nd, dtype, schedule=schedule)
    for call in range(2):
        ref, got = _both(lib, plan, _input(dtype, 1000 + call, nf, nt))
        torch.cuda.synchronize()
        assert torch.equal(got, ref), f"call {call}"


def test_static_two_plans_interleaved(lib):
    shapes = [("f32", 64, 1024, 64, "plain"), ("u8", 512, 2048, 700, "fused")]
    plans = [FD.Plan(1200.0, 1600.0, nf, nt, nd, dt, schedule=sc) for dt, nf, nt, nd, sc in shapes]
    for dt, nf, nt, nd, _ in shapes:
        assert _plain_scratch(nf, nt, nd, dt) <= LIMIT
    results = []
    for rnd in range(2):
        for i, (plan, (dt, nf, nt, nd, _)) in enumerate(zip(plans, shapes)):
            results.append(_both(lib, plan, _input(dt, 2000 + 10 * rnd + i, nf, nt)))
    torch.cuda.synchronize()
    for k, (ref, got) in enumerate(results):
        assert torch.equal(got, ref), f"call {k}"


def test_static_with_weights(lib):
    nf, nt, nd = 64, 2048, 64
    plan = FD.Plan(1200.0, 1600.0, nf, nt, nd, "f32")
    x = torch.from_numpy(fs.random_f32(5, nf, nt)).cuda()
    w = torch.from_numpy(np.linspace(0.5, 1.5, nf, dtype=np.float32)).cuda()
    ref = plan.execute(x, weights=w)
    got = torch.empty_like(ref)
    assert lib.fdmt_execute_static(plan._h, _p(x), _p(w), _p(got), _stream()) == N.OK
    torch.cuda.synchronize()
    assert torch.equal(got, ref)


def test_static_refuses_oversized_plan(lib):
    nf = nd = 1024
    nt = 1024
    while _plain_scratch(nf, nt, nd, "f32") <= LIMIT:
        nt *= 2
    for schedule in ("plain", "fused"):
        plan = FD.Plan(1200.0, 1600.0, nf, nt, nd, "f32", schedule=schedule)
        x = torch.zeros((nf, nt), device="cuda")
        out = torch.empty((nd, nt), device="cuda")
        assert lib.fdmt_execute_static(plan._h, _p(x), None, _p(out), _stream()) == N.ERR_WORKSPACE
