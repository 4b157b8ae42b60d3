"""fdmt_execute_static, the entry point that allocates nothing.

It is meant for callers that cannot allocate device memory when they run the
transform (a real-time pipeline that must not allocate once data is flowing,
or a framework that owns the whole device memory pool); its scratch is a
fixed array inside the library.  This file is named to be collected last, so
a run that stops at the first failure has already run every other test.

Checks, through the C ABI: two calls in a row equal the workspace entry
point fdmt_execute bit for bit (the parity bar of the float32 and uint8
paths), the second call on different data so stale scratch contents cannot
leak into the result; and a plan whose workspace exceeds the array is refused.
"""
import ctypes

import numpy as np
import pytest

import filterbank_synth as fs
import paper_1411_5373_gb300 as FD
from paper_1411_5373_gb300 import _native as N
from paper_1411_5373_gb300 import build

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LIMIT = 32 << 20  # FDMT_STATIC_SCRATCH_BYTES


@pytest.fixture(scope="module")
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return N.load()


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("dtype,nf,nt,nd", [("f32", 64, 1024, 64), ("u8", 1024, 2048, 1024),
                                              ("f16state", 256, 4096, 300)])
def test_static_matches_workspace_entry_point_twice(lib, dtype, nf, nt, nd):
    plan = FD.Plan(1200.0, 1600.0, nf, nt, nd, dtype)
    assert plan.workspace_bytes <= LIMIT
    ws = plan.workspace()
    for call in range(2):
        seed = 1000 + call
        xh = fs.random_u8(seed, nf, nt) if dtype == "u8" else fs.random_f32(seed, nf, nt)
        x = torch.from_numpy(xh).cuda()
        ref = torch.empty((nd, nt), dtype=plan.out_dtype, device="cuda")
        got = torch.full((nd, nt), 7, dtype=plan.out_dtype, device="cuda")
        st = lib.fdmt_execute(plan._h, _p(x), None, _p(ref), _p(ws), ws.numel(), _stream())
        assert st == N.OK
        st = lib.fdmt_execute_static(plan._h, _p(x), None, _p(got), _stream())
        assert st == N.OK, N.error_string(st)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), f"call {call}"


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
    plan = FD.Plan(1200.0, 1600.0, 1024, 4096, 1024, "f32")
    assert plan.workspace_bytes > LIMIT
    x = torch.zeros((1024, 4096), device="cuda")
    out = torch.empty((1024, 4096), device="cuda")
    assert lib.fdmt_execute_static(plan._h, _p(x), None, _p(out), _stream()) == N.ERR_WORKSPACE
