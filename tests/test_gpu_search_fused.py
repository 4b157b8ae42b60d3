"""The boxcar search (section 4.2, pulse profile) run inside the last fused
launch (``fdmt_execute_search`` on a plan made with search_widths = K),
through the C ABI.

Bars, against the oracle (its transform, then ``boxcar_search``): the
transform bit-exact, peaks bit-exact (int64 for uint8 input, float32
bit-for-bit otherwise) and the first times of the peaks equal, for
K = 1 .. 9 in the last launch and K = 10 .. 13 through the standalone search
the entry point falls back to; also at the headline size, Nf = Nd = 1024,
Nt = 65536.
"""
import numpy as np
import pytest

import filterbank_synth as fs
import oracle
import paper_1411_5373_gb300 as FD
from paper_1411_5373_gb300 import build

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    FD.load()


def _oracle(x, nf, nd, dtype, k, f_min=1200.0, f_max=1600.0):
    T = oracle.build_tables(f_min, f_max, nf, nd)
    mode = {"u8": "i64", "f32": "f32", "f16state": "f16state"}[dtype]
    A = oracle.fdmt(x, T, mode)
    A = A.astype(np.int32) if dtype == "u8" else A
    return A, oracle.boxcar_search(A, k)


def _check(got, want):
    A, peak, time = (v.cpu().numpy() for v in got)
    wA, (wp, wt) = want
    assert np.array_equal(A, wA), np.argwhere(A != wA)[:4]
    assert peak.dtype == wp.dtype
    if wp.dtype == np.float32:
        bad = np.argwhere(peak.view(np.int32) != wp.view(np.int32))
    else:
        bad = np.argwhere(peak != wp)
    assert bad.size == 0, f"peaks differ at {bad[:4].tolist()}"
    bad = np.argwhere(time != wt)
    assert bad.size == 0, f"times differ at {bad[:4].tolist()}"


CASES = [  # nf, nt, nd, dtype, K, schedule parameters
    (16, 512, 16, "f32", 1, {}),
    (16, 512, 16, "u8", 2, {"tile": 128}),
    (64, 4096, 64, "f32", 5, {}),
    (64, 4096, 64, "u8", 6, {"tile": 256}),
    (256, 8192, 300, "f32", 8, {"bounds": [0, 3, 5, 8]}),
    (256, 8208, 300, "u8", 8, {"tile": 448}),
    (128, 6000, 200, "f16state", 7, {"tile": 512}),
    (512, 16384, 512, "f32", 9, {"tile": 448, "bounds": [0, 3, 6, 9], "smem_budget": 150 * 1024}),
    (512, 16384, 700, "u8", 9, {"tile": 448, "smem_budget": 114688}),
    (1024, 4096, 1024, "f32", 8, {"bounds": [0, 3, 7, 10], "tile": 448}),
]


@pytest.mark.parametrize("nf,nt,nd,dtype,k,sched", CASES)
def test_search_in_last_launch_matches_oracle(nf, nt, nd, dtype, k, sched):
    x = fs.random_u8(7 + k, nf, nt) if dtype == "u8" else fs.random_f32(7 + k, nf, nt)
    p = FD.Plan(1200.0, 1600.0, nf, nt, nd, dtype, schedule="fused", search_widths=k, **sched)
    want = _oracle(x, nf, nd, dtype, k)
    xd = torch.from_numpy(x).cuda()
    for _ in range(2):  # a second call reuses the workspace's partials
        got = p.execute_search(xd, k)
        torch.cuda.synchronize()
        p.device_status()
        _check(got, want)
    # fdmt_execute on the same plan still gives the transform
    out = p.execute(xd)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), want[0])


@pytest.mark.parametrize("k", [10, 13])
@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_widths_beyond_the_last_launch_use_the_standalone_search(k, dtype):
    nf, nt, nd = 64, 8192, 64
    x = fs.random_u8(3, nf, nt) if dtype == "u8" else fs.random_f32(3, nf, nt)
    p = FD.Plan(1200.0, 1600.0, nf, nt, nd, dtype, schedule="fused", search_widths=8)
    got = p.execute_search(torch.from_numpy(x).cuda(), k)
    torch.cuda.synchronize()
    _check(got, _oracle(x, nf, nd, dtype, k))


def test_plain_plan_runs_transform_then_search():
    nf, nt, nd = 64, 2048, 100
    x = fs.random_f32(5, nf, nt)
    p = FD.Plan(1200.0, 1600.0, nf, nt, nd, "f32")
    got = p.execute_search(torch.from_numpy(x).cuda(), 6)
    torch.cuda.synchronize()
    _check(got, _oracle(x, nf, nd, "f32", 6))


@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_full_size_headline_shape(dtype):
    """Nf = Nd = 1024, Nt = 65536 (the benchmark's shape) with injected
    pulses, widths 1 .. 128 searched in the last launch."""
    w = fs.SINGLE_1K
    x = fs.filterbank_u8(w) if dtype == "u8" else fs.filterbank_f32(w)
    p = FD.Plan(w.f_min, w.f_max, w.nf, w.nt, w.nd, dtype, schedule="fused", search_widths=8,
                bounds=[0, 3, 7, 10], tile=448)
    got = p.execute_search(torch.from_numpy(x).cuda(), 8)
    torch.cuda.synchronize()
    p.device_status()
    _check(got, _oracle(x, w.nf, w.nd, dtype, 8, w.f_min, w.f_max))


def test_search_widths_argument_errors():
    with pytest.raises(FD.FdmtError):
        FD.Plan(1200.0, 1600.0, 64, 1024, 64, "f32", schedule="fused", search_widths=10)
    with pytest.raises(FD.FdmtError):
        FD.Plan(1200.0, 1600.0, 2, 1024, 4, "f32", schedule="fused", search_widths=3)  # one merge level
    p = FD.Plan(1200.0, 1600.0, 64, 1024, 64, "f32", schedule="fused", search_widths=4)
    x = torch.zeros((64, 1024), device="cuda")
    with pytest.raises(FD.FdmtError):
        p.execute_search(x, 0)
    with pytest.raises(FD.FdmtError):
        p.execute_search(x, 4, workspace=torch.empty(16, dtype=torch.uint8, device="cuda"))
