"""Parity of the CUDA boxcar search (``fdmt_search``, section 4.2 "Pulse
profile") with the oracle's ``boxcar_search``, through the C ABI.

Bars: integer outputs (int64 peaks) bit-exact; float32 outputs bit-exact
(the kernel keeps the oracle's binary-tree order of additions); peak times
equal everywhere (the first maximum).  Inputs are seeded and synthetic; the
oracle's inputs never come from the CUDA path.
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


def gpu_search(A_np, k, offset=0, bound=0):
    """Search on the device; offset > 0 places A that many elements past a
    16-byte boundary (the unaligned path); bound = value_bound (int32 A)."""
    nd, nt = A_np.shape
    dt = torch.int32 if A_np.dtype == np.int32 else torch.float32
    buf = torch.empty(nd * nt + offset, dtype=dt, device="cuda")
    A = buf[offset:].view(nd, nt)
    A.copy_(torch.from_numpy(np.ascontiguousarray(A_np)))
    peak, time = FD.search(A, k, value_bound=bound)
    torch.cuda.synchronize()
    return peak.cpu().numpy(), time.cpu().numpy()


def assert_same(got, ref):
    gp, gt = got
    rp, rt = ref
    assert gp.dtype == rp.dtype, (gp.dtype, rp.dtype)
    if rp.dtype == np.float32:  # bit-exact, signed zeros included
        bad = np.argwhere(gp.view(np.int32) != rp.view(np.int32))
    else:
        bad = np.argwhere(gp != rp)
    assert bad.size == 0, f"peaks differ at {bad[:6].tolist()}: {gp[tuple(bad[0])]} vs {rp[tuple(bad[0])]}"
    bad = np.argwhere(gt != rt)
    assert bad.size == 0, f"times differ at {bad[:6].tolist()}: {gt[tuple(bad[0])]} vs {rt[tuple(bad[0])]}"


def rand_f32(seed, nd, nt):
    return fs.random_f32(seed, nd, nt)


def rand_i32(seed, nd, nt, lo=-(1 << 30), hi=1 << 30):
    rng = np.random.Generator(np.random.PCG64([seed, nd, nt, 17]))
    return rng.integers(lo, hi, size=(nd, nt), dtype=np.int64).astype(np.int32)


# Shapes: one segment, a ragged tail, several segments, nt below the halo,
# nt not a multiple of 4 (scalar loads).
SHAPES = [(3, 1), (5, 7), (4, 4096), (2, 4097), (3, 12289), (2, 9000), (6, 130)]


@pytest.mark.parametrize("nd,nt", SHAPES)
@pytest.mark.parametrize("k", [1, 4, 5, 6, 9, 10, 13])
def test_float_random(nd, nt, k):
    A = rand_f32(1000 + k, nd, nt)
    assert_same(gpu_search(A, k), oracle.boxcar_search(A, k))


@pytest.mark.parametrize("nd,nt", SHAPES)
@pytest.mark.parametrize("k", [1, 5, 8, 13])
def test_int_random_wide_values(nd, nt, k):
    # |A| up to 2^30: window sums leave int32 from width 4 on
    A = rand_i32(2000 + k, nd, nt)
    assert_same(gpu_search(A, k), oracle.boxcar_search(A, k))


@pytest.mark.parametrize("nd,nt", SHAPES)
@pytest.mark.parametrize("k", [1, 2, 6, 10, 13])
def test_int_bounded_int32_sums(nd, nt, k):
    # value_bound 1000 keeps every window sum inside int32 up to width 4096;
    # a bound of 2^30 does so for widths 1 and 2 only (int64 above)
    A = rand_i32(3000 + k, nd, nt, -1000, 1001)
    assert_same(gpu_search(A, k, bound=1000), oracle.boxcar_search(A, k))
    B = rand_i32(3100 + k, nd, nt)
    assert_same(gpu_search(B, k, bound=1 << 30), oracle.boxcar_search(B, k))


@pytest.mark.parametrize("dtype", [np.float32, np.int32])
def test_unaligned_pointer(dtype):
    A = rand_f32(7, 4, 8192 + 12) if dtype == np.float32 else rand_i32(7, 4, 8192 + 12)
    assert_same(gpu_search(A, 11, offset=1), oracle.boxcar_search(A, 11))


def test_ties_and_degenerate_rows():
    nt = 9000
    A = np.zeros((6, nt), dtype=np.float32)
    A[1] = -1.0                                   # all negative: the max is at t = 0
    A[2, 100] = A[2, 5000] = A[2, 8999] = 7.0     # equal maxima in three segments
    A[3] = -0.0                                   # signed zeros keep their sign
    A[4, ::4096] = 3.0                            # maxima at segment starts
    A[5, 4095] = A[5, 4096] = 2.0                 # a window across a segment border
    for k in (1, 2, 6, 13):
        assert_same(gpu_search(A, k), oracle.boxcar_search(A, k))
    Ai = (A * 3).astype(np.int32)
    for k in (1, 3, 13):
        assert_same(gpu_search(Ai, k), oracle.boxcar_search(Ai, k))
        assert_same(gpu_search(Ai, k, bound=21), oracle.boxcar_search(Ai, k))


def test_transform_then_search_small():
    """Section 4.2 end to end on the small workload (Nf=64, Nt=1024, Nd=64):
    the GPU transform's output searched on the GPU equals the oracle's
    search of the oracle's transform (uint8 -> int32 and float32)."""
    w = fs.SINGLE_SMALL
    T = oracle.build_tables(w.f_min, w.f_max, w.nf, w.nd)
    for dtype, x, mode in (("u8", fs.filterbank_u8(w), "i64"), ("f32", fs.filterbank_f32(w), "f32")):
        for schedule in ("plain", "fused"):
            p = FD.Plan(w.f_min, w.f_max, w.nf, w.nt, w.nd, dtype, schedule=schedule)
            out = p.execute(torch.from_numpy(x).cuda())
            peak, time = p.search(out, 8)
            torch.cuda.synchronize()
            ref = oracle.fdmt(x, T, mode)
            ref = ref.astype(np.int32) if mode == "i64" else ref
            assert_same((peak.cpu().numpy(), time.cpu().numpy()), oracle.boxcar_search(ref, 8))
    # the planted pulse (D = 40, arrival 500, width 2) is the strongest event
    # of its row at width 2
    assert abs(int(time[40, 1].item()) - 501) <= 2


def test_full_size_float():
    """Nd = 1024 rows of Nt = 65536 float32 samples (the headline output's
    shape), widths 1 .. 256, compared in full."""
    A = rand_f32(fs.SEED_BASE + 40, 1024, 1 << 16)
    assert_same(gpu_search(A, 9), oracle.boxcar_search(A, 9))


def test_full_size_int():
    """The same shape as int32 transform sums of uint8 input (values up to
    255 * 2047, the bound of that plan), widths 1 .. 4096, with int32 sums
    (the bound) and int64 sums (no bound)."""
    A = rand_i32(fs.SEED_BASE + 41, 1024, 1 << 16, 0, 255 * 2047 + 1)
    ref = oracle.boxcar_search(A, 13)
    assert_same(gpu_search(A, 13, bound=255 * 2047), ref)
    assert_same(gpu_search(A, 13), ref)


def test_argument_errors():
    A = torch.zeros((4, 64), dtype=torch.float32, device="cuda")
    for k in (0, 14):
        with pytest.raises(FD.FdmtError):
            FD.search(A, k)
    ws = torch.empty(8, dtype=torch.uint8, device="cuda")
    with pytest.raises(FD.FdmtError) as e:
        FD.search(A, 3, workspace=ws)
    assert e.value.status == FD._native.ERR_WORKSPACE
