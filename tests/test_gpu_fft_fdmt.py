"""FFT-FDMT (``fdmt_fft_*``, section 5, Algorithm 2) against the oracle's
float64 ``fft_fdmt`` (pinned to the direct transform), through the C ABI.

Bar: the path computes in float32 complex arithmetic: a forward and an
inverse FFT of N points (about eps log2 N relative error each, RMS) and
ceil(log2 Nf) complex multiply-adds with rounded shift vectors per bin, so
each output row must match the float64 result within 1e-5 of the row's RMS
(about 30 eps for N = 4096, Nf = 1024: a margin of ~5 over the sum of those
terms).
"""
import numpy as np
import pytest

import filterbank_synth as fs
import oracle
import paper_1411_5373_gb300 as FD
from paper_1411_5373_gb300 import build

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    FD.load()


def check_rows(got, ref, tol=TOL):
    assert got.shape == ref.shape
    rms = np.sqrt(np.mean(ref ** 2, axis=1))
    err = np.sqrt(np.mean((got.astype(np.float64) - ref) ** 2, axis=1))
    worst = int(np.argmax(err / np.maximum(rms, 1e-300)))
    assert np.all(err <= tol * rms), f"row {worst}: rms err {err[worst]} vs rms {rms[worst]}"
    return float(np.max(err / np.maximum(rms, 1e-300)))


# (nf, nt, nd, block, bins, dtype): power-of-two and unequal splits, Nd
# above and below Nf, ragged tails (nt not a multiple of the hop), a single
# half-used block pair, every bins-per-CTA choice, both input types.
CASES = [
    (16, 100, 20, 0, 0, "f32"),
    (16, 1000, 20, 256, 1, "f32"),
    (6, 300, 40, 0, 0, "f32"),
    (2, 777, 8, 256, 0, "f32"),
    (3, 500, 50, 512, 2, "f32"),
    (64, 5000, 200, 1024, 0, "f32"),
    (64, 5000, 200, 1024, 8, "u8"),
    (37, 2048, 300, 2048, 4, "u8"),
    (128, 9000, 64, 0, 0, "f32"),
    (256, 4097, 511, 4096, 0, "f32"),
    (8, 1, 4, 0, 0, "f32"),
    (1000, 3000, 700, 0, 0, "u8"),
    (4, 600, 1, 256, 0, "f32"),  # Nd = 1: the channel sum, blocks without overlap
]


@pytest.mark.parametrize("nf,nt,nd,block,bins,dtype", CASES)
def test_fft_fdmt_matches_oracle(nf, nt, nd, block, bins, dtype):
    f_min, f_max = 1200.0, 1600.0
    x = fs.random_u8(nf + nd, nf, nt) if dtype == "u8" else fs.random_f32(nf + nd, nf, nt)
    p = FD.FFTPlan(f_min, f_max, nf, nt, nd, dtype, block=block, bins=bins)
    nblk = -(-nt // p.hop)
    assert p.hop == p.block - (nd - 1) and p.pairs == -(-nblk // 2)
    if bins:
        assert p.bins == bins
    got = p(torch.from_numpy(x).cuda()).cpu().numpy()
    T = oracle.build_tables(f_min, f_max, nf, nd)
    ref = oracle.fft_fdmt(x.astype(np.float64), T)
    check_rows(got, ref)


def test_fft_fdmt_impulse_lands_on_curves():
    """A unit impulse in channel k at time t0 reaches row d exactly where the
    curve of d covers it (the direct transform's impulse response); the
    float32 path must put ~1 there per covering offset and ~0 elsewhere."""
    nf, nt, nd = 32, 600, 48
    T = oracle.build_tables(1200.0, 1600.0, nf, nd)
    x = np.zeros((nf, nt), dtype=np.float32)
    x[5, 250] = 1.0
    got = FD.FFTPlan(1200.0, 1600.0, nf, nt, nd, block=256)(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.fdmt(x.astype(np.float64), T)
    assert np.max(np.abs(got - ref)) <= 1e-5


def _window_ref(w, t0, span, gen):
    """The oracle's output columns [t0, t0 + span), from the input window
    [t0 - Nd + 1, t0 + span) alone (causality: nothing earlier reaches them)."""
    T = oracle.build_tables(w.f_min, w.f_max, w.nf, w.nd)
    a = max(0, t0 - (w.nd - 1))
    xs = gen(w, a, t0 + span).astype(np.float64)
    return oracle.fdmt(xs, T)[:, t0 - a:]


@pytest.fixture(scope="module")
def full_size():
    w = fs.SINGLE_1K
    res = {}
    for dtype, gen in (("f32", fs.filterbank_f32), ("u8", fs.filterbank_u8)):
        x = torch.from_numpy(gen(w)).cuda()
        p = FD.FFTPlan(w.f_min, w.f_max, w.nf, w.nt, w.nd, dtype)
        res[dtype] = (p(x).cpu().numpy(), p, gen)
        del x
    return res


@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_fft_fdmt_full_size_windows(full_size, dtype):
    """Nf = Nd = 1024, Nt = 65536 in the launch configuration the benchmark
    times (block 4096, hop 3073): sampled column windows at the start, across
    block and pair boundaries, and at the ragged end."""
    w = fs.SINGLE_1K
    out, p, gen = full_size[dtype]
    assert (p.block, p.hop) == (4096, 3073)
    span = 96
    for t0 in (0, p.hop - 40, 2 * p.hop - 50, 7 * p.hop + 1000, w.nt - span):
        ref = _window_ref(w, t0, span, gen)
        check_rows(out[:, t0:t0 + span], ref, tol=2 * TOL)


def test_fft_fdmt_full_size_equals_direct(full_size):
    """The whole output against the direct float32 transform (the other
    path): the same sums, so within the FFT rounding everywhere."""
    w = fs.SINGLE_1K
    out, _, gen = full_size["f32"]
    x = torch.from_numpy(gen(w)).cuda()
    direct = FD.Plan(w.f_min, w.f_max, w.nf, w.nt, w.nd, "f32").execute(x).cpu().numpy().astype(np.float64)
    rms = np.sqrt(np.mean(direct ** 2, axis=1))
    err = np.sqrt(np.mean((out - direct) ** 2, axis=1))
    assert np.all(err <= TOL * rms)


def test_fft_fdmt_argument_errors():
    x = torch.zeros((16, 100), dtype=torch.float32, device="cuda")
    p = FD.FFTPlan(1200.0, 1600.0, 16, 100, 20)
    with pytest.raises(ValueError):
        p(x.to(torch.uint8))
    with pytest.raises(ValueError):
        p(torch.zeros((16, 99), dtype=torch.float32, device="cuda"))
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(FD.FdmtError):
        p(x, workspace=small)
    h = FD.FFTPlan(1200.0, 1600.0, 16, 100, 20, host_only=True)
    with pytest.raises(FD.FdmtError):
        h(x)
