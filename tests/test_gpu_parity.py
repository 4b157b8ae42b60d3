"""Parity of the CUDA path with the CPU oracle, through the C ABI.

Bars: uint8 -> int32 bit-exact; float32 bit-exact to the oracle's float32
mode (same association, no contraction) and within 1e-5 of each output
row's RMS against float64; fp16-stored state bit-exact to the oracle's
fp16-state mode and within 2e-3 (RMS over t) of the row RMS against float64.
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


def run_gpu(x_np, f_min, f_max, nd, dtype, weights=None, schedule="plain"):
    nf, nt = x_np.shape
    p = FD.Plan(f_min, f_max, nf, nt, nd, dtype, schedule=schedule)
    x = torch.from_numpy(np.ascontiguousarray(x_np)).cuda()
    w = None if weights is None else torch.from_numpy(weights).cuda()
    out = p.execute(x, weights=w)
    torch.cuda.synchronize()
    return out.cpu().numpy(), p


def row_rms(a):
    return np.sqrt(np.mean(np.asarray(a, dtype=np.float64) ** 2, axis=1))


def assert_rows_close(got, ref64, rel, metric="max"):
    diff = np.abs(got.astype(np.float64) - ref64)
    err = diff.max(axis=1) if metric == "max" else np.sqrt(np.mean(diff ** 2, axis=1))
    bound = rel * row_rms(ref64) + 1e-30
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, f"rows {bad[:8]} exceed {rel} x RMS ({metric}): {(err / bound)[bad[:8]]}"


# -- the small single-beam workload (Nf=64, Nt=1024, Nd=64, one pulse) ------

def test_small_f32_bitexact_and_within_tolerance():
    w = fs.SINGLE_SMALL
    x = fs.filterbank_f32(w)
    T = oracle.build_tables(w.f_min, w.f_max, w.nf, w.nd)
    got, _ = run_gpu(x, w.f_min, w.f_max, w.nd, "f32")
    assert np.array_equal(got, oracle.fdmt(x, T, "f32"))
    assert_rows_close(got, oracle.fdmt(x.astype(np.float64), T, "f64"), 1e-5)
    # the oracle itself agrees with brute force along the curves
    assert np.allclose(oracle.fdmt(x.astype(np.float64), T, "f64"),
                       oracle.bruteforce(x, T), rtol=1e-12, atol=1e-9)


def test_small_u8_bitexact():
    w = fs.SINGLE_SMALL
    x = fs.filterbank_u8(w)
    T = oracle.build_tables(w.f_min, w.f_max, w.nf, w.nd)
    got, _ = run_gpu(x, w.f_min, w.f_max, w.nd, "u8")
    assert got.dtype == np.int32
    assert np.array_equal(got, oracle.fdmt(x, T, "i64"))


# -- edge cases: ragged tails, tiny and degenerate shapes -------------------

EDGE = [
    # nf, nt, nd, dtype
    (2, 16, 1, "u8"), (2, 32, 32, "u8"), (2, 16, 16, "f32"), (4, 1040, 6, "u8"),
    (64, 1040, 64, "f32"), (64, 1040, 1, "f32"), (128, 2064, 300, "u8"),
    (256, 2048, 2048, "u8"), (1024, 4112, 100, "f32"), (4096, 1024, 256, "u8"),
    (8, 4096, 4096, "f32"), (16, 48, 40, "f16state"), (512, 3088, 700, "f16state"),
]


@pytest.mark.parametrize("nf,nt,nd,dtype", EDGE)
def test_edge_shapes(nf, nt, nd, dtype):
    f_min, f_max = 1200.0, 1600.0
    T = oracle.build_tables(f_min, f_max, nf, nd)
    seed = nf * 7919 + nt * 31 + nd
    if dtype == "u8":
        x = fs.random_u8(seed, nf, nt)
        got, _ = run_gpu(x, f_min, f_max, nd, dtype)
        assert np.array_equal(got, oracle.fdmt(x, T, "i64"))
    else:
        x = fs.random_f32(seed, nf, nt)
        got, _ = run_gpu(x, f_min, f_max, nd, dtype)
        mode = "f32" if dtype == "f32" else "f16state"
        assert np.array_equal(got, oracle.fdmt(x, T, mode))


def test_wide_band_large_sweep():
    """A band where single channels sweep many samples (level-0 rows > 3)."""
    nf, nt, nd = 256, 4096, 2048
    T = oracle.build_tables(1200.0, 1600.0, nf, nd)
    assert max(T.rows[0]) > 8
    x = fs.random_u8(5, nf, nt)
    got, _ = run_gpu(x, 1200.0, 1600.0, nd, "u8")
    assert np.array_equal(got, oracle.fdmt(x, T, "i64"))


def test_weights_bitexact():
    nf, nt, nd = 64, 2048, 80
    x = fs.random_f32(17, nf, nt)
    wts = np.random.default_rng(3).uniform(0.0, 2.0, nf).astype(np.float32)
    T = oracle.build_tables(1200.0, 1600.0, nf, nd)
    got, _ = run_gpu(x, 1200.0, 1600.0, nd, "f32", weights=wts)
    assert np.array_equal(got, oracle.fdmt(x, T, "f32", weights=wts))


def test_deterministic_repeat():
    x = fs.random_f32(23, 256, 8192)
    a, p = run_gpu(x, 1200.0, 1600.0, 512, "f32")
    xt = torch.from_numpy(x).cuda()
    b = p.execute(xt).cpu().numpy()
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


# -- the headline single-beam workload (Nf=1024, Nt=65536, Nd=1024) ---------

def test_1k_u8_full_bitexact():
    w = fs.SINGLE_1K
    x = fs.filterbank_u8(w)
    T = oracle.build_tables(w.f_min, w.f_max, w.nf, w.nd)
    got, _ = run_gpu(x, w.f_min, w.f_max, w.nd, "u8")
    assert np.array_equal(got, oracle.fdmt(x, T, "i64"))


def test_1k_f32_full_bitexact():
    w = fs.SINGLE_1K
    x = fs.filterbank_f32(w)
    T = oracle.build_tables(w.f_min, w.f_max, w.nf, w.nd)
    got, _ = run_gpu(x, w.f_min, w.f_max, w.nd, "f32")
    assert np.array_equal(got, oracle.fdmt(x, T, "f32"))
    assert_rows_close(got, oracle.fdmt(x.astype(np.float64), T, "f64"), 1e-5)


def _snr(row, t0, widths):
    best = -np.inf
    for wdt in widths:
        k = np.ones(wdt) / np.sqrt(wdt)
        f = np.convolve(row.astype(np.float64), k, mode="full")[: row.size]
        med = np.median(f)
        mad = 1.4826 * np.median(np.abs(f - med))
        lo, hi = max(0, t0 - 4), min(row.size, t0 + wdt + 8)
        best = max(best, (f[lo:hi].max() - med) / mad)
    return best


def test_1k_f16state_tolerance_and_snr():
    w = fs.SINGLE_1K
    x = fs.filterbank_f32(w)
    T = oracle.build_tables(w.f_min, w.f_max, w.nf, w.nd)
    got16, _ = run_gpu(x, w.f_min, w.f_max, w.nd, "f16state")
    assert np.array_equal(got16, oracle.fdmt(x, T, "f16state"))
    ref = oracle.fdmt(x.astype(np.float64), T, "f64")
    assert_rows_close(got16, ref, 2e-3, metric="rms")
    got32, _ = run_gpu(x, w.f_min, w.f_max, w.nd, "f32")
    for p in fs.draw_pulses(w):
        widths = [1, 2, 4, 8, 16, 32]
        s32 = _snr(got32[p.delay], p.t0, widths)
        s16 = _snr(got16[p.delay], p.t0, widths)
        assert abs(s16 / s32 - 1.0) <= 5e-3, (p.delay, s16, s32)


# -- adjoint and gradients -------------------------------------------------
# (fused plans run the fused adjoint here)
ADJ = {"plain": "plain", "fused": "fused"}

@pytest.mark.parametrize("schedule", ["plain", "fused"])
def test_adjoint_matches_oracle(schedule):
    nf, nt, nd = 128, 2064, 200
    T = oracle.build_tables(1200.0, 1600.0, nf, nd)
    p = FD.Plan(1200.0, 1600.0, nf, nt, nd, "f32", schedule=schedule, adjoint=ADJ[schedule])
    g = fs.random_f32(41, nd, nt)
    got = p.adjoint(torch.from_numpy(g).cuda()).cpu().numpy()
    ref = oracle.fdmt_adjoint(g.astype(np.float64), T)
    assert_rows_close(got, ref, 1e-5)


@pytest.mark.parametrize("schedule", ["plain", "fused"])
def test_adjoint_dot_product_exact_small_ints(schedule):
    nf, nt, nd = 256, 4096, 300
    p = FD.Plan(1200.0, 1600.0, nf, nt, nd, "f32", schedule=schedule, adjoint=ADJ[schedule])
    x = fs.small_ints(1, (nf, nt))
    y = fs.small_ints(2, (nd, nt))
    ax = p.execute(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    aty = p.adjoint(torch.from_numpy(y).cuda()).cpu().numpy().astype(np.float64)
    assert float(np.sum(ax * y)) == float(np.sum(x.astype(np.float64) * aty))


@pytest.mark.parametrize("schedule", ["plain", "fused"])
def test_weight_gradient_and_scaled_input_gradient(schedule):
    nf, nt, nd = 64, 1024, 64
    T = oracle.build_tables(1200.0, 1600.0, nf, nd)
    p = FD.Plan(1200.0, 1600.0, nf, nt, nd, "f32", schedule=schedule, adjoint=ADJ[schedule])
    x = fs.random_f32(51, nf, nt)
    g = fs.random_f32(52, nd, nt)
    wts = np.random.default_rng(9).uniform(0.5, 1.5, nf).astype(np.float32)
    gw = torch.empty(nf, device="cuda")
    gx = p.adjoint(torch.from_numpy(g).cuda(), x=torch.from_numpy(x).cuda(),
                   weights=torch.from_numpy(wts).cuda(), grad_weights=gw)
    gi = oracle.fdmt_adjoint(g.astype(np.float64), T)
    assert_rows_close(gx.cpu().numpy(), gi * wts[:, None], 1e-5)
    want = np.sum(x.astype(np.float64) * gi, axis=1)
    assert np.allclose(gw.cpu().numpy(), want, rtol=1e-4, atol=1e-3 * np.abs(want).max())


def _loss_np(A, sigma):
    z = A / sigma[:, None]
    m = z.max()
    return -(m + np.log(np.exp(z - m).sum()))


@pytest.mark.parametrize("schedule", ["plain", "fused"])
def test_autograd_finite_differences_fp64(schedule):
    """Gradient of loss(w) = -logsumexp_{d,t}(A[d,t] / sigma_d), sigma_d detached,
    from the CUDA adjoint vs central differences of the float64 oracle."""
    from paper_1411_5373_gb300 import fdmt
    w = fs.SINGLE_SMALL
    nf, nt, nd = w.nf, w.nt, w.nd
    x = fs.filterbank_f32(w)
    T = oracle.build_tables(w.f_min, w.f_max, nf, nd)
    sigma = np.std(oracle.fdmt(x.astype(np.float64), T, "f64"), axis=1)
    p = FD.Plan(w.f_min, w.f_max, nf, nt, nd, "f32", schedule=schedule, adjoint=ADJ[schedule])
    wt = torch.ones(nf, device="cuda", requires_grad=True)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    A = fdmt(xt, p, weights=wt)
    z = A / torch.from_numpy(sigma.astype(np.float32)).cuda()[:, None]
    loss = -torch.logsumexp(z.reshape(-1), dim=0)
    loss.backward()
    gw = wt.grad.cpu().numpy().astype(np.float64)
    eps = 1e-4
    for k in (0, 7, 31, 63):
        wp = np.ones(nf)
        wm = np.ones(nf)
        wp[k] += eps
        wm[k] -= eps
        lp = _loss_np(oracle.fdmt(x.astype(np.float64) * wp[:, None], T, "f64"), sigma)
        lm = _loss_np(oracle.fdmt(x.astype(np.float64) * wm[:, None], T, "f64"), sigma)
        fd = (lp - lm) / (2 * eps)
        assert abs(gw[k] - fd) <= 2e-3 * max(1.0, abs(fd)), (k, gw[k], fd)
    # input gradient: directional derivative along a random direction
    v = np.random.default_rng(5).standard_normal((nf, nt))
    lp = _loss_np(oracle.fdmt(x.astype(np.float64) + eps * v, T, "f64"), sigma)
    lm = _loss_np(oracle.fdmt(x.astype(np.float64) - eps * v, T, "f64"), sigma)
    fd = (lp - lm) / (2 * eps)
    got = float(np.sum(xt.grad.cpu().numpy().astype(np.float64) * v))
    assert abs(got - fd) <= 2e-3 * max(1.0, abs(fd)), (got, fd)


# -- host-buffer entry point and error paths --------------------------------

def test_execute_host_roundtrip():
    nf, nt, nd = 64, 4096, 64
    x = fs.random_f32(61, nf, nt)
    T = oracle.build_tables(1200.0, 1600.0, nf, nd)
    p = FD.Plan(1200.0, 1600.0, nf, nt, nd, "f32")
    xh = torch.from_numpy(x).pin_memory()
    oh = torch.empty((nd, nt), dtype=torch.float32).pin_memory()
    din = torch.empty((nf, nt), dtype=torch.float32, device="cuda")
    dout = torch.empty((nd, nt), dtype=torch.float32, device="cuda")
    p.execute_host(xh, oh, din, dout)
    assert np.array_equal(oh.numpy(), oracle.fdmt(x, T, "f32"))


def test_error_paths_on_device():
    import ctypes
    from paper_1411_5373_gb300 import _native as N
    p = FD.Plan(1200.0, 1600.0, 64, 1024, 64, "f32")
    x = torch.zeros((64, 1024), device="cuda")
    out = torch.empty((64, 1024), device="cuda")
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    lib = N.load()
    st = lib.fdmt_execute(p._h, ctypes.c_void_p(x.data_ptr()), None, ctypes.c_void_p(out.data_ptr()),
                          ctypes.c_void_p(small.data_ptr()), 256, None)
    assert st == N.ERR_WORKSPACE
    ws = p.workspace()
    st = lib.fdmt_execute(p._h, ctypes.c_void_p(x.data_ptr() + 4), None, ctypes.c_void_p(out.data_ptr()),
                          ctypes.c_void_p(ws.data_ptr()), ws.numel(), None)
    assert st == N.ERR_INVALID_ARG
    pu = FD.Plan(1200.0, 1600.0, 64, 1024, 64, "u8")
    wts = torch.ones(64, device="cuda")
    with pytest.raises(FD.FdmtError):
        pu.execute(torch.zeros((64, 1024), dtype=torch.uint8, device="cuda"), weights=wts)
