"""Full-size workloads: the large beam (Nf=4096 over 1100-1700 MHz, Nt=2^20,
Nd=4096) with float32 and fp16-stored state, and the adjoint identity at
the differentiable workload's full size (Nf=Nd=1024, Nt=65536).

The large beam is checked on a slice: A[:, t] depends only on input columns
t - (Nd - 1) .. t (section 4: every curve spans at most Nd - 1 samples), so
output columns [T0, T0 + S) of the full transform equal the oracle run on
input columns [T0 - Nd + 1, T0 + S), from its column Nd - 1 on.
"""
import numpy as np
import pytest

import filterbank_synth as fs
import oracle
import paper_1411_5373_gb300 as FD
from paper_1411_5373_gb300 import build

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

T0, S = 600_000, 1 << 14


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    FD.load()


@pytest.fixture(scope="module")
def large_outputs():
    w = fs.LARGE_4K
    x = torch.from_numpy(fs.filterbank_f32(w)).cuda()
    res = {}
    for dtype in ("f32", "f16state"):
        p = FD.Plan(w.f_min, w.f_max, w.nf, w.nt, w.nd, dtype, schedule="fused")
        out = p.execute(x)
        p.device_status()
        torch.cuda.synchronize()
        res[dtype] = out
        p.close()
    del x
    return res


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


def test_large_beam_slice_matches_oracle(large_outputs):
    w = fs.LARGE_4K
    xs = fs.filterbank_f32(w, T0 - (w.nd - 1), T0 + S)
    T = oracle.build_tables(w.f_min, w.f_max, w.nf, w.nd)
    k = w.nd - 1
    got32 = large_outputs["f32"][:, T0:T0 + S].cpu().numpy()
    assert np.array_equal(got32, oracle.fdmt(xs, T, "f32")[:, k:])
    got16 = large_outputs["f16state"][:, T0:T0 + S].cpu().numpy()
    assert np.array_equal(got16, oracle.fdmt(xs, T, "f16state")[:, k:])
    ref = oracle.fdmt(xs.astype(np.float64), T, "f64")[:, k:]
    rms = np.sqrt(np.mean(ref ** 2, axis=1))
    assert np.all(np.abs(got32 - ref).max(axis=1) <= 1e-5 * rms)
    assert np.all(np.sqrt(np.mean((got16 - ref) ** 2, axis=1)) <= 2e-3 * rms)


def test_large_beam_fp16_state_snr(large_outputs):
    w = fs.LARGE_4K
    widths = [1, 2, 4, 8, 16, 32, 64, 128]
    for p in fs.draw_pulses(w):
        lo, hi = max(0, p.t0 - 8192), min(w.nt, p.t0 + 8192)
        r32 = large_outputs["f32"][p.delay, lo:hi].cpu().numpy()
        r16 = large_outputs["f16state"][p.delay, lo:hi].cpu().numpy()
        s32 = _snr(r32, p.t0 - lo, widths)
        s16 = _snr(r16, p.t0 - lo, widths)
        assert abs(s16 / s32 - 1.0) <= 5e-3, (p.delay, p.width, s16, s32)


def test_adjoint_dot_product_full_size():
    """<A x, y> = <x, A^T y> at Nf=Nd=1024, Nt=65536 with small integers:
    every partial sum is an exact integer in float32, the inner products are
    accumulated in float64, so the identity holds exactly."""
    w = fs.DIFF_1K
    p = FD.Plan(w.f_min, w.f_max, w.nf, w.nt, w.nd, "f32", schedule="fused")
    x = torch.from_numpy(fs.small_ints(7, (w.nf, w.nt))).cuda()
    y = torch.from_numpy(fs.small_ints(8, (w.nd, w.nt))).cuda()
    ax = p.execute(x).double()
    aty = p.adjoint(y).double()
    lhs = float(torch.sum(ax * y.double()).item())
    rhs = float(torch.sum(x.double() * aty).item())
    assert lhs == rhs
