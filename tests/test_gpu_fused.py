"""Parity of the fused schedule (several merge levels per launch, cones staged
in shared memory by TMA) with the CPU oracle, through the C ABI.

Same bars as the plain schedule: bit-exact for uint8 -> int32, float32 and
fp16 state (the fused kernel keeps the oracle's association and rounding
points), plus the float64 tolerances; and no bounded device wait may have
given up (fdmt_device_status).
"""
import numpy as np
import pytest

import filterbank_synth as fs
import oracle
import paper_1411_5373_gb300 as FD
from paper_1411_5373_gb300 import build

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MODE = {"u8": "i64", "f32": "f32", "f16state": "f16state"}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    FD.load()


def run_fused(x_np, f_min, f_max, nd, dtype, weights=None, **sched):
    nf, nt = x_np.shape
    p = FD.Plan(f_min, f_max, nf, nt, nd, dtype, schedule="fused", **sched)
    x = torch.from_numpy(np.ascontiguousarray(x_np)).cuda()
    w = None if weights is None else torch.from_numpy(weights).cuda()
    out = p.execute(x, weights=w)
    p.device_status()
    return out.cpu().numpy(), p


def row_rms(a):
    return np.sqrt(np.mean(np.asarray(a, dtype=np.float64) ** 2, axis=1))


@pytest.mark.parametrize("dtype", ["f32", "u8", "f16state"])
def test_small_workload_bitexact(dtype):
    w = fs.SINGLE_SMALL
    x = fs.filterbank_u8(w) if dtype == "u8" else fs.filterbank_f32(w)
    T = oracle.build_tables(w.f_min, w.f_max, w.nf, w.nd)
    got, _ = run_fused(x, w.f_min, w.f_max, w.nd, dtype)
    assert np.array_equal(got, oracle.fdmt(x, T, MODE[dtype]))


EDGE = [
    (2, 16, 1, "u8", {}), (2, 32, 32, "f32", {}), (4, 1040, 6, "u8", {}),
    (64, 1040, 64, "f32", {}), (128, 2064, 300, "u8", {}), (256, 2048, 2048, "u8", {}),
    (1024, 4112, 100, "f32", {}), (4096, 1024, 256, "u8", {}), (8, 4096, 4096, "f32", {}),
    (16, 48, 40, "f16state", {}), (512, 3088, 700, "f16state", {}),
    (32, 1088, 50, "u8", {"tile": 64, "bounds": [0, 1, 2, 3, 4, 5]}),
    (64, 2112, 100, "f32", {"tile": 128, "smem_budget": 20 * 1024, "bounds": [0, 3, 6]}),
    (64, 1984, 64, "f16state", {"tile": 64, "smem_budget": 24 * 1024}),
    (256, 4096, 2048, "f32", {"tile": 512, "smem_budget": 200 * 1024}),
]


@pytest.mark.parametrize("nf,nt,nd,dtype,sched", EDGE)
def test_edge_shapes_bitexact(nf, nt, nd, dtype, sched):
    T = oracle.build_tables(1200.0, 1600.0, nf, nd)
    seed = nf * 7919 + nt * 31 + nd + 5
    x = fs.random_u8(seed, nf, nt) if dtype == "u8" else fs.random_f32(seed, nf, nt)
    got, _ = run_fused(x, 1200.0, 1600.0, nd, dtype, **sched)
    assert np.array_equal(got, oracle.fdmt(x, T, MODE[dtype]))


def test_weights_bitexact():
    nf, nt, nd = 64, 2048, 80
    x = fs.random_f32(17, nf, nt)
    wts = np.random.default_rng(3).uniform(0.0, 2.0, nf).astype(np.float32)
    T = oracle.build_tables(1200.0, 1600.0, nf, nd)
    got, _ = run_fused(x, 1200.0, 1600.0, nd, "f32", weights=wts)
    assert np.array_equal(got, oracle.fdmt(x, T, "f32", weights=wts))


@pytest.mark.parametrize("dtype", ["u8", "f32", "f16state"])
def test_1k_full_bitexact(dtype):
    w = fs.SINGLE_1K
    x = fs.filterbank_u8(w) if dtype == "u8" else fs.filterbank_f32(w)
    T = oracle.build_tables(w.f_min, w.f_max, w.nf, w.nd)
    got, p = run_fused(x, w.f_min, w.f_max, w.nd, dtype)
    assert np.array_equal(got, oracle.fdmt(x, T, MODE[dtype]))
    if dtype != "u8":
        ref = oracle.fdmt(x.astype(np.float64), T, "f64")
        err = np.abs(got.astype(np.float64) - ref)
        if dtype == "f32":
            assert np.all(err.max(axis=1) <= 1e-5 * row_rms(ref))
        else:
            assert np.all(np.sqrt(np.mean(err ** 2, axis=1)) <= 2e-3 * row_rms(ref))


def test_fused_equals_plain_and_is_deterministic():
    x = fs.random_f32(23, 256, 8192)
    xt = torch.from_numpy(x).cuda()
    pf = FD.Plan(1200.0, 1600.0, 256, 8192, 512, "f32", schedule="fused")
    pp = FD.Plan(1200.0, 1600.0, 256, 8192, 512, "f32", schedule="plain")
    a = pf.execute(xt)
    b = pf.execute(xt)
    c = pp.execute(xt)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(a, c)


@pytest.mark.parametrize("nf,nt,nd", [(1024, 4096, 1024), (4096, 2048, 256), (256, 4096, 2048)])
def test_uint16_state_saturated_input_exact(nf, nt, nd):
    """uint8 input stores the levels between launches as uint16 where the
    sums fit: with every sample at 255 each stored sum is at its largest, so
    a level wrongly narrowed would wrap and differ from the oracle."""
    T = oracle.build_tables(1200.0, 1600.0, nf, nd)
    for x in (np.full((nf, nt), 255, dtype=np.uint8), fs.random_u8(29, nf, nt)):
        want = oracle.fdmt(x, T, "i64")
        xt = torch.from_numpy(x).cuda()
        p16 = FD.Plan(1200.0, 1600.0, nf, nt, nd, "u8", schedule="fused")
        assert (p16.fused_table(0).reshape(-1, 16)[:, 15] == 2).any(), "expected uint16 launch-boundary state"
        p32 = FD.Plan(1200.0, 1600.0, nf, nt, nd, "u8", schedule="fused", state16=False)
        assert (p32.fused_table(0).reshape(-1, 16)[:, 14:16] == 4).sum() >= 1
        for p in (p16, p32):
            got = p.execute(xt).cpu().numpy()
            p.device_status()
            assert np.array_equal(got, want)


@pytest.mark.parametrize("gamma", [-1.0, 1.5])
@pytest.mark.parametrize("dtype", ["u8", "f32"])
@pytest.mark.parametrize("schedule", ["plain", "fused"])
def test_power_law_curves_bitexact(gamma, dtype, schedule):
    """Another functional form Dt ~ f^gamma (fdmt_plan_curve) runs through
    the same kernels: bit-exact to the oracle built with the same gamma."""
    nf, nt, nd = 256, 4096, 300
    T = oracle.build_tables(1200.0, 1600.0, nf, nd, gamma=gamma)
    x = fs.random_u8(31, nf, nt) if dtype == "u8" else fs.random_f32(31, nf, nt)
    p = FD.Plan(1200.0, 1600.0, nf, nt, nd, dtype, schedule=schedule, gamma=gamma)
    got = p.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    p.device_status()
    assert np.array_equal(got, oracle.fdmt(x, T, MODE[dtype]))
