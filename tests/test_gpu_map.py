"""The input mapping in front of the transform (d_min pre-shift of section
4.2, descending channel order) against the oracle's map_input followed by
its transform, through the C ABI: bit-exact for uint8, float32 and fp16
state; the adjoint (input and weight gradients) against the float64 oracle
adjoint taken back through map_input_adjoint."""
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


def reference(raw, w, d_min, desc, dtype):
    T = oracle.build_tables(w.f_min, w.f_max, w.nf, w.nd)
    s = oracle.input_shifts(w.f_min, w.f_max, w.nf, d_min)
    ref = oracle.fdmt(oracle.map_input(raw, s, desc), T, MODE[dtype])
    return ref.astype(np.int32) if dtype == "u8" else ref


@pytest.mark.parametrize("dtype", ["u8", "f32", "f16state"])
@pytest.mark.parametrize("schedule", ["plain", "fused"])
@pytest.mark.parametrize("d_min,desc", [(37, False), (0, True), (200, True)])
def test_mapped_transform_bitexact(dtype, schedule, d_min, desc):
    w = fs.SINGLE_SMALL
    x = fs.filterbank_u8(w) if dtype == "u8" else fs.filterbank_f32(w)
    raw = np.ascontiguousarray(x[::-1]) if desc else x
    p = FD.Plan(w.f_min, w.f_max, w.nf, w.nt, w.nd, dtype, schedule=schedule, d_min=d_min, descending=desc)
    got = p.execute(torch.from_numpy(raw).cuda()).cpu().numpy()
    assert np.array_equal(got, reference(raw, w, d_min, desc, dtype))


def test_mapped_pulse_moves_to_its_row():
    """A pulse of total delay 140 lands in row 140 - d_min of a d_min = 100
    plan (the planted pulse of the small workload has delay 40 at t = 500)."""
    w = fs.SINGLE_SMALL
    x = fs.filterbank_f32(w)
    base = FD.Plan(w.f_min, w.f_max, w.nf, w.nt, w.nd, "f32").execute(torch.from_numpy(x).cuda())
    d_ref = int(base[:, 499:503].amax(dim=1).argmax())
    assert abs(d_ref - 40) <= 1
    # the same input read as a d_min = 30 plan: the pulse now sits in row 10
    p = FD.Plan(w.f_min, w.f_max, w.nf, w.nt, w.nd, "f32", d_min=30)
    out = p.execute(torch.from_numpy(x).cuda())
    assert abs(int(out[:, 499:503].amax(dim=1).argmax()) - (d_ref - 30)) <= 1


def test_static_execute_refuses_mapped_plans():
    import ctypes
    w = fs.SINGLE_SMALL
    p = FD.Plan(w.f_min, w.f_max, w.nf, w.nt, w.nd, "f32", d_min=5)
    x = torch.zeros((w.nf, w.nt), device="cuda")
    y = torch.empty((w.nd, w.nt), device="cuda")
    st = FD.load().fdmt_execute_static(p._h, ctypes.c_void_p(x.data_ptr()), None, ctypes.c_void_p(y.data_ptr()),
                                        None)
    assert st == FD._native.ERR_UNSUPPORTED


@pytest.mark.parametrize("d_min,desc", [(90, False), (45, True)])
def test_mapped_adjoint_and_weight_gradient(d_min, desc):
    nf, nt, nd = 64, 1024, 64
    w = fs.SINGLE_SMALL
    T = oracle.build_tables(w.f_min, w.f_max, nf, nd)
    s = oracle.input_shifts(w.f_min, w.f_max, nf, d_min)
    p = FD.Plan(w.f_min, w.f_max, nf, nt, nd, "f32", d_min=d_min, descending=desc)
    x = fs.random_f32(61, nf, nt)
    g = fs.random_f32(62, nd, nt)
    wts = np.random.default_rng(3).uniform(0.5, 1.5, nf).astype(np.float32)
    gw = torch.empty(nf, device="cuda")
    gx = p.adjoint(torch.from_numpy(g).cuda(), x=torch.from_numpy(x).cuda(),
                   weights=torch.from_numpy(wts).cuda(), grad_weights=gw).cpu().numpy()
    ga = oracle.fdmt_adjoint(g.astype(np.float64), T)
    want = oracle.map_input_adjoint(ga * wts[:, None], s, desc)
    rms = np.sqrt(np.mean(want ** 2, axis=1)) + 1e-30
    assert np.all(np.max(np.abs(gx - want), axis=1) <= 1e-5 * rms + 1e-6)
    want_w = np.sum(oracle.map_input(x.astype(np.float64), s, desc) * ga, axis=1)
    assert np.allclose(gw.cpu().numpy(), want_w, rtol=1e-4, atol=1e-3 * np.abs(want_w).max())
    # the forward of the same plan with those weights is the oracle's, bit for bit
    out = p.execute(torch.from_numpy(x).cuda(), weights=torch.from_numpy(wts).cuda()).cpu().numpy()
    assert np.array_equal(out, oracle.fdmt(oracle.map_input(x, s, desc), T, "f32", weights=wts))


def test_mapped_full_size_uint8():
    """Nf = Nd = 1024, Nt = 65536 uint8 with d_min = 500, descending rows,
    fused schedule: the whole output against the oracle."""
    w = fs.SINGLE_1K
    x = np.ascontiguousarray(fs.filterbank_u8(w)[::-1])
    p = FD.Plan(w.f_min, w.f_max, w.nf, w.nt, w.nd, "u8", schedule="fused", d_min=500, descending=True)
    got = p.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.array_equal(got, reference(x, w, 500, True, "u8"))
