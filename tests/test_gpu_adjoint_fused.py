"""The fused adjoint (pull cones of several transposed levels per launch,
ending with the transpose of the Option-1 initialisation) on the GPU,
through the C ABI.

Bars: bit-exact against the CPU emulator of the same cone tables (same
float32 order of additions); exact against the float64 oracle adjoint on
small-integer gradients (every partial sum is an exact integer in float32);
within 1e-5 of the row RMS against the oracle on random gradients; the
dot-product identity <A x, y> = <x, A^T y> exact at full size.
"""
import numpy as np
import pytest

import filterbank_synth as fs
import oracle
import paper_1411_5373_gb300 as FD
from adjoint_emulator import check_adjoint_tables, emulate_adjoint
from paper_1411_5373_gb300 import build

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    FD.load()


def rows_close(got, ref, tol):
    rms = np.sqrt(np.mean(ref ** 2, axis=1)) + 1e-30
    err = np.max(np.abs(got - ref), axis=1) / rms
    assert np.all(err <= tol), (int(np.argmax(err)), float(err.max()))


CASES = [
    # (f_min, f_max, nf, nt, nd), plan keywords
    ((1200.0, 1600.0, 16, 256, 16), {}),
    ((1200.0, 1600.0, 64, 512, 64), {}),
    ((1200.0, 1600.0, 64, 1040, 80), {"adjoint_tile": 64, "adjoint_bounds": [0, 1, 2, 4, 6]}),
    ((1200.0, 1600.0, 128, 2064, 200), {"adjoint_tile": 128, "adjoint_smem_budget": 48 * 1024}),
    ((1200.0, 1600.0, 256, 4096, 300), {"adjoint_tile": 512, "adjoint_bounds": [0, 2, 5, 8]}),
    ((1200.0, 1600.0, 48, 1024, 64), {}),
    ((1200.0, 1600.0, 3, 64, 7), {}),
    ((1200.0, 1600.0, 100, 512, 90), {"adjoint_tile": 128, "adjoint_smem_budget": 40 * 1024}),
    ((1300.0, 1450.0, 257, 1024, 200), {}),
]


@pytest.mark.parametrize("shape,kw", CASES)
def test_fused_adjoint_equals_emulator_and_oracle(shape, kw):
    f0, f1, nf, nt, nd = shape
    p = FD.Plan(f0, f1, nf, nt, nd, "f32", schedule="fused", adjoint="fused", **kw)
    assert len(p.fused_table(10)) > 0, "the plan has no fused adjoint"
    check_adjoint_tables(p)
    T = oracle.build_tables(f0, f1, nf, nd)
    # small integers: exact against the float64 oracle
    y = fs.small_ints(61, (nd, nt)).astype(np.float32)
    got = p.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    assert np.array_equal(got, oracle.fdmt_adjoint(y.astype(np.float64), T).astype(np.float32))
    # random floats: the emulator's order bit for bit, the oracle within 1e-5
    g = fs.random_f32(62, nd, nt)
    got = p.adjoint(torch.from_numpy(g).cuda()).cpu().numpy()
    emu = emulate_adjoint(p, g)
    assert np.array_equal(got.view(np.int32), emu.view(np.int32))
    rows_close(got, oracle.fdmt_adjoint(g.astype(np.float64), T), 1e-5)


def test_fused_adjoint_weights():
    f0, f1, nf, nt, nd = 1200.0, 1600.0, 64, 1024, 64
    p = FD.Plan(f0, f1, nf, nt, nd, "f32", schedule="fused", adjoint="fused")
    T = oracle.build_tables(f0, f1, nf, nd)
    x = fs.random_f32(71, nf, nt)
    g = fs.random_f32(72, nd, nt)
    wts = np.random.default_rng(7).uniform(0.5, 1.5, nf).astype(np.float32)
    # scaled in the launch that applies the initialisation transpose
    got = p.adjoint(torch.from_numpy(g).cuda(), weights=torch.from_numpy(wts).cuda()).cpu().numpy()
    assert np.array_equal(got.view(np.int32), emulate_adjoint(p, g, wts).view(np.int32))
    # with the weight gradient: unscaled adjoint, then the weights epilogue
    gw = torch.empty(nf, device="cuda")
    gx = p.adjoint(torch.from_numpy(g).cuda(), x=torch.from_numpy(x).cuda(),
                   weights=torch.from_numpy(wts).cuda(), grad_weights=gw).cpu().numpy()
    gi = oracle.fdmt_adjoint(g.astype(np.float64), T)
    rows_close(gx, gi * wts[:, None], 1e-5)
    want = np.sum(x.astype(np.float64) * gi, axis=1)
    assert np.allclose(gw.cpu().numpy(), want, rtol=1e-4, atol=1e-3 * np.abs(want).max())


@pytest.mark.parametrize("d_min,descending", [(40, False), (0, True), (25, True)])
def test_fused_adjoint_mapped_input(d_min, descending):
    """Plans with the d_min pre-shift or descending channels: the gradient
    is taken through the mapping (dot-product identity, exact)."""
    f0, f1, nf, nt, nd = 1200.0, 1600.0, 64, 1024, 64
    p = FD.Plan(f0, f1, nf, nt, nd, "f32", schedule="fused", adjoint="fused", d_min=d_min,
                descending=descending)
    q = FD.Plan(f0, f1, nf, nt, nd, "f32", schedule="plain", d_min=d_min, descending=descending)
    x = torch.from_numpy(fs.small_ints(73, (nf, nt))).cuda()
    y = torch.from_numpy(fs.small_ints(74, (nd, nt))).cuda()
    ax = p.execute(x).double()
    aty = p.adjoint(y)
    assert float(torch.sum(ax * y.double())) == float(torch.sum(x.double() * aty.double()))
    assert torch.equal(aty, q.adjoint(y))  # exact integers either way


def test_fused_adjoint_full_size_against_plain():
    """Nf = Nd = 1024, Nt = 65536 (the differentiable workload): the fused
    and plain adjoints agree to float32 rounding (5e-6 of the row RMS); the
    static table checks hold."""
    w = fs.DIFF_1K
    p = FD.Plan(w.f_min, w.f_max, w.nf, w.nt, w.nd, "f32", schedule="fused", adjoint="fused")
    q = FD.Plan(w.f_min, w.f_max, w.nf, w.nt, w.nd, "f32", schedule="fused", adjoint="plain")
    assert len(q.fused_table(10)) == 0
    check_adjoint_tables(p)
    g = torch.from_numpy(fs.random_f32(75, w.nd, w.nt)).cuda()
    a = p.adjoint(g).cpu().numpy().astype(np.float64)
    b = q.adjoint(g).cpu().numpy().astype(np.float64)
    rows_close(a, b, 5e-6)
