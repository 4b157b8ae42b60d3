"""Nf not a power of two (section 4.2: unequal split, f1 the border) on the
GPU, through the C ABI: plain schedule bit-exact to the oracle for uint8,
float32 and fp16 state; adjoint within 1e-5 of the float64 adjoint; level-
item batches bit-exact; the fused schedule refuses such plans."""
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


def data(dtype, seed, nf, nt):
    return fs.random_u8(seed, nf, nt) if dtype == "u8" else fs.random_f32(seed, nf, nt)


@pytest.mark.parametrize("dtype", ["u8", "f32", "f16state"])
@pytest.mark.parametrize("nf,nt,nd", [(3, 64, 7), (48, 1024, 64), (100, 512, 100), (257, 1024, 300),
                                      (1000, 2048, 700)])
def test_unequal_split_bitexact(dtype, nf, nt, nd):
    x = data(dtype, 70 + nf, nf, nt)
    p = FD.Plan(1200.0, 1600.0, nf, nt, nd, dtype)
    got = p.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.fdmt(x, oracle.build_tables(1200.0, 1600.0, nf, nd), MODE[dtype])
    assert np.array_equal(got, ref.astype(np.int32) if dtype == "u8" else ref)


def test_unequal_split_full_size_uint8():
    """Nf = 1000 channels, Nt = 65536, Nd = 1000: the whole output."""
    nf, nt, nd = 1000, 1 << 16, 1000
    x = fs.random_u8(fs.SEED_BASE + 50, nf, nt)
    got = FD.Plan(1200.0, 1600.0, nf, nt, nd, "u8").execute(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.fdmt(x, oracle.build_tables(1200.0, 1600.0, nf, nd), "i64")
    assert np.array_equal(got, ref.astype(np.int32))


@pytest.mark.parametrize("nf,nt,nd", [(48, 1024, 64), (5, 256, 9)])
def test_unequal_split_adjoint(nf, nt, nd):
    T = oracle.build_tables(1200.0, 1600.0, nf, nd)
    p = FD.Plan(1200.0, 1600.0, nf, nt, nd, "f32")
    g = fs.random_f32(81, nd, nt)
    got = p.adjoint(torch.from_numpy(g).cuda()).cpu().numpy()
    ref = oracle.fdmt_adjoint(g.astype(np.float64), T)
    rms = np.sqrt(np.mean(ref ** 2, axis=1)) + 1e-30
    assert np.all(np.max(np.abs(got - ref), axis=1) <= 1e-5 * rms)
    # dot-product identity on small integers (exact in float32)
    x = fs.small_ints(82, (nf, nt))
    y = fs.small_ints(83, (nd, nt))
    ax = p.execute(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    aty = p.adjoint(torch.from_numpy(y).cuda()).cpu().numpy().astype(np.float64)
    assert np.sum(ax * y) == np.sum(x * aty)


def test_unequal_split_batch_levels_and_fused_refusal():
    beams = [(1200.0, 1600.0, 48, 1024, 64), (1200.0, 1600.0, 64, 2048, 80), (1200.0, 1600.0, 7, 512, 20)]
    xs = [fs.random_u8(90 + i, b[2], b[3]) for i, b in enumerate(beams)]
    bp = FD.BatchPlan(beams, "u8", schedule="levels")
    outs = bp.execute([torch.from_numpy(v).cuda() for v in xs], bp.outputs("cuda"))
    for (f0, f1, nf, nt, nd), v, y in zip(beams, xs, outs):
        ref = oracle.fdmt(v, oracle.build_tables(f0, f1, nf, nd), "i64")
        assert np.array_equal(y.cpu().numpy(), ref.astype(np.int32))
    bp.close()
    with pytest.raises(FD.FdmtError) as e:
        FD.BatchPlan(beams, "u8", schedule="fused")
    assert e.value.status == FD._native.ERR_UNSUPPORTED
    with pytest.raises(FD.FdmtError) as e:
        FD.Plan(1200.0, 1600.0, 48, 1024, 64, "u8", schedule="fused")
    assert e.value.status == FD._native.ERR_UNSUPPORTED
