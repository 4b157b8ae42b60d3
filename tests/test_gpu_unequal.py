"""Nf not a power of two (section 4.2: unequal split, f1 the border) on the
GPU, through the C ABI: the plain and fused schedules bit-exact to the
oracle for uint8, float32 and fp16 state; the fused search epilogue bit-
exact; adjoint within 1e-5 of the float64 adjoint; level-item, persistent
fused and per-beam launch batches bit-exact."""
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
@pytest.mark.parametrize("schedule", ["plain", "fused"])
def test_unequal_split_bitexact(dtype, nf, nt, nd, schedule):
    x = data(dtype, 70 + nf, nf, nt)
    p = FD.Plan(1200.0, 1600.0, nf, nt, nd, dtype, schedule=schedule)
    got = p.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.fdmt(x, oracle.build_tables(1200.0, 1600.0, nf, nd), MODE[dtype])
    assert np.array_equal(got, ref.astype(np.int32) if dtype == "u8" else ref)


@pytest.mark.parametrize("dtype", ["u8", "f32"])
@pytest.mark.parametrize("nf,nt,nd,sched", [(48, 1024, 64, {"tile": 128, "bounds": [0, 1, 3, 6]}),
                                            (100, 2048, 100, {"tile": 64, "smem_budget": 40 * 1024}),
                                            (257, 1024, 300, {"tile": 128, "bounds": [0, 3, 6, 9]}),
                                            (1000, 2048, 700, {"bounds": [0, 2, 5, 7, 10]})])
def test_unequal_split_fused_forced(dtype, nf, nt, nd, sched):
    """Forced groupings, tiles and budgets: single and paired stages, row
    splits and walks over bands without an upper half."""
    x = data(dtype, 170 + nf, nf, nt)
    p = FD.Plan(1200.0, 1600.0, nf, nt, nd, dtype, schedule="fused", **sched)
    got = p.execute(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.fdmt(x, oracle.build_tables(1200.0, 1600.0, nf, nd), MODE[dtype])
    assert np.array_equal(got, ref.astype(np.int32) if dtype == "u8" else ref)


@pytest.mark.parametrize("schedule", ["plain", "fused"])
def test_unequal_split_full_size_uint8(schedule):
    """Nf = 1000 channels, Nt = 65536, Nd = 1000: the whole output."""
    nf, nt, nd = 1000, 1 << 16, 1000
    x = fs.random_u8(fs.SEED_BASE + 50, nf, nt)
    got = FD.Plan(1200.0, 1600.0, nf, nt, nd, "u8", schedule=schedule).execute(
        torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.fdmt(x, oracle.build_tables(1200.0, 1600.0, nf, nd), "i64")
    assert np.array_equal(got, ref.astype(np.int32))


@pytest.mark.parametrize("dtype,nf,nt,nd,k", [("f32", 48, 2048, 64, 6), ("u8", 100, 4096, 90, 9),
                                              ("f32", 1000, 4096, 700, 8)])
def test_unequal_split_fused_search(dtype, nf, nt, nd, k):
    """The search epilogue in the last fused launch of an unequal split."""
    x = data(dtype, 190 + nf, nf, nt)
    p = FD.Plan(1200.0, 1600.0, nf, nt, nd, dtype, schedule="fused", search_widths=k)
    out, peak, when = p.execute_search(torch.from_numpy(x).cuda(), k)
    ref = oracle.fdmt(x, oracle.build_tables(1200.0, 1600.0, nf, nd), MODE[dtype])
    ref = ref.astype(np.int32) if dtype == "u8" else ref
    assert np.array_equal(out.cpu().numpy(), ref)
    rp, rt = oracle.boxcar_search(ref, k)
    assert np.array_equal(peak.cpu().numpy(), rp)
    assert np.array_equal(when.cpu().numpy(), rt)


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


@pytest.mark.parametrize("schedule", ["levels", "fused", "launches"])
@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_unequal_split_batches(schedule, dtype):
    beams = [(1200.0, 1600.0, 48, 1024, 64), (1200.0, 1600.0, 64, 2048, 80), (1200.0, 1600.0, 7, 512, 20),
             (1100.0, 1500.0, 100, 2048, 100), (1200.0, 1600.0, 48, 1024, 64), (1300.0, 1450.0, 257, 1024, 200)]
    xs = [data(dtype, 90 + i, b[2], b[3]) for i, b in enumerate(beams)]
    bp = FD.BatchPlan(beams, dtype, schedule=schedule)
    outs = bp.execute([torch.from_numpy(v).cuda() for v in xs], bp.outputs("cuda"))
    for (f0, f1, nf, nt, nd), v, y in zip(beams, xs, outs):
        ref = oracle.fdmt(v, oracle.build_tables(f0, f1, nf, nd), MODE[dtype])
        assert np.array_equal(y.cpu().numpy(), ref.astype(np.int32) if dtype == "u8" else ref)
    bp.close()
