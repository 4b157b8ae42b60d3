"""Batched uneven beams in one persistent, graph-recorded launch
(fdmt_plan_batch / fdmt_execute_batch), through the C ABI, with both work
schedules: one merge level per item, and every beam's fused cone programme.

Every beam must equal the oracle bit for bit (uint8 -> int32 and float32),
replays of the recorded launch must agree, and a work list with a missing
producer (injected on the host) must end in FDMT_ERR_TIMEOUT without a
device fault, after which the same batch still runs correctly.
"""
import time

import numpy as np
import pytest

import filterbank_synth as fs
import oracle
import paper_1411_5373_gb300 as FD
from paper_1411_5373_gb300 import _native as N
from paper_1411_5373_gb300 import build

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

BEAMS = [  # (f_min, f_max, nf, nt, nd): uneven shapes, ragged tiles
    (1200.0, 1600.0, 256, 4096, 256),
    (1200.0, 1600.0, 512, 8192, 1024),
    (1200.0, 1600.0, 64, 2064, 64),
    (1100.0, 1700.0, 1024, 4112, 512),
    (1200.0, 1600.0, 4096, 1024, 256),
    (1200.0, 1600.0, 256, 2048, 2048),
    (300.0, 310.0, 128, 3088, 100),
    (1200.0, 1600.0, 2, 16, 1),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    FD.load()


def _inputs(dtype):
    xs = []
    for i, (_, _, nf, nt, _) in enumerate(BEAMS):
        xs.append(fs.random_u8(100 + i, nf, nt) if dtype == "u8" else fs.random_f32(100 + i, nf, nt))
    return xs


@pytest.mark.parametrize("dtype,params", [("u8", {}), ("u8", {"rows_per_item": 4, "tile": 1024}),
                                          ("f32", {"rows_per_item": 32, "tile": 4096}),
                                          ("f16state", {}),
                                          ("u8", {"schedule": "fused"}),
                                          ("u8", {"schedule": "fused", "fused_tile": 256}),
                                          ("f32", {"schedule": "fused", "fused_tile": 128,
                                                   "smem_budget": 40 * 1024}),
                                          ("f32", {"schedule": "fused", "smem_budget": 150 * 1024})])
def test_batch_bitexact_against_oracle(dtype, params):
    bp = FD.BatchPlan(BEAMS, dtype, **params)
    xs = _inputs(dtype)
    ins = [torch.from_numpy(x).cuda() for x in xs]
    outs = bp.outputs()
    bp.execute(ins, outs)
    mode = {"u8": "i64", "f32": "f32", "f16state": "f16state"}[dtype]
    for (f_min, f_max, nf, nt, nd), x, y in zip(BEAMS, xs, outs):
        T = oracle.build_tables(f_min, f_max, nf, nd)
        assert np.array_equal(y.cpu().numpy(), oracle.fdmt(x, T, mode)), (nf, nt, nd)
    # replay of the recorded launch gives the same bits
    outs2 = [torch.empty_like(y) for y in outs]
    bp.execute(ins, outs2)   # new pointers: re-recorded
    bp.execute(ins, outs2)   # replay
    for a, b in zip(outs, outs2):
        assert torch.equal(a, b)


@pytest.mark.parametrize("schedule,drop", [("levels", 2), ("fused", 0)])
def test_missing_producer_times_out_then_recovers(schedule, drop):
    bp = FD.BatchPlan(BEAMS[:4], "u8", wait_ms=300, schedule=schedule)
    xs = _inputs("u8")[:4]
    ins = [torch.from_numpy(x).cuda() for x in xs]
    outs = bp.outputs()
    bp.drop_level(1, drop)         # beam 1's level (group) never runs: the next one waits for it
    t0 = time.time()
    with pytest.raises(FD.FdmtError) as ei:
        bp.execute(ins, outs)
    assert ei.value.status == N.ERR_TIMEOUT
    assert time.time() - t0 < 30
    bp.drop_level(0, -1)           # full work list again: the context is still usable
    bp.execute(ins, outs)
    for (f_min, f_max, nf, nt, nd), x, y in zip(BEAMS[:4], xs, outs):
        T = oracle.build_tables(f_min, f_max, nf, nd)
        assert np.array_equal(y.cpu().numpy(), oracle.fdmt(x, T, "i64"))


def test_batch_argument_errors():
    with pytest.raises(FD.FdmtError):
        FD.BatchPlan([(1200.0, 1600.0, 64, 1024, 2048)], "u8")    # Nd > Nt
    with pytest.raises(FD.FdmtError):
        FD.BatchPlan(BEAMS[:2], "u8", tile=1000)                 # tile not a multiple of 1024
    with pytest.raises(FD.FdmtError):
        FD.BatchPlan(BEAMS[:2], "u8", schedule="fused", fused_tile=100)   # not a multiple of 64
    with pytest.raises(FD.FdmtError):
        FD.BatchPlan(BEAMS[:2], "f16state", schedule="fused")             # fused batch: u8 / f32
    bp = FD.BatchPlan(BEAMS[:2], "u8")
    xs = [torch.zeros((nf, nt), dtype=torch.uint8, device="cuda") for (_, _, nf, nt, _) in BEAMS[:2]]
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(FD.FdmtError) as ei:
        bp.execute(xs, bp.outputs(), workspace=small)
    assert ei.value.status == N.ERR_WORKSPACE


def test_batch_launch_schedule_bitexact():
    """schedule "launches": one plan per beam over four streams; every beam
    bit-exact, including a beam whose Nf is not a power of two (plain)."""
    beams = list(BEAMS[:4]) + [(1200.0, 1600.0, 48, 1024, 40)]
    xs = [fs.random_u8(120 + i, b[2], b[3]) for i, b in enumerate(beams)]
    bp = FD.BatchPlan(beams, "u8", schedule="launches")
    outs = bp.execute([torch.from_numpy(v).cuda() for v in xs], bp.outputs("cuda"))
    for (f0, f1, nf, nt, nd), v, y in zip(beams, xs, outs):
        ref = oracle.fdmt(v, oracle.build_tables(f0, f1, nf, nd), "i64")
        assert np.array_equal(y.cpu().numpy(), ref.astype(np.int32))
    g, bounds, sizes = None, None, None
    bounds, sizes = bp.levels(0, sizes=True)
    assert bounds[0] == 0 and bounds[-1] > 0 and len(sizes) == len(bounds)
    with pytest.raises(FD.FdmtError) as e:
        bp.drop_level(0, 1)
    assert e.value.status == N.ERR_UNSUPPORTED
    bp.close()
