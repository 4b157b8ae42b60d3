"""Pipelined host execution (``fdmt_pipeline_*``): every queued transform's
output, read after wait, equals the oracle's (bit-exact), with consecutive
steps overlapping on separate streams and two device slots taking turns."""
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


@pytest.mark.parametrize("dtype,schedule", [("u8", "fused"), ("f32", "plain")])
def test_pipeline_outputs_equal_oracle(dtype, schedule):
    w = fs.SINGLE_SMALL
    T = oracle.build_tables(w.f_min, w.f_max, w.nf, w.nd)
    p = FD.Plan(w.f_min, w.f_max, w.nf, w.nt, w.nd, dtype, schedule=schedule)
    xs = [fs.random_u8(10 + i, w.nf, w.nt) if dtype == "u8" else fs.random_f32(10 + i, w.nf, w.nt)
          for i in range(7)]
    hin = [torch.from_numpy(x).pin_memory() for x in xs]
    hout = [torch.empty((w.nd, w.nt), dtype=torch.int32 if dtype == "u8" else torch.float32).pin_memory()
            for _ in xs]
    pipe = FD.Pipeline(p)
    for a, b in zip(hin[:2], hout[:2]):
        pipe.push(a, b)
    pipe.wait()
    for a, b in zip(hin[2:], hout[2:]):
        pipe.push(a, b)
    pipe.wait()
    for x, y in zip(xs, hout):
        ref = oracle.fdmt(x, T, "i64" if dtype == "u8" else "f32")
        assert np.array_equal(y.numpy(), ref.astype(np.int32) if dtype == "u8" else ref)
    pipe.close()
