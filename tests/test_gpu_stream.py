"""Overlap-save streaming (``fdmt_stream_*``) against one oracle transform of
the whole stream: each push's output must equal the matching output columns
bit for bit, because output column t depends only on input columns
[t - Nd + 1, t] (the recursion looks back in time only; samples before the
first are zero by the copy rule)."""
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


def stream_all(x, f_min, f_max, nd, chunk, dtype, schedule="plain"):
    nf, nt = x.shape
    st = FD.Stream(f_min, f_max, nf, chunk, nd, dtype, schedule=schedule)
    outs = [st.push(torch.from_numpy(np.ascontiguousarray(x[:, i:i + chunk])).cuda()).cpu().numpy()
            for i in range(0, nt, chunk)]
    torch.cuda.synchronize()
    return np.concatenate(outs, axis=1), st


@pytest.mark.parametrize("dtype", ["u8", "f32", "f16state"])
@pytest.mark.parametrize("schedule", ["plain", "fused"])
@pytest.mark.parametrize("chunk", [256, 16])  # 16 < carry: the carry spans several chunks
def test_stream_equals_whole_transform(dtype, schedule, chunk):
    w = fs.SINGLE_SMALL
    nt = 1024 if chunk == 256 else 320
    x = fs.filterbank_u8(w, 0, nt) if dtype == "u8" else fs.filterbank_f32(w, 0, nt)
    got, st = stream_all(x, w.f_min, w.f_max, w.nd, chunk, dtype, schedule)
    assert st.carry == 64 and st.window == 64 + chunk
    ref = oracle.fdmt(x, oracle.build_tables(w.f_min, w.f_max, w.nf, w.nd), MODE[dtype])
    ref = ref.astype(np.int32) if dtype == "u8" else ref
    assert np.array_equal(got, ref)
    st.close()


def test_stream_reset_starts_over():
    w = fs.SINGLE_SMALL
    x = fs.filterbank_f32(w, 0, 512)
    st = FD.Stream(w.f_min, w.f_max, w.nf, 256, w.nd, "f32")
    a = st.push(torch.from_numpy(np.ascontiguousarray(x[:, :256])).cuda()).cpu().numpy()
    st.push(torch.from_numpy(np.ascontiguousarray(x[:, 256:])).cuda())
    st.reset()
    b = st.push(torch.from_numpy(np.ascontiguousarray(x[:, :256])).cuda()).cpu().numpy()
    assert np.array_equal(a, b)
    st.close()


def test_stream_full_size_uint8():
    """The Nf = Nd = 1024 workload (uint8) in four chunks of 16384 samples
    against the oracle over all 65536 samples."""
    w = fs.SINGLE_1K
    x = fs.filterbank_u8(w)
    got, st = stream_all(x, w.f_min, w.f_max, w.nd, 16384, "u8", "fused")
    assert st.carry == 1024
    ref = oracle.fdmt(x, oracle.build_tables(w.f_min, w.f_max, w.nf, w.nd), "i64")
    assert np.array_equal(got, ref.astype(np.int32))
    st.close()


@pytest.mark.parametrize("schedule", ["plain", "fused"])
def test_stream_unequal_split(schedule):
    """Nf = 48 (not a power of two) streamed in chunks of 128 samples."""
    nf, nt, nd = 48, 1024, 64
    x = fs.random_u8(23, nf, nt)
    got, st = stream_all(x, 1200.0, 1600.0, nd, 128, "u8", schedule)
    ref = oracle.fdmt(x, oracle.build_tables(1200.0, 1600.0, nf, nd), "i64")
    assert np.array_equal(got, ref.astype(np.int32))
    st.close()
