"""C ABI checks that need no GPU: the library loads, exports every symbol the
header declares, validates arguments, and its host-side delay tables equal
the oracle's independently built tables (integer equality)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_1411_5373_gb300 as F
from paper_1411_5373_gb300 import _native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fdmt_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1411_5373_gb300 import build
    build.build()
    return N.load()


def test_library_exports_every_declared_symbol(lib):
    declared = _header_functions()
    assert {"fdmt_plan", "fdmt_execute", "fdmt_adjoint", "fdmt_destroy"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(N.SIGNATURES), declared ^ set(N.SIGNATURES)


def test_error_strings(lib):
    for st in (N.OK, N.ERR_INVALID_ARG, N.ERR_UNSUPPORTED, N.ERR_CUDA, N.ERR_NO_MEMORY,
               N.ERR_TIMEOUT, N.ERR_WORKSPACE):
        assert N.error_string(st) and N.error_string(st) != "unknown status"
    assert N.error_string(12345) == "unknown status"


def _plan_status(*args):
    lib = N.load()
    h = ctypes.c_void_p()
    st = lib.fdmt_plan(*args, ctypes.byref(h))
    if st == N.OK:
        lib.fdmt_destroy(h)
    return st


@pytest.mark.parametrize("args,want", [
    ((1200.0, 1600.0, 64, 1024, 64, N.F32_F32, N.PLAN_HOST_ONLY), N.OK),
    ((1200.0, 1600.0, 48, 1024, 64, N.F32_F32, N.PLAN_HOST_ONLY), N.OK),
    ((1200.0, 1600.0, 48, 1024, 64, N.F32_F32, N.PLAN_HOST_ONLY | N.SCHED_FUSED), N.OK),
    ((1200.0, 1600.0, 3, 1024, 64, N.U8_I32, N.PLAN_HOST_ONLY | N.SCHED_FUSED), N.OK),
    ((1200.0, 1600.0, 1, 1024, 64, N.F32_F32, N.PLAN_HOST_ONLY), N.ERR_INVALID_ARG),
    ((1600.0, 1200.0, 64, 1024, 64, N.F32_F32, N.PLAN_HOST_ONLY), N.ERR_INVALID_ARG),
    ((0.0, 1200.0, 64, 1024, 64, N.F32_F32, N.PLAN_HOST_ONLY), N.ERR_INVALID_ARG),
    ((float("nan"), 1200.0, 64, 1024, 64, N.F32_F32, N.PLAN_HOST_ONLY), N.ERR_INVALID_ARG),
    ((1200.0, 1600.0, 64, 1024, 2048, N.F32_F32, N.PLAN_HOST_ONLY), N.ERR_INVALID_ARG),
    ((1200.0, 1600.0, 64, 1024, 0, N.F32_F32, N.PLAN_HOST_ONLY), N.ERR_INVALID_ARG),
    ((1200.0, 1600.0, 64, 1026, 64, N.F32_F32, N.PLAN_HOST_ONLY), N.ERR_INVALID_ARG),
    ((1200.0, 1600.0, 64, 1032, 64, N.U8_I32, N.PLAN_HOST_ONLY), N.ERR_INVALID_ARG),
    ((1200.0, 1600.0, 64, 1040, 64, N.U8_I32, N.PLAN_HOST_ONLY), N.OK),
    ((1200.0, 1600.0, 64, 1028, 64, N.F32_F16STATE, N.PLAN_HOST_ONLY), N.ERR_INVALID_ARG),
    ((1200.0, 1600.0, 64, 1032, 64, N.F32_F16STATE, N.PLAN_HOST_ONLY), N.OK),
    ((1200.0, 1600.0, 64, 1024, 64, 7, N.PLAN_HOST_ONLY), N.ERR_INVALID_ARG),
    ((1200.0, 1600.0, 64, 1024, 64, N.F32_F32, 1 << 9), N.ERR_INVALID_ARG),
])
def test_plan_argument_validation(lib, args, want):
    assert _plan_status(*args) == want


def test_host_only_plan_refuses_execution(lib):
    p = F.Plan(1200, 1600, 64, 1024, 64, "f32", host_only=True)
    ws = ctypes.c_void_p(256)
    st = lib.fdmt_execute(p._h, ctypes.c_void_p(16), None, ctypes.c_void_p(16), ws, 1 << 30, None)
    assert st == N.ERR_INVALID_ARG
    assert lib.fdmt_execute(None, None, None, None, None, 0, None) == N.ERR_INVALID_ARG
    lib.fdmt_destroy(None)  # NULL-safe


def test_workspace_sizes(lib):
    p = F.Plan(1200, 1600, 1024, 65536, 1024, "f32", host_only=True)
    # ping-pong of the largest even level (0: 2047 rows) and odd level (1: 1535 rows)
    assert p.workspace_bytes == (2047 + 1535) * 65536 * 4
    p16 = F.Plan(1200, 1600, 1024, 65536, 1024, "f16state", host_only=True)
    assert p16.workspace_bytes == (2047 + 1535) * 65536 * 2
    # transposed programme, two levels per step: steps write levels 8, 6, 4, 2, 0
    # into buffers 0, 1, 0, 1, 0
    assert p16.adjoint_workspace_bytes == (2047 + 1279) * 65536 * 4
    pu = F.Plan(1200, 1600, 1024, 65536, 1024, "u8", host_only=True)
    with pytest.raises(F.FdmtError):
        pu.adjoint_workspace_bytes


CASES = [(1200.0, 1600.0, 64, 64), (1200.0, 1600.0, 1024, 1024), (1100.0, 1700.0, 4096, 4096),
         (1200.0, 1600.0, 256, 2048), (1200.0, 1600.0, 4096, 256), (1.0, 2.0, 4, 6),
         (1.0, 2.0, 2, 1), (300.0, 310.0, 512, 100), (100.0, 900.0, 128, 1000),
         # Nf not a power of two (the unequal split of section 4.2)
         (1200.0, 1600.0, 3, 7), (1200.0, 1600.0, 96, 80), (1100.0, 1700.0, 1000, 700), (1.0, 2.0, 5, 6),
         (300.0, 310.0, 37, 50)]


@pytest.mark.parametrize("f_min,f_max,nf,nd", CASES)
def test_tables_equal_oracle(lib, f_min, f_max, nf, nd):
    nt = max(16, ((nd + 15) // 16) * 16)
    p = F.Plan(f_min, f_max, nf, nt, nd, "f32", host_only=True)
    T = oracle.build_tables(f_min, f_max, nf, nd)
    assert p.levels == T.levels
    for l in range(T.levels + 1):
        assert np.array_equal(p.band_rows(l), np.asarray(T.rows[l]))
    for l in range(1, T.levels + 1):
        for b in range(len(T.rows[l])):
            assert np.array_equal(p.band_dl(l, b), T.dl[l][b]), (l, b)


@pytest.mark.parametrize("gamma", [-1.0, 1.0, 0.5, 2.5, -3.0])
def test_tables_equal_oracle_power_law(lib, gamma):
    """Other curve families (fdmt_plan_curve): the host tables equal the
    oracle's for the same power law."""
    for (f_min, f_max, nf, nd) in [(1200.0, 1600.0, 64, 100), (1024.0, 2048.0, 256, 300), (300.0, 310.0, 32, 5)]:
        p = F.Plan(f_min, f_max, nf, ((nd + 15) // 16) * 16, nd, "f32", host_only=True, gamma=gamma)
        T = oracle.build_tables(f_min, f_max, nf, nd, gamma=gamma)
        for l in range(T.levels + 1):
            assert np.array_equal(p.band_rows(l), np.asarray(T.rows[l]))
        for l in range(1, T.levels + 1):
            for b in range(len(T.rows[l])):
                assert np.array_equal(p.band_dl(l, b), T.dl[l][b]), (gamma, l, b)
    with pytest.raises(F.FdmtError):
        F.Plan(1200.0, 1600.0, 64, 128, 64, "f32", host_only=True, gamma=0.0)


def test_tables_equal_oracle_random_bands(lib):
    rng = np.random.default_rng(77)
    for _ in range(20):
        f_min = float(rng.uniform(50, 2000))
        f_max = f_min * float(rng.uniform(1.01, 3.0))
        nf = int(2 ** rng.integers(1, 10)) if rng.integers(2) else int(rng.integers(2, 600))
        nd = int(rng.integers(1, 1500))
        p = F.Plan(f_min, f_max, nf, ((nd + 15) // 16) * 16, nd, "f32", host_only=True)
        T = oracle.build_tables(f_min, f_max, nf, nd)
        for l in range(1, T.levels + 1):
            for b in range(len(T.rows[l])):
                assert np.array_equal(p.band_dl(l, b), T.dl[l][b])


def test_search_workspace_and_argument_checks(lib):
    """fdmt_search validates its arguments before any device work."""
    v = ctypes.c_size_t()
    assert lib.fdmt_search_workspace_bytes(1024, 65536, 8, ctypes.byref(v)) == N.OK
    # one (value, time) partial per (row, width, segment); segments of 2^12 samples or a little less
    assert v.value % (1024 * 8 * 12) == 0 and 16 <= v.value // (1024 * 8 * 12) <= 20
    assert lib.fdmt_search_workspace_bytes(3, 4097, 1, ctypes.byref(v)) == N.OK and v.value == 3 * 2 * 12
    for args in ((1024, 65536, 0), (1024, 65536, 14), (0, 64, 3), (4, 0, 3)):
        assert lib.fdmt_search_workspace_bytes(*args, ctypes.byref(v)) == N.ERR_INVALID_ARG, args
    fake = ctypes.c_void_p(1 << 20)
    big = 1 << 40
    assert lib.fdmt_search(None, N.F32_F32, 4, 64, 3, 0, fake, fake, fake, big, None) == N.ERR_INVALID_ARG
    assert lib.fdmt_search(fake, 7, 4, 64, 3, 0, fake, fake, fake, big, None) == N.ERR_INVALID_ARG
    assert lib.fdmt_search(fake, N.F32_F32, 4, 64, 14, 0, fake, fake, fake, big, None) == N.ERR_INVALID_ARG
    assert lib.fdmt_search(fake, N.F32_F32, 4, 1 << 31, 3, 0, fake, fake, fake, big, None) == N.ERR_UNSUPPORTED
    assert lib.fdmt_search(fake, N.F32_F32, 4, 64, 3, 0, fake, fake, fake, 4 * 3 * 12 - 1, None) == N.ERR_WORKSPACE
    assert lib.fdmt_search(fake, N.F32_F32, 4, 64, 3, 0, fake, fake, ctypes.c_void_p((1 << 20) + 4), big,
                           None) == N.ERR_WORKSPACE
    assert lib.fdmt_search(fake, N.U8_I32, 4, 64, 3, 0, fake, fake, None, big, None) == N.ERR_WORKSPACE
    assert lib.fdmt_search(fake, N.U8_I32, 4, 64, 3, -1, fake, fake, fake, big, None) == N.ERR_INVALID_ARG


def test_fft_fdmt_plan_shapes_and_argument_checks(lib):
    """FFT-FDMT plans (section 5) on the host: block, hop, pairs, bins and
    workspace follow from the shape; bad arguments are refused before any
    device work."""
    p = F.FFTPlan(1200.0, 1600.0, 1024, 1 << 16, 1024, "f32", host_only=True)
    assert (p.block, p.hop) == (4096, 4096 - 1023)
    assert p.pairs == -(-(-(-(1 << 16) // p.hop)) // 2) == 11
    # merge state: rows of levels 1 and 2 (1535 + 1279, the input tile in the
    # even buffer), the Option-1 geometric sums and the shift vectors, 8 bytes
    # per bin: four blocks per SM hold 2 bins each
    assert p.bins == 2
    assert p.workspace_bytes == 1024 * 11 * 4096 * 8
    q = F.FFTPlan(1200.0, 1600.0, 16, 100, 20, "u8", host_only=True)
    assert (q.block, q.hop, q.pairs, q.bins) == (256, 237, 1, 2)
    assert F.FFTPlan(1200.0, 1600.0, 6, 1000, 300, block=2048, bins=2, host_only=True).bins == 2
    h = ctypes.c_void_p()
    ok = (1200.0, 1600.0, 64, 4096, 64, N.F32_F32, 0, 0, N.PLAN_HOST_ONLY)
    assert lib.fdmt_fft_plan(*ok, ctypes.byref(h)) == N.OK
    lib.fdmt_fft_destroy(h)
    for i, bad, want in ((5, N.F32_F16STATE, N.ERR_INVALID_ARG), (6, 300, N.ERR_INVALID_ARG),
                         (6, 128, N.ERR_INVALID_ARG), (6, 8192, N.ERR_INVALID_ARG), (7, 3, N.ERR_INVALID_ARG),
                         (7, 16, N.ERR_INVALID_ARG), (8, 1 << 9, N.ERR_INVALID_ARG), (2, 1, N.ERR_INVALID_ARG),
                         (4, 0, N.ERR_INVALID_ARG), (3, 0, N.ERR_INVALID_ARG), (1, 1000.0, N.ERR_INVALID_ARG)):
        args = list(ok)
        args[i] = bad
        assert lib.fdmt_fft_plan(*args, ctypes.byref(h)) == want, (i, bad)
    # Nd - 1 >= block: no output column per block
    assert lib.fdmt_fft_plan(1200.0, 1600.0, 64, 4096, 257, N.F32_F32, 256, 0, N.PLAN_HOST_ONLY,
                             ctypes.byref(h)) == N.ERR_UNSUPPORTED
    assert lib.fdmt_fft_plan(1200.0, 1600.0, 64, 4096, 5000, N.F32_F32, 0, 0, N.PLAN_HOST_ONLY,
                             ctypes.byref(h)) == N.ERR_UNSUPPORTED
    # large-4k: state rows of two levels exceed shared memory even at one bin
    assert lib.fdmt_fft_plan(1100.0, 1700.0, 4096, 1 << 20, 4096, N.F32_F32, 0, 0, N.PLAN_HOST_ONLY,
                             ctypes.byref(h)) == N.ERR_UNSUPPORTED
    assert lib.fdmt_fft_plan(*ok, None) == N.ERR_INVALID_ARG
    v = ctypes.c_size_t()
    assert lib.fdmt_fft_workspace_bytes(None, ctypes.byref(v)) == N.ERR_INVALID_ARG
    assert lib.fdmt_fft_info(None, None, None, None, None) == N.ERR_INVALID_ARG
    assert lib.fdmt_fft_execute(None, None, None, None, 0, None) == N.ERR_INVALID_ARG
    assert lib.fdmt_fft_plan(*ok, ctypes.byref(h)) == N.OK
    fake = ctypes.c_void_p(1 << 20)
    assert lib.fdmt_fft_execute(h, fake, fake, fake, 1 << 40, None) == N.ERR_INVALID_ARG  # host-only plan
    lib.fdmt_fft_destroy(h)
    lib.fdmt_fft_destroy(None)  # NULL-safe
    with pytest.raises(ValueError):
        F.FFTPlan(1200.0, 1600.0, 64, 4096, 64, "f16state", host_only=True)
    with pytest.raises(F.FdmtError):
        F.FFTPlan(1200.0, 1600.0, 64, 4096, 64, bins=3, host_only=True)


def test_stream_argument_checks(lib):
    """fdmt_stream_create checks the shape on the host before allocating."""
    h = ctypes.c_void_p()
    args = (1200.0, 1600.0, 64, 1024, 64, N.F32_F32, 0)
    assert lib.fdmt_stream_create(*args[:3], 1000, *args[4:], ctypes.byref(h)) == N.ERR_INVALID_ARG  # chunk % 16
    assert lib.fdmt_stream_create(*args[:3], 0, *args[4:], ctypes.byref(h)) == N.ERR_INVALID_ARG
    assert lib.fdmt_stream_create(1200.0, 1600.0, 64, 1024, 0, N.F32_F32, 0, ctypes.byref(h)) == N.ERR_INVALID_ARG
    assert lib.fdmt_stream_create(1200.0, 1600.0, 64, 1024, 64, 9, 0, ctypes.byref(h)) == N.ERR_INVALID_ARG
    assert lib.fdmt_stream_create(*args[:6], N.PLAN_HOST_ONLY, ctypes.byref(h)) == N.ERR_INVALID_ARG
    assert lib.fdmt_stream_create(*args, None) == N.ERR_INVALID_ARG
    assert lib.fdmt_stream_push(None, None, None, None) == N.ERR_INVALID_ARG
    assert lib.fdmt_stream_reset(None, None) == N.ERR_INVALID_ARG
    assert lib.fdmt_stream_info(None, None, None) == N.ERR_INVALID_ARG
    lib.fdmt_stream_destroy(None)  # NULL-safe


@pytest.mark.parametrize("f_min,f_max,nf,d_min,gamma", [
    (1200.0, 1600.0, 64, 200, -2.0), (1200.0, 1600.0, 1024, 3000, -2.0), (1100.0, 1700.0, 4096, 12345, -2.0),
    (1024.0, 2048.0, 64, 100, 1.0), (300.0, 310.0, 512, 77, -2.0), (100.0, 900.0, 128, 999, -1.5)])
def test_input_shifts_equal_oracle(lib, f_min, f_max, nf, d_min, gamma):
    p = F.Plan(f_min, f_max, nf, 4096, 64, "f32", host_only=True, d_min=d_min, gamma=gamma)
    s, desc = p.input_map()
    assert not desc
    assert np.array_equal(s, oracle.input_shifts(f_min, f_max, nf, d_min, gamma))
    q = F.Plan(f_min, f_max, nf, 4096, 64, "f32", host_only=True, descending=True)
    s0, desc = q.input_map()
    assert desc and not s0.any()


def test_mapped_plan_workspace(lib):
    base = F.Plan(1200, 1600, 1024, 65536, 1024, "u8", host_only=True)
    m = F.Plan(1200, 1600, 1024, 65536, 1024, "u8", host_only=True, d_min=500)
    # the mapped input follows the schedule's own workspace
    assert m.workspace_bytes == -(-base.workspace_bytes // 256) * 256 + 1024 * 65536
    f = F.Plan(1200, 1600, 1024, 65536, 1024, "f32", host_only=True, descending=True)
    fb = F.Plan(1200, 1600, 1024, 65536, 1024, "f32", host_only=True)
    assert f.adjoint_workspace_bytes == fb.adjoint_workspace_bytes + 2 * 1024 * 65536 * 4
    h = ctypes.c_void_p()
    for d_min, desc in ((-1, 0), ((1 << 30) + 1, 0), (0, 2)):
        cp = N.CurveParams(-2.0, d_min, desc)
        assert lib.fdmt_plan_curve(1200.0, 1600.0, 64, 1024, 64, N.F32_F32, N.PLAN_HOST_ONLY, ctypes.byref(cp),
                                   None, ctypes.byref(h)) == N.ERR_INVALID_ARG


def test_filterbank_argument_checks(lib):
    fake = ctypes.c_void_p(1 << 20)
    assert lib.fdmt_filterbank(None, 1024, 64, 1, fake, 16, None) == N.ERR_INVALID_ARG
    assert lib.fdmt_filterbank(ctypes.c_void_p((1 << 20) + 8), 1024, 64, 1, fake, 16, None) == N.ERR_INVALID_ARG
    assert lib.fdmt_filterbank(fake, 1024, 48, 1, fake, 16, None) == N.ERR_INVALID_ARG   # nf not 2^k
    assert lib.fdmt_filterbank(fake, 1024, 8192, 1, fake, 1, None) == N.ERR_INVALID_ARG  # nf > 4096
    assert lib.fdmt_filterbank(fake, 1024, 64, 1, fake, 17, None) == N.ERR_INVALID_ARG   # nt > n / nf
    assert lib.fdmt_filterbank(fake, 1024, 64, 0, fake, 16, None) == N.ERR_INVALID_ARG
    assert lib.fdmt_filterbank(fake, 1 << 30, 4096, 64, fake, 16, None) == N.ERR_UNSUPPORTED  # bin too big


def test_pipeline_and_shape_argument_checks(lib):
    h = ctypes.c_void_p()
    assert lib.fdmt_pipeline_create(None, ctypes.byref(h)) == N.ERR_INVALID_ARG
    assert lib.fdmt_pipeline_push(None, None, None) == N.ERR_INVALID_ARG
    assert lib.fdmt_pipeline_wait(None) == N.ERR_INVALID_ARG
    lib.fdmt_pipeline_destroy(None)  # NULL-safe
    p = F.Plan(1200.0, 1600.0, 64, 1024, 40, "u8", host_only=True)
    nf, nt, nd, dt = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
    assert lib.fdmt_plan_shape(p._h, ctypes.byref(nf), ctypes.byref(nt), ctypes.byref(nd), ctypes.byref(dt)) == N.OK
    assert (nf.value, nt.value, nd.value, dt.value) == (64, 1024, 40, N.U8_I32)
    assert lib.fdmt_plan_shape(None, None, None, None, None) == N.ERR_INVALID_ARG
