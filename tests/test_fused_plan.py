"""CPU checks of the fused schedule's planner (no GPU).

The cone tables a host-only fused plan exposes are executed by a byte-level
emulator (tests/fused_emulator.py) with bounds and alignment checks on every
shared-memory access and TMA copy; the result must equal the oracle bit for
bit.  Forced schedules (one level per launch, tiny tiles, tiny shared-memory
budgets that force row splits) exercise every branch of the planner.
"""
import numpy as np
import pytest

import filterbank_synth as fs
import oracle
import paper_1411_5373_gb300 as FD
from fused_emulator import check_bounds, emulate


def _run(nf, nt, nd, dtype, seed=3, weights=None, **sched):
    p = FD.Plan(1200.0, 1600.0, nf, nt, nd, dtype, schedule="fused", host_only=True, **sched)
    x = fs.random_u8(seed, nf, nt) if dtype == "u8" else fs.random_f32(seed, nf, nt)
    T = oracle.build_tables(1200.0, 1600.0, nf, nd)
    got = emulate(p, x, weights)
    mode = {"u8": "i64", "f32": "f32", "f16state": "f16state"}[dtype]
    want = oracle.fdmt(x, T, mode, weights=weights)
    return p, got, want


CASES = [
    # nf, nt, nd, dtype, schedule parameters
    (16, 256, 16, "f32", {}),
    (16, 256, 16, "u8", {}),
    (32, 320, 50, "f32", {"tile": 64}),
    (32, 320, 50, "u8", {"tile": 64, "bounds": [0, 1, 2, 3, 4, 5]}),
    (32, 320, 50, "f16state", {"tile": 128, "bounds": [0, 2, 5]}),
    (64, 448, 64, "f32", {"tile": 64, "smem_budget": 24 * 1024}),
    (64, 448, 100, "u8", {"tile": 128, "smem_budget": 20 * 1024, "bounds": [0, 3, 6]}),
    (8, 192, 150, "f32", {"tile": 64, "smem_budget": 16 * 1024}),
    (2, 64, 1, "f32", {}),
    (4, 128, 6, "u8", {"tile": 64}),
    (128, 512, 40, "f16state", {"tile": 64, "bounds": [0, 4, 7]}),
]


@pytest.mark.parametrize("nf,nt,nd,dtype,sched", CASES)
def test_emulated_fused_schedule_equals_oracle(nf, nt, nd, dtype, sched):
    p, got, want = _run(nf, nt, nd, dtype, **sched)
    assert np.array_equal(got, want), np.argwhere(got != want)[:5]
    tile, bounds = p.schedule_info()
    if "tile" in sched:
        assert tile == sched["tile"]
    if "bounds" in sched:
        assert bounds == sched["bounds"]


@pytest.mark.parametrize("staging", ["boxes", "blocks"])
@pytest.mark.parametrize("nf,nt,nd,dtype,sched", [c for c in CASES if c[1] % 64 == 0 and c[1] >= 256])
def test_emulated_staging_formats(nf, nt, nd, dtype, sched, staging):
    """Both ways of copying staged rows (row boxes through a 2-D map, row
    blocks of 2^p rows through a 3-D chunked map) give the oracle's result."""
    p, got, want = _run(nf, nt, nd, dtype, staging=staging, **sched)
    assert np.array_equal(got, want), np.argwhere(got != want)[:5]
    chunk = p.fused_table(0).reshape(-1, 16)[:, 11]
    assert (chunk > 0).all() if staging == "blocks" else (chunk == 0).all()


def test_row_blocks_need_whole_chunks():
    # nt = 200 is not a multiple of a 128-byte chunk of float32 samples
    with pytest.raises(FD.FdmtError):
        FD.Plan(1200.0, 1600.0, 16, 200, 16, "f32", schedule="fused", host_only=True, staging="blocks")
    p = FD.Plan(1200.0, 1600.0, 16, 200, 16, "f32", schedule="fused", host_only=True)
    assert (p.fused_table(0).reshape(-1, 16)[:, 11] == 0).all()


@pytest.mark.parametrize("gamma", [-1.0, 1.0, 2.5])
def test_emulated_power_law_curves(gamma):
    """The fused programme of another curve family (Dt ~ f^gamma) equals the
    oracle built with the same gamma."""
    nf, nt, nd = 64, 448, 80
    p = FD.Plan(1200.0, 1600.0, nf, nt, nd, "u8", schedule="fused", host_only=True, tile=64, gamma=gamma)
    x = fs.random_u8(5, nf, nt)
    T = oracle.build_tables(1200.0, 1600.0, nf, nd, gamma=gamma)
    assert np.array_equal(emulate(p, x), oracle.fdmt(x, T, "i64"))


def test_emulated_fused_with_weights():
    w = np.random.default_rng(2).uniform(0.2, 1.8, 32).astype(np.float32)
    _, got, want = _run(32, 320, 40, "f32", weights=w, tile=64, bounds=[0, 2, 5])
    assert np.array_equal(got, want)


def test_row_splits_happen_under_small_budget():
    p = FD.Plan(1200.0, 1600.0, 64, 448, 64, "f32", schedule="fused", host_only=True,
                tile=64, smem_budget=24 * 1024)
    groups = p.fused_table(0).reshape(-1, 16)
    nb_top = [64 >> int(g[1]) for g in groups]
    assert any(int(g[4]) > nb for g, nb in zip(groups, nb_top)), "expected some bands split into row ranges"
    assert all(int(g[5]) <= 24 * 1024 for g in groups)


def test_headline_schedule_fits_and_models():
    p = FD.Plan(1200.0, 1600.0, 1024, 65536, 1024, "f32", schedule="fused", host_only=True)
    tile, bounds = p.schedule_info()
    assert tile % 64 == 0 and bounds[0] == 0 and bounds[-1] == 10
    groups = p.fused_table(0).reshape(-1, 16)
    assert all(int(g[5]) <= 112 * 1024 for g in groups)
    # fewer passes over HBM than one launch per level
    assert len(groups) < 10


def test_invalid_schedule_parameters():
    with pytest.raises(FD.FdmtError):
        FD.Plan(1200.0, 1600.0, 64, 1024, 64, "f32", schedule="fused", host_only=True, tile=100)
    with pytest.raises(FD.FdmtError):
        FD.Plan(1200.0, 1600.0, 64, 1024, 64, "f32", schedule="fused", host_only=True,
                bounds=[0, 3, 2, 6])
    with pytest.raises(FD.FdmtError):  # nothing fits a 1 KiB budget
        FD.Plan(1200.0, 1600.0, 64, 1024, 64, "f32", schedule="fused", host_only=True,
                smem_budget=1024)


@pytest.mark.parametrize("nf,nt,nd,dtype,sched", [
    (1024, 65536, 1024, "f32", {}),
    (1024, 65536, 1024, "u8", {}),
    (1024, 65536, 1024, "f16state", {}),
    (1024, 65536, 1024, "f32", {"bounds": [0, 3, 6, 10], "tile": 512}),
    (1024, 65536, 1024, "f32", {"bounds": [0, 2, 4, 6, 8, 10], "tile": 256}),
    (4096, 1 << 20, 4096, "f32", {"bounds": [0, 3, 6, 9, 12], "tile": 512}),
    (256, 1 << 14, 2048, "u8", {}),
])
def test_full_size_plans_stay_in_shared_memory(nf, nt, nd, dtype, sched):
    """Every descriptor of a full-size plan (the benchmark shapes) stays
    inside its launch's shared memory and regions (static check; the
    emulator covers the values at small sizes)."""
    p = FD.Plan(1200.0, 1600.0, nf, nt, nd, dtype, schedule="fused", host_only=True, **sched)
    assert check_bounds(p) > 0


@pytest.mark.parametrize("nf,nt,nd,dtype,k,sched", [
    (16, 512, 16, "f32", 1, {}),
    (16, 512, 16, "u8", 5, {"tile": 128}),
    (32, 640, 50, "f32", 8, {"tile": 128, "bounds": [0, 3, 5]}),
    (32, 640, 50, "u8", 9, {"tile": 256, "bounds": [0, 2, 5]}),
    (64, 960, 64, "f16state", 6, {"tile": 64, "smem_budget": 48 * 1024}),
    (64, 1040, 90, "f32", 7, {"tile": 256, "bounds": [0, 3, 4, 6]}),
    (8, 512, 20, "u8", 3, {"tile": 64}),
])
def test_emulated_search_epilogue_equals_oracle(nf, nt, nd, dtype, k, sched):
    """A plan whose last launch ends with the boxcar search: the emulated
    launches and the partials' finalize give the oracle's transform, peaks
    and first times, bit for bit."""
    from fused_emulator import emulate_search
    p = FD.Plan(1200.0, 1600.0, nf, nt, nd, dtype, schedule="fused", host_only=True, search_widths=k, **sched)
    x = fs.random_u8(11, nf, nt) if dtype == "u8" else fs.random_f32(11, nf, nt)
    T = oracle.build_tables(1200.0, 1600.0, nf, nd)
    mode = {"u8": "i64", "f32": "f32", "f16state": "f16state"}[dtype]
    want = oracle.fdmt(x, T, mode)
    A, peak, when = emulate_search(p, x, k)
    assert np.array_equal(A, want)
    rp, rt = oracle.boxcar_search(want.astype(np.int32) if dtype == "u8" else want, k)
    assert np.array_equal(peak, rp)
    assert np.array_equal(when, rt)
    check_bounds(p)


@pytest.mark.parametrize("nf,nt,nd,dtype,sched", [
    (3, 256, 12, "f32", {"tile": 64}),
    (3, 256, 12, "u8", {"tile": 64, "bounds": [0, 1, 2]}),
    (48, 448, 60, "f32", {"tile": 64}),
    (48, 448, 60, "u8", {"tile": 128, "bounds": [0, 1, 3, 6]}),
    (100, 512, 90, "f32", {"tile": 64, "smem_budget": 40 * 1024}),
    (100, 512, 90, "f16state", {"tile": 128, "bounds": [0, 2, 4, 7]}),
    (257, 640, 140, "u8", {"tile": 64}),
    (257, 640, 140, "f32", {"tile": 128, "bounds": [0, 3, 6, 9]}),
    (1000, 1024, 200, "u8", {"tile": 128}),
    (5, 192, 40, "f32", {"tile": 64, "bounds": [0, 1, 2, 3]}),
    (7, 256, 30, "u8", {"tile": 64, "bounds": [0, 3]}),
])
def test_emulated_fused_unequal_bands(nf, nt, nd, dtype, sched):
    """Nf not a power of two: the last band of a level is short and bands
    without an upper half pass their rows up unchanged; the emulated cones
    equal the oracle bit for bit and stay in bounds."""
    p, got, want = _run(nf, nt, nd, dtype, **sched)
    assert np.array_equal(got, want), np.argwhere(got != want)[:5]
    check_bounds(p)


@pytest.mark.parametrize("nf,nt,nd,dtype,k,sched", [
    (48, 640, 60, "f32", 6, {"tile": 128}),
    (100, 960, 90, "u8", 8, {"tile": 256, "bounds": [0, 3, 7]}),
])
def test_emulated_search_unequal_bands(nf, nt, nd, dtype, k, sched):
    from fused_emulator import emulate_search
    p = FD.Plan(1200.0, 1600.0, nf, nt, nd, dtype, schedule="fused", host_only=True, search_widths=k, **sched)
    x = fs.random_u8(13, nf, nt) if dtype == "u8" else fs.random_f32(13, nf, nt)
    T = oracle.build_tables(1200.0, 1600.0, nf, nd)
    want = oracle.fdmt(x, T, "i64" if dtype == "u8" else "f32")
    A, peak, when = emulate_search(p, x, k)
    assert np.array_equal(A, want)
    rp, rt = oracle.boxcar_search(want.astype(np.int32) if dtype == "u8" else want, k)
    assert np.array_equal(peak, rp) and np.array_equal(when, rt)
