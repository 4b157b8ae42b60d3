"""CPU checks of the fused adjoint's planner (no GPU).

The pull-cone tables of host-only fused plans are run by the emulator in
tests/adjoint_emulator.py (NaN-filled shared memory, region checks, every
output written exactly once); on small-integer gradients the result must
equal the float64 oracle adjoint exactly.  Full-size plans get the static
table checks.
"""
import numpy as np
import pytest

import filterbank_synth as fs
import oracle
import paper_1411_5373_gb300 as FD
from adjoint_emulator import AdjointTableError, check_adjoint_tables, emulate_adjoint

CASES = [
    ((1200.0, 1600.0, 16, 256, 16), {}),
    ((1200.0, 1600.0, 64, 512, 64), {}),
    ((1200.0, 1600.0, 64, 512, 64), {"adjoint_tile": 64, "adjoint_bounds": [0, 1, 2, 4, 6]}),
    ((1200.0, 1600.0, 64, 448, 100), {"adjoint_tile": 128, "adjoint_bounds": [0, 3, 6]}),
    ((1200.0, 1600.0, 128, 640, 150), {"adjoint_tile": 192, "adjoint_smem_budget": 32 * 1024}),
    ((1200.0, 1600.0, 2, 64, 1), {}),
    ((1200.0, 1600.0, 3, 64, 7), {}),
    ((1200.0, 1600.0, 48, 1024, 64), {}),
    ((1200.0, 1600.0, 100, 512, 90), {"adjoint_tile": 128, "adjoint_smem_budget": 40 * 1024}),
    ((1300.0, 1450.0, 257, 640, 140), {"adjoint_tile": 64}),
]


@pytest.mark.parametrize("shape,kw", CASES)
def test_emulated_fused_adjoint_equals_oracle(shape, kw):
    f0, f1, nf, nt, nd = shape
    p = FD.Plan(f0, f1, nf, nt, nd, "f32", schedule="fused", host_only=True, adjoint="fused", **kw)
    T = oracle.build_tables(f0, f1, nf, nd)
    g = fs.small_ints(31, (nd, nt)).astype(np.float32)
    got = emulate_adjoint(p, g)
    assert np.array_equal(got, oracle.fdmt_adjoint(g.astype(np.float64), T).astype(np.float32))
    assert check_adjoint_tables(p) > 0
    groups = p.fused_table(10).reshape(-1, 15)
    assert groups[-1, 1] == 0 and groups[-1, 2] == 1       # ends at level 0 with the init transpose
    assert groups[0, 0] == p.levels
    if "adjoint_bounds" in kw:
        b = kw["adjoint_bounds"]
        assert [int(r[0]) for r in groups] == b[:0:-1] and [int(r[1]) for r in groups] == b[-2::-1]


def test_emulated_fused_adjoint_weights():
    f0, f1, nf, nt, nd = 1200.0, 1600.0, 32, 320, 40
    p = FD.Plan(f0, f1, nf, nt, nd, "f32", schedule="fused", host_only=True, adjoint="fused", adjoint_tile=64)
    T = oracle.build_tables(f0, f1, nf, nd)
    g = fs.small_ints(32, (nd, nt)).astype(np.float32)
    w = np.arange(1, nf + 1, dtype=np.float32)  # integers: the products stay exact
    got = emulate_adjoint(p, g, w)
    assert np.array_equal(got, (oracle.fdmt_adjoint(g.astype(np.float64), T) * w[:, None]).astype(np.float32))


def test_plain_adjoint_option_and_uint8():
    p = FD.Plan(1200.0, 1600.0, 64, 512, 64, "f32", schedule="fused", host_only=True, adjoint="plain")
    assert len(p.fused_table(10)) == 0
    q = FD.Plan(1200.0, 1600.0, 64, 512, 64, "u8", schedule="fused", host_only=True)
    assert len(q.fused_table(10)) == 0          # the adjoint is float-only
    r = FD.Plan(1200.0, 1600.0, 64, 512, 64, "f32", schedule="plain", host_only=True)
    assert len(r.fused_table(10)) == 0
    with pytest.raises(AdjointTableError):
        emulate_adjoint(p, np.zeros((64, 512), np.float32))


def test_fused_adjoint_is_the_default_of_fused_float_plans():
    p = FD.Plan(1200.0, 1600.0, 64, 512, 64, "f32", schedule="fused", host_only=True)
    assert len(p.fused_table(10)) > 0
    q = FD.Plan(1200.0, 1600.0, 64, 512, 64, "f16state", schedule="fused", host_only=True)
    assert len(q.fused_table(10)) > 0


def test_adjoint_parameters_need_the_fused_adjoint():
    with pytest.raises(FD.FdmtError):
        FD.Plan(1200.0, 1600.0, 64, 512, 64, "f32", schedule="fused", host_only=True, adjoint="plain",
                adjoint_tile=128)


def test_invalid_adjoint_parameters():
    for kw in ({"adjoint_tile": 100}, {"adjoint_bounds": [0, 3, 2, 6]}, {"adjoint_bounds": [1, 6]},
               {"adjoint_smem_budget": 4096, "adjoint_tile": 64}):
        with pytest.raises(FD.FdmtError):
            FD.Plan(1200.0, 1600.0, 64, 512, 64, "f32", schedule="fused", host_only=True, adjoint="fused", **kw)


@pytest.mark.parametrize("shape", [(1200.0, 1600.0, 1024, 65536, 1024), (1200.0, 1600.0, 1000, 65536, 1000),
                                   (1100.0, 1700.0, 4096, 1 << 20, 4096)])
def test_full_size_adjoint_tables(shape):
    p = FD.Plan(*shape, "f32", schedule="fused", host_only=True, adjoint="fused")
    assert check_adjoint_tables(p) > 0


def test_folded_initialisation_transpose():
    """A last launch over two levels or more folds the level 1 -> 0 gather
    into the transpose (stage kind 3, no level-0 region, three times the
    tile by default); one over a single level keeps the two stages."""
    p = FD.Plan(1200.0, 1600.0, 1024, 65536, 1024, "f32", schedule="fused", host_only=True, adjoint="fused")
    groups = p.fused_table(10).reshape(-1, 15)
    last = groups[-1]
    assert last[1] == 0 and last[2] == 1 and last[0] >= 2 and last[3] == 3 * 512
    stages = p.fused_table(14).reshape(-1, 10)
    tpls = p.fused_table(11).reshape(-1, 8)
    first, count = int(last[5]), int(last[6])
    for t in tpls[first:first + count]:
        kinds = [int(stages[t[4] // 10 + s, 0]) for s in range(t[5])]
        assert kinds == [1] * (int(last[0]) - 1) + [3]
    q = FD.Plan(1200.0, 1600.0, 64, 512, 64, "f32", schedule="fused", host_only=True, adjoint="fused",
                adjoint_tile=64, adjoint_bounds=[0, 1, 2, 4, 6])
    qs = q.fused_table(14).reshape(-1, 10)[:, 0]
    assert 3 not in qs.tolist() and 2 in qs.tolist()


def test_unfolded_transpose_for_channels_with_many_rows():
    """Channels with more than 7 level-0 rows (few channels, many delays)
    keep the level 1 -> 0 gather and the transpose as two stages, and the
    emulated tables still equal the oracle's adjoint."""
    f0, f1, nf, nt, nd = 1200.0, 1600.0, 8, 256, 64
    p = FD.Plan(f0, f1, nf, nt, nd, "f32", schedule="fused", host_only=True, adjoint="fused")
    assert int(p.band_rows(0).max()) > 7
    kinds = set(p.fused_table(14).reshape(-1, 10)[:, 0].tolist())
    assert 2 in kinds and 3 not in kinds
    T = oracle.build_tables(f0, f1, nf, nd)
    g = fs.small_ints(31, (nd, nt)).astype(np.float32)
    got = emulate_adjoint(p, g)
    assert np.array_equal(got, oracle.fdmt_adjoint(g.astype(np.float64), T).astype(np.float32))
    assert check_adjoint_tables(p) > 0
