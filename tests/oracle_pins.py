"""Pins of the CPU oracle: checks against what the paper and the mathematics
fix, not against the oracle itself.

Each pin takes the oracle module ``O`` as an argument so the same checks run
on the real oracle (tests/test_oracle_pins.py) and on copies with planted
mistakes (tests/test_oracle_mutations.py), which must fail at least one pin.
Every pin raises AssertionError on a violation.
"""
from __future__ import annotations

import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "nf4_worked_example.txt")


def _r(f_min, f_max, f):
    """Ideal delay fraction of the f^-2 law (Eq. DtD), written independently."""
    a = 1.0 / f_min ** 2
    return (a - 1.0 / f ** 2) / (a - 1.0 / f_max ** 2)


def _edges(f_min, f_max, nf):
    return [f_min + (f_max - f_min) * k / nf for k in range(nf + 1)]


def _shift(x, s):
    y = np.zeros_like(x)
    if s < x.shape[-1]:
        y[..., s:] = x[..., : x.shape[-1] - s]
    return y


def parse_golden(path=GOLDEN):
    g = {"rows": {}, "dl": {}, "offsets": {}, "values": []}
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            head, _, tail = line.partition(":")
            parts = head.split()
            nums = [int(v) for v in tail.split()]
            if parts[0] == "rows":
                g["rows"][int(parts[1])] = nums
            elif parts[0] == "dl":
                g["dl"][(int(parts[1]), int(parts[2]))] = nums
            elif parts[0] == "offsets":
                g["offsets"][int(parts[1])] = nums
            elif parts[0] == "value":
                g["values"].append((int(parts[1]), int(parts[2]), nums[0]))
    return g


# --------------------------------------------------------------------------
# Tables


def pin_golden_tables(O):
    """The hand-worked Nf=4 example (tests/golden): row extents, dl tables and
    curve offsets derived by hand from Eq. (C_{f2,f0}) and the addition rule."""
    g = parse_golden()
    T = O.build_tables(1.0, 2.0, 4, 6)
    for l, rows in g["rows"].items():
        assert list(T.rows[l]) == rows, (l, T.rows[l], rows)
    for (l, b), dl in g["dl"].items():
        assert list(int(v) for v in T.dl[l][b]) == dl, (l, b)
    for d, off in g["offsets"].items():
        assert list(int(v) for v in O.curve_offsets(T, d)) == off, d


def pin_golden_values(O):
    """Hand sums of the worked example, and a brute force over the hand
    offsets (no oracle tables involved) for the whole output."""
    g = parse_golden()
    T = O.build_tables(1.0, 2.0, 4, 6)
    nt = 8
    I = np.array([[t + 1 + 10 * k for t in range(nt)] for k in range(4)], dtype=np.int64)
    A = O.fdmt(I, T, "i64")
    for d, t, v in g["values"]:
        assert int(A[d, t]) == v, (d, t, int(A[d, t]), v)
    B = np.zeros((6, nt), dtype=np.int64)
    for d, off in g["offsets"].items():
        for k in range(4):
            for o in range(off[k], off[k + 1] + 1):
                B[d] += _shift(I[k], o)
    assert np.array_equal(A, B)


def pin_offsets_follow_dispersion_law(O):
    """Curve offsets are monotone, start at 0, end at d, and stay within a
    rounding bound of the ideal f^-2 curve d * r(e_k).  At the whole band's
    merge point the offset is the ideal delay rounded half up (one rounding).

    Bound: each level adds at most 1/2 sample of rounding to the split point
    and shrinks inherited error by the split fraction, so every edge is
    within L/2 + 1/2 of the ideal delay (L = log2 Nf)."""
    for (f_min, f_max, nf, nd) in [(1200.0, 1600.0, 64, 64), (1200.0, 1600.0, 256, 300),
                                   (1100.0, 1700.0, 128, 512), (1.0, 3.0, 32, 20),
                                   (1200.0, 1600.0, 96, 80), (1200.0, 1600.0, 37, 50)]:
        T = O.build_tables(f_min, f_max, nf, nd)
        L = (nf - 1).bit_length()
        e = _edges(f_min, f_max, nf)
        for d in range(nd):
            o = O.curve_offsets(T, d)
            assert o[0] == 0 and o[nf] == d
            assert np.all(np.diff(o) >= 0)
            ideal = np.array([d * _r(f_min, f_max, f) for f in e])
            assert np.max(np.abs(o - ideal)) <= 0.5 * L + 0.5 + 1e-9, (nf, d)
            m = 1 << (L - 1)  # the whole band's merge point (border after 2^(L-1) channels)
            mid = d * _r(f_min, f_max, e[m])
            assert abs(o[m] - mid) <= 0.5 + 1e-9
            assert o[m] == math.floor(mid + 0.5) or abs(mid - round(mid) - 0.5) < 1e-9


def pin_row_extents(O):
    """Every sub-band holds exactly the rows its parent reads: the level-0
    sweeps of all channels telescope to Nd - 1, the last level has Nd rows,
    and the c1/c2 extents match the counts from the f^-2 law."""
    for (f_min, f_max, nf, nd) in [(1200.0, 1600.0, 64, 64), (1200.0, 1600.0, 1024, 1024),
                                   (1200.0, 1600.0, 256, 2048), (1.0, 2.0, 2, 1)]:
        T = O.build_tables(f_min, f_max, nf, nd)
        assert T.rows[T.levels] == [nd]
        assert sum(r - 1 for r in T.rows[0]) == nd - 1
        for l in range(T.levels):
            assert all(r >= 1 for r in T.rows[l])
    T = O.build_tables(1200.0, 1600.0, 64, 64)
    assert [T.level_rows(l) for l in range(7)] == [127, 95, 79, 71, 67, 65, 64]


def pin_scale_invariance(O):
    """Only ratios of f^-2 enter (Eq. DtD): scaling both band edges by a power
    of two (exact in FP64) leaves every table unchanged."""
    T = O.build_tables(1200.0, 1600.0, 128, 200)
    for lam in (0.25, 2.0, 1024.0):
        U = O.build_tables(1200.0 * lam, 1600.0 * lam, 128, 200)
        assert U.rows == T.rows
        for l in range(1, T.levels + 1):
            for b in range(len(T.dl[l])):
                assert np.array_equal(U.dl[l][b], T.dl[l][b])


def pin_power_law_curves(O):
    """Other functional forms Dt ~ f^gamma (section 4.2) change only C.
    gamma = 1 with edges exact in FP64 makes every merge split the band in
    half (C = 1/2 exactly), so dl = floor(Dt/2 + 1/2) at every level; any
    gamma keeps the offsets monotone and within the rounding bound of the
    ideal f^gamma curve; gamma = -2 reproduces the default tables."""
    T = O.build_tables(1024.0, 2048.0, 64, 90, gamma=1.0)
    for l in range(1, T.levels + 1):
        for b in range(len(T.dl[l])):
            dt = np.arange(len(T.dl[l][b]))
            assert np.array_equal(T.dl[l][b], (dt + 1) // 2), (l, b)
    for gamma in (-1.0, 0.5, 1.5, 3.0):
        f_min, f_max, nf, nd = 1200.0, 1600.0, 64, 70
        T = O.build_tables(f_min, f_max, nf, nd, gamma=gamma)
        L = int(math.log2(nf))
        e = _edges(f_min, f_max, nf)
        r = [(f_min ** gamma - f ** gamma) / (f_min ** gamma - f_max ** gamma) for f in e]
        for d in range(nd):
            o = O.curve_offsets(T, d)
            assert o[0] == 0 and o[nf] == d and np.all(np.diff(o) >= 0)
            assert np.max(np.abs(o - d * np.array(r))) <= 0.5 * L + 0.5 + 1e-9, (gamma, d)
    A = O.build_tables(1200.0, 1600.0, 32, 40)
    B = O.build_tables(1200.0, 1600.0, 32, 40, gamma=-2.0)
    assert A.rows == B.rows


# --------------------------------------------------------------------------
# Transform


def pin_bruteforce_exhaustive(O):
    """Recursion (Algorithm 1) equals the direct sum of Eq. "parametrization"
    along the unrolled curves, on integers, for every small Nf and many Nd."""
    rng = np.random.default_rng(1411)
    for nf in (2, 4, 8, 16, 32):
        for nd in sorted({1, 2, 3, nf - 1, nf, nf + 1, 2 * nf} - {0}):
            nt = int(rng.integers(max(nd, 2), 3 * nd + 40))
            T = O.build_tables(1200.0, 1600.0, nf, nd)
            I = rng.integers(-50, 50, size=(nf, nt))
            assert np.array_equal(O.fdmt(I, T, "i64"), O.bruteforce(I, T, np.int64)), (nf, nd)
    for nf in (3, 5, 6, 7, 12, 13, 24):  # Nf not a power of two (section 4.2)
        for nd in sorted({1, 2, nf - 1, nf, 2 * nf + 1} - {0}):
            nt = int(rng.integers(max(nd, 2), 3 * nd + 40))
            T = O.build_tables(1200.0, 1600.0, nf, nd)
            I = rng.integers(-50, 50, size=(nf, nt))
            assert np.array_equal(O.fdmt(I, T, "i64"), O.bruteforce(I, T, np.int64)), (nf, nd)
    for gamma in (-1.0, 1.0, 2.5):  # other curve families (section 4.2)
        for nf, nd in ((8, 11), (16, 16), (32, 7)):
            T = O.build_tables(1200.0, 1600.0, nf, nd, gamma=gamma)
            I = rng.integers(-50, 50, size=(nf, nd + 30))
            assert np.array_equal(O.fdmt(I, T, "i64"), O.bruteforce(I, T, np.int64)), (gamma, nf, nd)


def pin_channel_sum(O):
    """Row d = 0 is the plain sum over channels (no dispersion)."""
    rng = np.random.default_rng(7)
    for nf, nd in ((8, 8), (64, 40), (5, 9), (100, 40)):
        T = O.build_tables(1200.0, 1600.0, nf, nd)
        I = rng.integers(0, 256, size=(nf, 96))
        A = O.fdmt(I, T, "i64")
        assert np.array_equal(A[0], I.sum(axis=0))


def pin_constant_input(O):
    """Constant input c: every curve covers Nf + d samples (each channel's
    sweep plus the shared edge samples), so A[d][t] = c (Nf + d) once the
    whole curve lies at t >= 0, i.e. for t >= d."""
    for nf, nd in ((16, 16), (32, 50), (64, 64), (3, 7), (20, 33), (96, 64)):
        T = O.build_tables(1200.0, 1600.0, nf, nd)
        c = 3
        A = O.fdmt(np.full((nf, 2 * nd + 8), c, dtype=np.int64), T, "i64")
        for d in range(nd):
            assert np.all(A[d, d:] == c * (nf + d)), d
            assert np.all(A[d, :d] < c * (nf + d))


def pin_impulse_response(O):
    """An impulse at (k, s) appears in row d as a run of ones whose position
    follows the ideal delay of channel k's edges, with Nf + d ones over all
    channels; the run of channel k lies within the dispersion-law bound."""
    nf, nd, nt = 32, 48, 160
    f_min, f_max = 1200.0, 1600.0
    T = O.build_tables(f_min, f_max, nf, nd)
    L = int(math.log2(nf))
    e = _edges(f_min, f_max, nf)
    s = 20
    total = np.zeros(nd, dtype=np.int64)
    for k in range(nf):
        I = np.zeros((nf, nt), dtype=np.int64)
        I[k, s] = 1
        A = O.fdmt(I, T, "i64")
        assert set(np.unique(A)) <= {0, 1}
        for d in range(nd):
            ts = np.nonzero(A[d])[0]
            assert len(ts) >= 1
            assert np.all(np.diff(ts) == 1)           # one contiguous run
            lo = s + d * _r(f_min, f_max, e[k]) - (0.5 * L + 0.5)
            hi = s + d * _r(f_min, f_max, e[k + 1]) + (0.5 * L + 0.5)
            assert ts[0] >= lo - 1e-9 and ts[-1] <= hi + 1e-9, (k, d, ts, lo, hi)
            total[d] += len(ts)
    assert np.array_equal(total, nf + np.arange(nd))


def pin_linearity_and_shift(O):
    """FDMT is linear, and shifting the input by tau shifts the output by tau
    wherever the whole curve stays inside the data (t >= tau + d)."""
    rng = np.random.default_rng(3)
    nf, nd, nt = 16, 24, 128
    T = O.build_tables(1200.0, 1600.0, nf, nd)
    x = rng.integers(-9, 9, size=(nf, nt))
    y = rng.integers(-9, 9, size=(nf, nt))
    Ax, Ay = O.fdmt(x, T, "i64"), O.fdmt(y, T, "i64")
    assert np.array_equal(O.fdmt(3 * x - 2 * y, T, "i64"), 3 * Ax - 2 * Ay)
    tau = 11
    As = O.fdmt(_shift(x, tau), T, "i64")
    for d in range(nd):
        assert np.array_equal(As[d, tau + d:], Ax[d, d:nt - tau])


def pin_flux(O):
    """With the last Nd - 1 input columns zero, every curve lies wholly in
    the output window, so sum_t A[d, t] = sum_k n_k(d) sum_t I[k, t] with
    n_k(d) the samples the curve takes from channel k, and sum_k n_k = Nf + d."""
    rng = np.random.default_rng(5)
    nf, nd, nt = 32, 40, 200
    T = O.build_tables(1200.0, 1600.0, nf, nd)
    I = rng.integers(0, 100, size=(nf, nt))
    I[:, nt - (nd - 1):] = 0
    A = O.fdmt(I, T, "i64")
    S = I.sum(axis=1)
    for d in range(nd):
        n = np.diff(O.curve_offsets(T, d)) + 1
        assert n.sum() == nf + d
        assert A[d].sum() == int((n * S).sum())


def pin_precision(O):
    """float32 (fixed association) is within 1e-5 of the row RMS of float64;
    float16-stored state within 2e-3; integer input is exact in float64."""
    rng = np.random.default_rng(9)
    nf, nd, nt = 64, 64, 512
    T = O.build_tables(1200.0, 1600.0, nf, nd)
    x = rng.standard_normal((nf, nt)).astype(np.float32)
    a64 = O.fdmt(x.astype(np.float64), T, "f64")
    rms = np.sqrt(np.mean(a64 ** 2, axis=1))
    a32 = O.fdmt(x, T, "f32")
    assert a32.dtype == np.float32
    assert np.all(np.max(np.abs(a32 - a64), axis=1) <= 1e-5 * rms)
    a16 = O.fdmt(x, T, "f16state")
    err = np.sqrt(np.mean((a16 - a64) ** 2, axis=1))
    assert np.all(err <= 2e-3 * rms)
    xi = rng.integers(0, 256, size=(nf, nt))
    assert np.array_equal(O.fdmt(xi, T, "f64"), O.fdmt(xi, T, "i64").astype(np.float64))


def pin_f16_state_rounding(O):
    """Where the stored state is rounded: with Nd = 1 every curve is the
    straight d = 0 sum, so the fp16-state result has a closed form: level-0
    rows (the inputs) are stored as fp16, each merge adds in fp32 and stores
    fp16, and only the last merge's sum stays fp32."""
    rng = np.random.default_rng(21)
    h = lambda a: a.astype(np.float16).astype(np.float32)
    x = (1.0 + rng.random((4, 64)) * 1e-3).astype(np.float32)
    T2 = O.build_tables(1200.0, 1600.0, 2, 1)
    assert np.array_equal(O.fdmt(x[:2], T2, "f16state")[0], h(x[0]) + h(x[1]))
    T4 = O.build_tables(1200.0, 1600.0, 4, 1)
    want = h(h(x[0]) + h(x[1])) + h(h(x[2]) + h(x[3]))
    assert np.array_equal(O.fdmt(x, T4, "f16state")[0], want)
    assert not np.array_equal(want, (x[0] + x[1]) + (x[2] + x[3]))


def pin_weights(O):
    """Per-channel weights scale each channel before the transform: with
    weights that are powers of two the result equals the transform of the
    pre-scaled input exactly."""
    rng = np.random.default_rng(4)
    nf, nd, nt = 16, 16, 64
    T = O.build_tables(1200.0, 1600.0, nf, nd)
    x = rng.integers(-20, 20, size=(nf, nt)).astype(np.float32)
    w = (2.0 ** rng.integers(-2, 3, size=nf)).astype(np.float32)
    assert np.array_equal(O.fdmt(x, T, "f32", weights=w), O.fdmt(x * w[:, None], T, "f32"))


# --------------------------------------------------------------------------
# Adjoint


def pin_adjoint_dot(O):
    """<A x, y> = <x, A^T y> exactly for small-integer x, y (all partial sums
    are exact integers in float64)."""
    rng = np.random.default_rng(11)
    for nf, nd, nt in ((8, 8, 40), (32, 45, 100), (64, 64, 130)):
        T = O.build_tables(1200.0, 1600.0, nf, nd)
        x = rng.integers(-2, 3, size=(nf, nt)).astype(np.float64)
        y = rng.integers(-2, 3, size=(nd, nt)).astype(np.float64)
        lhs = float(np.sum(O.fdmt(x, T, "f64") * y))
        rhs = float(np.sum(x * O.fdmt_adjoint(y, T)))
        assert lhs == rhs, (nf, nd, lhs, rhs)


def pin_adjoint_dense(O):
    """A^T equals the transpose of the dense matrix of the forward map,
    assembled column by column from unit impulses (tiny sizes)."""
    rng = np.random.default_rng(12)
    nf, nd, nt = 4, 6, 12
    T = O.build_tables(1.0, 2.0, nf, nd)
    M = np.zeros((nd * nt, nf * nt))
    for k in range(nf):
        for s in range(nt):
            e = np.zeros((nf, nt))
            e[k, s] = 1.0
            M[:, k * nt + s] = O.fdmt(e, T, "f64").ravel()
    y = rng.standard_normal((nd, nt))
    assert np.allclose(O.fdmt_adjoint(y, T).ravel(), M.T @ y.ravel(), rtol=0, atol=1e-12)


def pin_boxcar_search(O):
    """Boxcar search (section 4.2, pulse profile): brute-force window sums
    with zeros before t = 0 and the first maximum; width 1 is the row max;
    float32 sums follow the binary tree ((a0 + a1) + (a2 + a3)); and the
    search commutes with the transform as the paper states (boxcar of the
    output = output of the boxcar-filtered input, exact on integers)."""
    rng = np.random.default_rng(21)
    A = rng.integers(-20, 21, size=(7, 53))
    A[3, 10] = A[3, 40] = 99  # a tie: the first one wins
    peak, time = O.boxcar_search(A, 5)
    for d in range(A.shape[0]):
        for k in range(5):
            w = 1 << k
            sums = [sum(int(A[d, t - i]) for i in range(w) if t - i >= 0) for t in range(A.shape[1])]
            m = max(sums)
            assert peak[d, k] == m and time[d, k] == sums.index(m), (d, k)
    assert time[3, 0] == 10
    big = np.full((1, 8), 2**31 - 1, dtype=np.int32)  # integer sums never wrap
    assert O.boxcar_search(big, 4)[0][0, 3] == 8 * (2**31 - 1)
    X = rng.standard_normal((3, 40)).astype(np.float32)
    pk, tm = O.boxcar_search(X, 3)
    for d in range(3):
        b4 = [((np.float32(X[d, t]) + np.float32(X[d, t - 1] if t >= 1 else 0))
               + (np.float32(X[d, t - 2] if t >= 2 else 0) + np.float32(X[d, t - 3] if t >= 3 else 0)))
              for t in range(40)]
        b4 = np.array(b4, dtype=np.float32)
        assert pk[d, 2] == b4.max() and tm[d, 2] == int(np.argmax(b4))
    T = O.build_tables(1200.0, 1600.0, 16, 20)
    I = rng.integers(0, 30, size=(16, 90))
    for w in (2, 4, 8):
        Iw = sum(_shift(I, i) for i in range(w))
        Aw = sum(_shift(O.fdmt(I, T, "i64"), i) for i in range(w))
        assert np.array_equal(O.fdmt(Iw, T, "i64"), Aw)
        k = w.bit_length() - 1
        assert np.array_equal(O.boxcar_search(O.fdmt(Iw, T, "i64"), 1)[0][:, 0],
                              O.boxcar_search(O.fdmt(I, T, "i64"), k + 1)[0][:, k])


def pin_input_map(O):
    """The d_min pre-shift (section 4.2) and the channel order of the input.

    (1) gamma = 1 on [1024, 2048] with 64 channels makes r(e_k) = k/64
        exactly, so s_k = floor(d_min k / 64 + 1/2) in closed form.
    (2) For the f^-2 law the shifts start at 0, never decrease and stay
        <= d_min, and the combined offsets s_k + o_k(d) of row d stay within
        L/2 + 1 samples of the ideal curve of total delay d_min + d: row d
        follows delay d_min + d.
    (3) An impulse in raw channel k at time u lands in row d exactly at
        u + s_k + [o_k(d), o_{k+1}(d)].
    (4) d_min = 0 with ascending rows is the identity; descending rows give
        the same transform input as the same channels in ascending rows.
    (5) <M x, g> = <x, M^T g> exactly on integers (the adjoint map)."""
    s = O.input_shifts(1024.0, 2048.0, 64, 100, gamma=1.0)
    assert [int(v) for v in s] == [(100 * k + 32) // 64 for k in range(64)]
    for (f_min, f_max, nf, nd, d_min) in [(1200.0, 1600.0, 64, 64, 200), (1100.0, 1700.0, 128, 100, 777)]:
        s = O.input_shifts(f_min, f_max, nf, d_min)
        assert s[0] == 0 and np.all(np.diff(s) >= 0) and s[-1] <= d_min
        T = O.build_tables(f_min, f_max, nf, nd)
        L = int(math.log2(nf))
        e = _edges(f_min, f_max, nf)[:nf]
        for d in range(0, nd, 7):
            o = O.curve_offsets(T, d)[:nf]
            ideal = np.array([(d_min + d) * _r(f_min, f_max, f) for f in e])
            assert np.max(np.abs(s + o - ideal)) <= 0.5 * L + 1.0 + 1e-9, (nf, d)
    f_min, f_max, nf, nd, d_min, nt = 1200.0, 1600.0, 16, 24, 50, 160
    T = O.build_tables(f_min, f_max, nf, nd)
    s = O.input_shifts(f_min, f_max, nf, d_min)
    for k, u in [(0, 3), (5, 10), (15, 0), (9, 40)]:
        I = np.zeros((nf, nt), dtype=np.int64)
        I[k, u] = 1
        A = O.fdmt(O.map_input(I, s), T, "i64")
        for d in (0, 11, nd - 1):
            o = O.curve_offsets(T, d)
            want = np.zeros(nt, dtype=np.int64)
            want[u + s[k] + o[k]: u + s[k] + o[k + 1] + 1] = 1
            assert np.array_equal(A[d], want), (k, u, d)
    rng = np.random.default_rng(33)
    I = rng.integers(-9, 10, size=(nf, nt))
    assert np.array_equal(O.map_input(I, np.zeros(nf, dtype=np.int64)), I)
    assert np.array_equal(O.map_input(I[::-1], s, descending=True), O.map_input(I, s))
    G = rng.integers(-9, 10, size=(nf, nt))
    for desc in (False, True):
        assert int(np.sum(O.map_input(I, s, desc) * G)) == int(np.sum(I * O.map_input_adjoint(G, s, desc)))


def pin_unequal_split(O):
    """Nf not a power of two (section 4.2: unequal split, f1 the border).
    With gamma = 1 and exact edges (f_min = 1024, delta_f = 256, Nf = 6) the
    delay fraction is linear, so the whole band [0, 6) merges at the border
    after 4 channels with C = 4/6: dl = floor(2 Dt / 3 + 1/2) = (4 Dt + 3) // 6
    (never a tie); the level-2 band of channels 4-5 has no upper half and
    passes up unchanged (dl = Dt), and every level-1 merge halves exactly.
    Row extents still telescope: the level-0 sweeps sum to Nd - 1."""
    T = O.build_tables(1024.0, 1024.0 + 6 * 256.0, 6, 40, gamma=1.0)
    assert T.levels == 3 and [len(T.rows[l]) for l in range(4)] == [6, 3, 2, 1]
    dt = np.arange(40)
    assert np.array_equal(T.dl[3][0], (4 * dt + 3) // 6)
    assert not T.has_upper(2, 1) and np.array_equal(T.dl[2][1], np.arange(T.rows[2][1]))
    assert T.rows[1][2] == T.rows[2][1]
    for b in range(3):
        r = np.arange(T.rows[1][b])
        assert np.array_equal(T.dl[1][b], (r + 1) // 2)
    for nf, nd in ((6, 40), (37, 50), (1000, 700)):
        T = O.build_tables(1200.0, 1600.0, nf, nd)
        assert sum(r - 1 for r in T.rows[0]) == nd - 1 and T.rows[T.levels] == [nd]


def pin_stft_filterbank(O):
    """Front end (section 2: blocks of Nf voltages, Fourier transform,
    squared magnitude, optional binning).
    (1) brute-force DFT of every block (direct sums) on a tiny series;
    (2) a tone at bin frequency q puts a^2 Nf^2 in channel (q + Nf/2) mod Nf
        and nothing elsewhere (negative q in the lower half);
    (3) Parseval: the channels of a spectrum sum to Nf times the block's
        energy;
    (4) binning sums consecutive spectra; trailing samples are dropped."""
    rng = np.random.default_rng(55)
    nf = 8
    v = rng.standard_normal(5 * nf + 3) + 1j * rng.standard_normal(5 * nf + 3)
    P = O.stft_filterbank(v, nf)
    assert P.shape == (nf, 5)
    for t in range(5):
        for c in range(nf):
            k = (c + nf // 2) % nf
            x = sum(v[t * nf + m] * np.exp(-2j * np.pi * k * m / nf) for m in range(nf))
            assert abs(P[c, t] - abs(x) ** 2) <= 1e-9 * (1 + abs(x) ** 2)
    nf = 64
    n = np.arange(4 * nf)
    for q, a in ((5, 1.5), (-3, 0.5), (31, 2.0), (-32, 1.0)):
        P = O.stft_filterbank(a * np.exp(2j * np.pi * q * n / nf), nf)
        c = (q + nf // 2) % nf
        assert np.allclose(P[c], a * a * nf * nf, rtol=1e-12)
        others = np.delete(P, c, axis=0)
        assert np.max(others) <= 1e-18 * nf * nf * a * a + 1e-12
        assert (c < nf // 2) == (q < 0)
    v = rng.standard_normal(6 * nf) + 1j * rng.standard_normal(6 * nf)
    P = O.stft_filterbank(v, nf)
    e = np.sum(np.abs(v.reshape(6, nf)) ** 2, axis=1)
    assert np.allclose(P.sum(axis=0), nf * e, rtol=1e-12)
    P2 = O.stft_filterbank(v, nf, nbin=2)
    assert P2.shape == (nf, 3) and np.allclose(P2, P[:, 0::2] + P[:, 1::2], rtol=1e-12)
    assert O.stft_filterbank(v[: 5 * nf + 7], nf, nbin=2).shape == (nf, 2)


def pin_fft_fdmt(O):
    """FFT-FDMT (Algorithm 2, section 5).
    (1) with the zero padding of the zero-padding paragraph it is the direct
        transform (Algorithm 1, pinned above), to rounding, for power-of-two
        and unequal splits and Nd above and below Nf;
    (2) without padding every shift is cyclic: the result is the brute-force
        sum along the unrolled curves with time taken modulo Nt;
    (3) two instances packed in the real and imaginary parts come back
        separately (the machine-word paragraph);
    (4) the shift vector of s is exp(-2 pi i k s / n), and V(s) V(r) = V(s+r)."""
    rng = np.random.default_rng(77)
    for f_min, f_max, nf, nd, nt in ((1200.0, 1600.0, 16, 20, 50), (1200.0, 1600.0, 6, 40, 37),
                                      (400.0, 800.0, 8, 64, 90), (1100.0, 1700.0, 32, 12, 33)):
        T = O.build_tables(f_min, f_max, nf, nd)
        I = rng.standard_normal((nf, nt))
        A = O.fdmt(I, T)
        B = O.fft_fdmt(I, T)
        assert B.shape == A.shape and B.dtype == np.float64
        assert np.max(np.abs(A - B)) <= 1e-10 * (1 + np.max(np.abs(A)))
        # (2) cyclic without padding
        C = O.fft_fdmt(I, T, n_fft=nt)
        D = np.zeros((nd, nt))
        for d in range(nd):
            o = O.curve_offsets(T, d)
            for k in range(nf):
                for off in range(int(o[k]), int(o[k + 1]) + 1):
                    D[d] += np.roll(I[k], off)
        assert np.max(np.abs(C - D)) <= 1e-10 * (1 + np.max(np.abs(D)))
        # (3) packing
        J = rng.standard_normal((nf, nt))
        P = O.fft_fdmt(I + 1j * J, T)
        assert np.iscomplexobj(P)
        assert np.max(np.abs(P.real - A)) <= 1e-10 * (1 + np.max(np.abs(A)))
        AJ = O.fdmt(J, T)
        assert np.max(np.abs(P.imag - AJ)) <= 1e-10 * (1 + np.max(np.abs(AJ)))
    n = 24
    k = np.arange(n)
    for s in (0, 1, 5, 23, 31):
        assert np.allclose(O.shift_vector(s, n), np.exp(-2j * np.pi * k * s / n), atol=1e-12)
    assert np.allclose(O.shift_vector(5, n) * O.shift_vector(7, n), O.shift_vector(12, n), atol=1e-12)


ALL_PINS = [
    pin_golden_tables,
    pin_golden_values,
    pin_offsets_follow_dispersion_law,
    pin_row_extents,
    pin_scale_invariance,
    pin_power_law_curves,
    pin_bruteforce_exhaustive,
    pin_channel_sum,
    pin_constant_input,
    pin_impulse_response,
    pin_linearity_and_shift,
    pin_flux,
    pin_precision,
    pin_f16_state_rounding,
    pin_weights,
    pin_adjoint_dot,
    pin_adjoint_dense,
    pin_boxcar_search,
    pin_input_map,
    pin_unequal_split,
    pin_stft_filterbank,
    pin_fft_fdmt,
]
