"""Byte-level CPU emulation of the fused schedule's cone program.

Reads the tables a plan exposes through fdmt_fused_tables and executes them
the way the fused kernel does: shared memory as a byte array, TMA row
copies with zero fill outside [0, Nt), the Option-1 partial sums of a cone
that starts at level 0, then one add per op.  Every shared-memory access is
bounds- and alignment-checked, so a planner error is caught on the CPU
before any GPU runs the tables.  Test infrastructure only.
"""
from __future__ import annotations

import numpy as np

BARRIER_BYTES = 128


class SmemError(AssertionError):
    pass


def _types(dtype):
    # input, state, accumulator, output
    if dtype == "u8":
        return np.uint8, np.int32, np.int64, np.int32
    if dtype == "f32":
        return np.float32, np.float32, np.float32, np.float32
    if dtype == "f16state":
        return np.float32, np.float16, np.float32, np.float32
    raise ValueError(dtype)


class Smem:
    def __init__(self, nbytes):
        self.buf = np.zeros(nbytes, dtype=np.uint8)
        self.n = nbytes

    stage = 0
    s_end = 0

    def _check(self, off, count, es, write=False):
        # stage 0: TMA copies write S only; 1: first stage reads S, writes
        # outside it; 2: later stages never touch S.
        lo_in_s = off < self.s_end
        if self.stage == 0 and off + count * es > self.s_end:
            raise SmemError("staged copy outside the staging region")
        if self.stage == 1 and write and lo_in_s:
            raise SmemError("first stage writes into the staging region")
        if self.stage == 2 and lo_in_s:
            raise SmemError("later stage touches the staging region")
        if off % es != 0:
            raise SmemError(f"misaligned access at {off} (element {es} B)")
        if off < BARRIER_BYTES or off + count * es > self.n:
            raise SmemError(f"out of range [{off}, {off + count * es}) of {self.n}")

    def write(self, off, arr):
        arr = np.ascontiguousarray(arr)
        self._check(off, arr.size, arr.itemsize, write=True)
        self.buf[off:off + arr.nbytes] = arr.view(np.uint8)

    def read(self, off, count, dt):
        es = np.dtype(dt).itemsize
        self._check(off, count, es)
        return self.buf[off:off + count * es].copy().view(dt)


def emulate(plan, x, weights=None):
    """Run the plan's fused tables on input x ([nf][nt]) on the CPU."""
    TI, TB, A, TO = _types(plan.dtype)
    acc = np.float32 if A is np.float32 else np.int64
    r16 = plan.dtype == "f16state"
    _, s_state, s_in, s_acc = [int(v) for v in plan.fused_table(6)]
    groups = plan.fused_table(0).reshape(-1, 16)
    tpls = plan.fused_table(1).reshape(-1, 8)
    loads = plan.fused_table(2).reshape(-1, 4)
    inits = plan.fused_table(3).reshape(-1, 8)
    ops = plan.fused_table(4).reshape(-1, 4)
    level_ops = plan.fused_table(5)
    nt = plan.nt
    rows = [int(plan.band_rows(l).sum()) for l in range(plan.levels + 1)]
    L = plan.levels
    state = None
    for gi, (lb, lt, from_input, tb, tc, smem_bytes, ntiles, W, s_end, pa_end, box, chunk, kchunks,
             max_p, in_size, out_size) in enumerate(groups):
        lb, lt, tb, tc, ntiles, W = int(lb), int(lt), int(tb), int(tc), int(ntiles), int(W)
        s_end, pa_end = int(s_end), int(pa_end)
        last = gi == len(groups) - 1
        base = x if from_input else state
        # Levels between launches: the state type, or uint16 where the plan
        # stores integer sums that fit in 16 bits.
        def stored(size):
            if TB is np.int32 and int(size) == 2:
                return np.uint16
            if np.dtype(TB).itemsize != int(size):
                raise SmemError(f"stored sample size {int(size)} does not match the state type")
            return TB
        base_t = TI if from_input else stored(in_size)
        if not from_input and state is not None and state.dtype != base_t:
            raise SmemError("staged type differs from the previous launch's output type")
        out_t = TO if last else stored(out_size)
        dst = np.zeros((rows[lt], nt), dtype=out_t)
        box, chunk, kchunks, max_p = int(box), int(chunk), int(kchunks), int(max_p)
        esz = np.dtype(base_t).itemsize
        nrows_base = plan.nf if from_input else rows[lb]
        if chunk > 0:
            # Row blocks: a 3-D map over [rows][nt / chunk][chunk].
            if nt % chunk != 0 or (chunk * esz) % 16 != 0 or not 1 <= kchunks <= 256:
                raise SmemError("bad row-block map")
            if (kchunks * chunk * esz) % 128 != 0 or not 0 <= max_p <= 5 or (1 << max_p) > nrows_base:
                raise SmemError("bad row-block copy shape")
        elif box < 1 or box > 256 or (box * esz) % 128 != 0:
            raise SmemError("TMA box width must be 1..256 elements and a multiple of 128 bytes")
        for ti in range(tb, tb + tc):
            lb_, lc, ib, ic, lvb, nlv, tx, sb = [int(v) for v in tpls[ti]]
            if sb != int(smem_bytes):
                raise SmemError("template layout differs from its launch's layout")
            for tile in range(ntiles):
                T0 = tile * W
                sm = Smem(int(smem_bytes))
                # Prefetch safety: staged rows live in [128, s_end) and are read
                # only by the first computed stage; everything after it must
                # stay out of that region (the next cone is being staged there).
                sm.stage = 0
                sm.s_end = s_end
                got_tx = 0
                for row, soff, xoff, nbox in loads[lb_:lb_ + lc]:
                    x0 = T0 + int(xoff)
                    if (x0 * np.dtype(base_t).itemsize) % 16 != 0:
                        raise SmemError("TMA column not 16-byte aligned")
                    if int(soff) % 128 != 0:
                        raise SmemError("TMA destination not 128-byte aligned")
                    if chunk > 0:
                        if x0 % chunk != 0 or not 0 <= int(nbox) <= max_p:
                            raise SmemError("row block not on a chunk boundary / too many rows")
                        width, nr = kchunks * chunk, 1 << int(nbox)
                    else:
                        width, nr = int(nbox) * box, 1
                    cols = x0 + np.arange(width)
                    ok = (cols >= 0) & (cols < nt)
                    for r in range(nr):
                        vals = np.zeros(width, dtype=base_t)
                        g = int(row) + r
                        if 0 <= g < nrows_base:
                            vals[ok] = base[g][cols[ok]]
                        sm.write(int(soff) + r * width * esz, vals)
                        got_tx += vals.nbytes
                if got_tx != tx:
                    raise SmemError(f"TMA bytes {got_tx} != expected {tx}")
                if from_input:
                    sm.stage = 1
                    for xs, ds, a, e, width, chan, stride, _ in inits[ib:ib + ic]:
                        xs, ds, a, e, width, stride = map(int, (xs, ds, a, e, width, stride))
                        xv = sm.read(xs - e * s_in, width + e, TI).astype(acc)
                        if weights is not None:
                            xv = (xv.astype(np.float32) * np.float32(weights[int(chan)])).astype(acc)
                        run = None
                        for i in range(e + 1):
                            v = xv[e - i:e - i + width]
                            run = v.copy() if i == 0 else (run + v).astype(acc)
                            if i >= a:
                                st = run.astype(np.float16).astype(np.float32) if r16 else run
                                sm.write(ds + ((i - a) * stride) * s_acc, st.astype(
                                    np.float32 if A is np.float32 else np.int32))
                for lv in range(nlv):
                    sm.stage = 1 if (lv == 0 and not from_input) else 2
                    o0, o1 = int(level_ops[lvb + lv]), int(level_ops[lvb + lv + 1])
                    top = lv == nlv - 1
                    src_t = base_t if (not from_input and lv == 0) else (np.float32 if A is np.float32 else np.int32)
                    for d, lo, hi, width in ops[o0:o1]:
                        width = int(width)
                        a_ = sm.read(int(lo), width, src_t).astype(acc)
                        b_ = sm.read(int(hi), width, src_t).astype(acc)
                        s = (a_ + b_).astype(acc)
                        if top:
                            lim = min(W, nt - T0)
                            if out_t is np.uint16 and (s[:lim].min(initial=0) < 0 or s[:lim].max(initial=0) > 65535):
                                raise SmemError("a sum stored as uint16 does not fit")
                            dst[int(d), T0:T0 + lim] = s[:lim].astype(out_t)
                        else:
                            st = s.astype(np.float16).astype(np.float32) if r16 else s
                            sm.write(int(d), st.astype(np.float32 if A is np.float32 else np.int32))
        state = dst
    return state
