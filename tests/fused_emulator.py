"""Byte-level CPU emulation of the fused schedule's cone program.

Reads the tables a plan exposes through fdmt_fused_tables and executes them
the way the fused kernel does: shared memory as a byte array, TMA row
copies with zero fill outside [0, Nt), then the item's stages warp by warp:
level 1 walked from the staged input (running Option-1 sums, the upper
half's sums moved one column later when dl grows), single levels (one add
per op) and pairs of levels ((lo + hi) + (lo + hi) per op), with each op's
reuse flags applied to the previous op of the same warp exactly as the
kernel does.  Every shared-memory access is bounds- and alignment-checked,
so a planner error is caught on the CPU before any GPU runs the tables.
Test infrastructure only.
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
    def __init__(self, nbytes, write_end=None):
        self.buf = np.zeros(nbytes, dtype=np.uint8)
        self.n = nbytes
        # writes end before the warps' descriptor slots and the slack
        self.write_end = nbytes if write_end is None else write_end

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
        if write and off + count * es > self.write_end:
            raise SmemError(f"write [{off}, {off + count * es}) reaches the descriptor slots at {self.write_end}")

    def write(self, off, arr):
        arr = np.ascontiguousarray(arr)
        self._check(off, arr.size, arr.itemsize, write=True)
        self.buf[off:off + arr.nbytes] = arr.view(np.uint8)

    def read(self, off, count, dt):
        es = np.dtype(dt).itemsize
        self._check(off, count, es)
        return self.buf[off:off + count * es].copy().view(dt)


WALK, SINGLE, PAIR, SEARCH = 0, 1, 2, 3
PADDED, KIND_MASK, GENERAL = 16, 15, 32
LO_SAME, HI_SHIFT, LO_ONE, HI_ONE, NO_HI = 1, 2, 4, 8, 16
WALK_NO_UPPER = 1
STAGE_WORDS = 10
WARPS = 8
PIECE = 256


def pidx(c):
    """Search layout of a row of 4-byte values: 4 words of padding after
    every 16 columns."""
    return c + 4 * (c >> 4)


def emulate(plan, x, weights=None, partials=None):
    """Run the plan's fused tables on input x ([nf][nt]) on the CPU.  A plan
    whose last launch ends with the boxcar search stores its per-tile
    partials in `partials` (a dict (row, width, tile) -> (value, region))."""
    TI, TB, A, TO = _types(plan.dtype)
    acc = np.float32 if A is np.float32 else np.int64
    smem_acc = np.float32 if A is np.float32 else np.int32
    r16 = plan.dtype == "f16state"
    _, s_state, s_in, s_acc, over_read, desc = [int(v) for v in plan.fused_table(6)]
    groups = plan.fused_table(0).reshape(-1, 16)
    tpls = plan.fused_table(1).reshape(-1, 8)
    loads = plan.fused_table(2).reshape(-1, 4)
    walks = plan.fused_table(3).reshape(-1, 12)
    ops = plan.fused_table(4).reshape(-1, 8)
    stages = plan.fused_table(5)
    nt = plan.nt
    rows = [int(plan.band_rows(l).sum()) for l in range(plan.levels + 1)]
    L = plan.levels
    wvec = None if weights is None else np.asarray(weights, dtype=np.float32)
    search_k = int(getattr(plan, "search_widths", 0))

    def rnd(v):  # a value of a stored (not last) level in fp16-state mode
        return v.astype(np.float16).astype(np.float32) if r16 else v

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
        top_rounds = lt < L  # the group's top level is a stored state level
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
            lb_, lc, wb, wc, sb, nst, tx, smb = [int(v) for v in tpls[ti]]
            if smb != int(smem_bytes):
                raise SmemError("template layout differs from its launch's layout")
            for tile in range(ntiles):
                T0 = tile * W
                lim = min(W, nt - T0)
                sm = Smem(int(smem_bytes), int(smem_bytes) - over_read - desc)
                # Prefetch safety: staged rows live in [128, s_end) and are read
                # only by the first stage; everything after it must stay out of
                # that region (the next cone is being staged there).
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

                def put(d, col, v, stored_out):
                    """Store one output row piece: shared memory, or the
                    group's top level in global memory."""
                    if stored_out:
                        sm.write(int(d), v.astype(smem_acc))
                        return
                    n = max(0, min(len(v), lim - col))
                    if out_t is np.uint16 and n and (v[:n].min() < 0 or v[:n].max() > 65535):
                        raise SmemError("a sum stored as uint16 does not fit")
                    dst[int(d), T0 + col:T0 + col + n] = v[:n].astype(out_t)

                for si in range(nst):
                    blk = [int(v) for v in stages[sb + si * STAGE_WORDS: sb + (si + 1) * STAGE_WORDS]]
                    kind, offs = blk[0] & KIND_MASK, blk[1:]
                    padded = bool(blk[0] & PADDED)
                    sm.stage = 1 if si == 0 else 2
                    is_top = si == nst - 1 and not padded
                    src_t = (TI if from_input else base_t) if si == 0 else smem_acc
                    sz = np.dtype(src_t).itemsize
                    if any(offs[w] > offs[w + 1] for w in range(WARPS)):
                        raise SmemError("warp ranges out of order")
                    for w in range(WARPS):
                        prev = None  # (lo part, hi part) of the warp's previous op
                        if kind == WALK:
                            if si != 0 or not from_input:
                                raise SmemError("walk stage outside the first stage of an input launch")
                            for (d, drow, xlo, xhi, width, col, a, e, dl0, bits, chan, wfl) in walks[offs[w]:offs[w + 1]]:
                                d, drow, xlo, xhi, width, col, a, e, dl0, bits, chan, wfl = map(
                                    int, (d, drow, xlo, xhi, width, col, a, e, dl0, bits, chan, wfl))
                                upper = not (wfl & WALK_NO_UPPER)
                                if not (0 < width <= PIECE and 0 <= e - a < 32 and 0 <= dl0 <= a):
                                    raise SmemError("bad walk descriptor")
                                # history the walk reads: the lower channel up to
                                # its last dl, the upper one up to dl + j = e
                                hl = dl0 + bin(bits & ((1 << (e - a)) - 1)).count("1")
                                he = e
                                if not upper:
                                    hl = e  # a single channel: dl = row, up to e
                                xl = sm.read(xlo - hl * sz, width + hl, TI).astype(acc)
                                if upper:
                                    xh = sm.read(xhi - he * sz, width + he, TI).astype(acc)
                                else:
                                    xh = np.zeros(width + he, dtype=acc)
                                if wvec is not None:
                                    xl = (xl.astype(np.float32) * wvec[chan]).astype(acc)
                                    if upper:
                                        xh = (xh.astype(np.float32) * wvec[chan + 1]).astype(acc)
                                XL = lambda s_: xl[hl - s_: hl - s_ + width]  # x_lo[tau - s]
                                XH = lambda s_: xh[he - s_: he - s_ + width]  # x_hi[tau - s]
                                dl, j = dl0, a - dl0
                                plo = XL(0).copy()
                                for i in range(1, dl + 1):
                                    plo = (plo + XL(i)).astype(acc)
                                phi = XH(dl).copy()
                                for i in range(1, j + 1):
                                    phi = (phi + XH(dl + i)).astype(acc)
                                for r in range(a, e + 1):
                                    if r > a and not upper:
                                        dl += 1
                                        plo = (plo + XL(dl)).astype(acc)
                                    elif r > a:
                                        if (bits >> (r - a - 1)) & 1:
                                            dl += 1
                                            plo = (plo + XL(dl)).astype(acc)
                                            first = xh[he - dl] + 0
                                            for i in range(1, j + 1):
                                                first = first + xh[he - dl - i]
                                            phi = np.concatenate(([first], phi[:-1])).astype(acc)
                                        else:
                                            j += 1
                                            phi = (phi + XH(dl + j)).astype(acc)
                                    v = (rnd(plo) + rnd(phi)).astype(acc) if upper else rnd(plo)
                                    if (not is_top) or top_rounds:
                                        v = rnd(v)
                                    if is_top:
                                        put(d + (r - a), col, v, False)
                                    else:
                                        put(d + (r - a) * drow, col, v, True)
                            continue
                        if kind == SEARCH:
                            if si != nst - 1:
                                raise SmemError("search stage before the last stage")
                            for (d, p0, _, _, _, width, _, hist) in ops[offs[w]:offs[w + 1]]:
                                d, p0, width, hist = int(d), int(p0), int(width), int(hist)
                                n = width + hist
                                if n % 16 or hist % 16:
                                    raise SmemError("search window not in runs of 16 columns")
                                v = np.array([sm.read(p0 + pidx(c) * s_acc, 1, smem_acc)[0] for c in range(n)],
                                             dtype=acc)
                                own = np.arange(hist, hist + lim)
                                dst[d, T0:T0 + lim] = v[own].astype(out_t)
                                nk = search_k
                                B = v.copy()
                                t0 = T0 - hist
                                for k in range(nk):
                                    if k > 0:
                                        h = 1 << (k - 1)
                                        B = (B + np.concatenate((np.zeros(h, dtype=acc), B[:-h]))).astype(acc)
                                    vals = B[own]
                                    c = hist + int(np.argmax(vals))
                                    g = 16 if k <= 4 else 256
                                    partials[(d, k, tile)] = (vals.max(), t0 + g * (c // g))
                            continue
                        for (d, p0, p1, p2, p3, width, flags, col) in ops[offs[w]:offs[w + 1]]:
                            d, p0, p1, p2, p3, width, flags, col = map(int, (d, p0, p1, p2, p3, width, flags, col))
                            if not 0 < width <= PIECE:
                                raise SmemError("op wider than a piece")
                            if flags & (LO_SAME | HI_SHIFT) and prev is None:
                                raise SmemError("a warp's first op reuses an earlier op")
                            if kind == SINGLE:
                                lo = prev[0] if flags & LO_SAME else sm.read(p0, width, src_t).astype(acc)
                                if flags & NO_HI:
                                    hi = None
                                    v = lo.copy()
                                else:
                                    hi = sm.read(p1, width, src_t).astype(acc)
                                    v = (lo + hi).astype(acc)
                                prev = (lo, hi)
                            elif kind == PAIR:
                                if flags & LO_SAME:
                                    lp = prev[0]
                                elif flags & LO_ONE:
                                    lp = rnd(sm.read(p0, width, src_t).astype(acc))
                                else:
                                    lp = rnd((sm.read(p0, width, src_t).astype(acc) +
                                              sm.read(p1, width, src_t).astype(acc)).astype(acc))
                                hp = None
                                if flags & NO_HI:
                                    v = lp.copy()
                                else:
                                    one = bool(flags & HI_ONE)
                                    if flags & HI_SHIFT:
                                        h0 = sm.read(p2, 1, src_t).astype(acc)
                                        if not one:
                                            h0 = (h0 + sm.read(p3, 1, src_t).astype(acc)).astype(acc)
                                        h0 = rnd(h0)
                                        if prev[1] is None or len(prev[1]) < width - 1:
                                            raise SmemError("shifted upper half without a previous one")
                                        hp = np.concatenate((h0, prev[1][:width - 1])).astype(acc)
                                    elif one:
                                        hp = rnd(sm.read(p2, width, src_t).astype(acc))
                                    else:
                                        hp = rnd((sm.read(p2, width, src_t).astype(acc) +
                                                  sm.read(p3, width, src_t).astype(acc)).astype(acc))
                                    v = (lp + hp).astype(acc)
                                prev = (lp, hp)
                            else:
                                raise SmemError(f"unknown stage kind {kind}")
                            if padded:  # the top level into Pt, search layout, not rounded
                                for j in range(width):
                                    sm.write(d + pidx(j) * s_acc, np.array([v[j]]).astype(smem_acc))
                                continue
                            if (not is_top) or top_rounds:
                                v = rnd(v)
                            put(d, col, v, not is_top)
        state = dst
    return state


def check_bounds(plan):
    """Static check of every template of a plan, without running a tile:
    each walk's and op's shared-memory reads and writes lie inside the
    launch's dynamic shared memory (after the barrier slot), the first stage
    writes nothing into the staging region and later stages do not touch
    it, descriptors are well formed and every stage's warp ranges tile its
    ops.  Cheap enough for full-size plans."""
    groups = plan.fused_table(0).reshape(-1, 16)
    tpls = plan.fused_table(1).reshape(-1, 8)
    walks = plan.fused_table(3).reshape(-1, 12).astype(np.int64)
    ops = plan.fused_table(4).reshape(-1, 8).astype(np.int64)
    stages = plan.fused_table(5)
    _, s_state, s_in, s_acc, over_read, desc = [int(v) for v in plan.fused_table(6)]
    checked = 0
    for (lb, lt, from_input, tb, tc, smem_bytes, ntiles, W, s_end, pa_end, box, chunk, kchunks,
         max_p, in_size, out_size) in groups:
        smem_bytes, s_end = int(smem_bytes), int(s_end)
        for ti in range(int(tb), int(tb) + int(tc)):
            _, _, wb, wc, sb, nst, _, _ = [int(v) for v in tpls[ti]]
            for si in range(nst):
                blk = [int(v) for v in stages[sb + si * STAGE_WORDS: sb + (si + 1) * STAGE_WORDS]]
                kind, offs = blk[0] & KIND_MASK, blk[1:]
                padded = bool(blk[0] & PADDED)
                if any(offs[w] > offs[w + 1] for w in range(WARPS)):
                    raise SmemError("warp ranges out of order")
                # the kernel tests the structural flags only in stages marked general
                if kind == WALK:
                    structural = bool((walks[offs[0]:offs[-1], 11] & WALK_NO_UPPER).any())
                elif kind != SEARCH:
                    structural = bool((ops[offs[0]:offs[-1], 6] & (LO_ONE | HI_ONE | NO_HI)).any())
                else:
                    structural = False
                if structural != bool(blk[0] & GENERAL):
                    raise SmemError("stage's general flag does not match its ops")
                top = si == nst - 1 and not padded
                first = si == 0
                if kind == SEARCH:
                    op = ops[offs[0]:offs[-1]]
                    if len(op) == 0:
                        continue
                    n = op[:, 5] + op[:, 7]
                    if np.any(op[:, 1] < s_end) or np.any(op[:, 1] + pidx(n) * s_acc > smem_bytes):
                        raise SmemError("search row outside Pt")
                    checked += len(op)
                    continue
                lo_ok = BARRIER_BYTES if first else s_end
                if kind == WALK:
                    wk = walks[offs[0]:offs[-1]]
                    if len(wk) == 0:
                        continue
                    d, drow, xlo, xhi, width, col, a, e, dl0, bits = (wk[:, i] for i in range(10))
                    if np.any(width <= 0) or np.any(width > PIECE) or np.any(e - a >= 32) or np.any(e < a):
                        raise SmemError("bad walk descriptor")
                    hl = dl0 + np.array([bin(int(b) & ((1 << int(n)) - 1)).count("1") for b, n in zip(bits, e - a)])
                    up = (wk[:, 11] & WALK_NO_UPPER) == 0
                    hl = np.where(up, hl, e)
                    for base, hist, wd in ((xlo, hl, width), (xhi[up], e[up], width[up])):
                        if np.any(base - hist * s_in < BARRIER_BYTES) or np.any(base + wd * s_in > s_end):
                            raise SmemError("walk reads outside the staged input")
                        if np.any(base + PIECE * s_in > smem_bytes):
                            raise SmemError("a whole-piece read runs past the end of shared memory")
                    if not top:
                        w0 = d
                        w1 = d + (e - a) * drow + width * s_acc
                        if np.any(w0 < s_end) or np.any(w1 > smem_bytes - over_read - desc):
                            raise SmemError("walk writes outside Pa / Pb")
                    checked += len(wk)
                    continue
                op = ops[offs[0]:offs[-1]]
                if len(op) == 0:
                    continue
                width = op[:, 5]
                if np.any(width <= 0) or np.any(width > PIECE):
                    raise SmemError("bad op width")
                es = (int(in_size) if first and not int(from_input) else s_acc)
                fl = op[:, 6]
                if kind == PAIR:
                    srcs = [op[:, 1], op[fl & LO_ONE == 0, 2], op[fl & NO_HI == 0, 3],
                            op[(fl & (NO_HI | HI_ONE)) == 0, 4]]
                    width_of = [width, width[fl & LO_ONE == 0], width[fl & NO_HI == 0],
                                width[(fl & (NO_HI | HI_ONE)) == 0]]
                else:
                    srcs = [op[:, 1], op[fl & NO_HI == 0, 2]]
                    width_of = [width, width[fl & NO_HI == 0]]
                for p, width in zip(srcs, width_of):
                    if np.any(p < lo_ok) or np.any(p + width * es > (s_end if first else smem_bytes)) or np.any(p % es):
                        raise SmemError("op reads outside its source region")
                    # the kernel reads whole pieces: they must stay inside the block's memory
                    if np.any(p + PIECE * es > smem_bytes):
                        raise SmemError("a whole-piece read runs past the end of shared memory")
                width = op[:, 5]
                if not top:
                    span = pidx(width) if padded else width
                    if np.any(op[:, 0] < s_end) or np.any(op[:, 0] + span * s_acc > smem_bytes - over_read - desc):
                        raise SmemError("op writes outside Pa / Pb / Pt")
                starts = [offs[w] for w in range(WARPS) if offs[w] < offs[w + 1]]
                if np.any(ops[starts, 6] & (LO_SAME | HI_SHIFT)):
                    raise SmemError("a warp's first op reuses an earlier op")
                checked += len(op)
    return checked


def emulate_search(plan, x, n_widths, weights=None):
    """(A, peak, time) of a plan made with search_widths == n_widths: the
    emulated launches, then the finalize step from the partials: per row and
    width the largest value over the tiles, the earliest region holding it,
    and the first time in that region where the width's sum has the value
    (the sum recomputed from A, B_1 = A, B_2w[t] = B_w[t] + B_w[t - w])."""
    parts = {}
    A = emulate(plan, x, weights, partials=parts)
    nd, nt = A.shape
    tiles = 1 + max(t for (_, _, t) in parts)
    acc = np.float32 if A.dtype == np.float32 else np.int64
    peak = np.zeros((nd, n_widths), dtype=acc)
    when = np.zeros((nd, n_widths), dtype=np.int32)
    for d in range(nd):
        B = A[d].astype(acc)
        for k in range(n_widths):
            if k > 0:
                h = 1 << (k - 1)
                B = (B + np.concatenate((np.zeros(h, dtype=acc), B[:-h]))).astype(acc)
            cand = [parts[(d, k, t)] for t in range(tiles)]
            m = max(v for v, _ in cand)
            reg = min(r for v, r in cand if v == m)
            g = 16 if k <= 4 else 256
            hit = [t for t in range(max(reg, 0), min(reg + g, nt)) if B[t] == m]
            if not hit:
                raise SmemError(f"row {d} width {1 << k}: no time with the peak in region {reg}")
            peak[d, k] = m
            when[d, k] = hit[0]
    return A, peak, when
