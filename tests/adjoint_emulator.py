"""CPU emulator of the fused adjoint's cone tables (test infrastructure).

Runs the tables a host-only fused plan exposes (fdmt_fused_tables kinds
10-14) the way the CUDA kernel does: per launch, per template and time
tile, the TMA copies of the staged level-lt gradient rows (zeros past Nt),
then the gather stages and the initialisation transpose, in float32 and in
the kernel's order of additions.  Shared memory starts as NaN so a read of
anything no copy or op wrote shows up in the result; every read, write and
whole-piece over-read is checked against its region, and every output
element must be written exactly once.
"""
import numpy as np

PIECE = 256          # columns of one op (32 lanes x 8)
BARRIER = 128
WARPS = 8
STAGE_WORDS = 2 + WARPS
GATHER, INIT, INITF = 1, 2, 3


def term_groups(kind, p0, p1, p2, flags):
    """The word addresses an op sums, as groups: each group's terms are
    added in order into one value, and the groups' values in order into the
    result (a gather is one group; the initialisation transpose one group
    per term; the folded transpose one group per level-0 value, its run of
    level-1 rows)."""
    if kind == GATHER:
        return [[(p0 + j * p1) // 4 for j in range(p2)]]
    if kind == INIT:
        return [[(p0 + j * p1) // 4 + i] for j in range(p2) for i in range(j + 1)]
    if kind == INITF:
        groups, pj, up = [], p0, flags & 1
        for j in range(p2):
            cnt = (flags >> (1 + 4 * j)) & 15
            if cnt < 1:
                raise AdjointTableError("folded init op with an empty run")
            for i in range(j + 1):
                groups.append([(pj + 4 * i + q * p1) // 4 for q in range(cnt)])
            pj += cnt * p1 - 4 * up
        return groups
    raise AdjointTableError("unknown stage kind")


class AdjointTableError(AssertionError):
    pass


def layout(plan):
    """(over-read slack, descriptor slot bytes) that end a block's shared memory."""
    return tuple(int(v) for v in plan.fused_table(6)[4:6])


def tables(plan):
    return (plan.fused_table(10).reshape(-1, 15), plan.fused_table(11).reshape(-1, 8),
            plan.fused_table(12).reshape(-1, 4), plan.fused_table(13).reshape(-1, 8), plan.fused_table(14))


def emulate_adjoint(plan, g_out, weights=None):
    """grad_in of the plan's fused adjoint for the output gradient g_out
    ([nd, nt] float32), scaled by weights ([nf]) when given."""
    groups, tpls, loads, ops, stages = tables(plan)
    if len(groups) == 0:
        raise AdjointTableError("the plan has no fused adjoint")
    over_read, desc = layout(plan)
    nt = plan.nt
    L = plan.levels
    level_rows = [int(plan.band_rows(l).sum()) for l in range(L + 1)]
    cur = np.asarray(g_out, dtype=np.float32)
    if cur.shape != (plan.nd, nt):
        raise ValueError("g_out must be [nd, nt]")
    w = None if weights is None else np.asarray(weights, dtype=np.float32)
    for gi, grp in enumerate(groups):
        lt, lb, init, W, box, tb, tc, smem_bytes, s_end, pa_end, ntiles, _, chunk, kchunks, max_p = (
            int(v) for v in grp)
        if (box > 0) == (chunk > 0) or (chunk > 0 and (nt % chunk or not 1 <= kchunks <= 256 or max_p > 5)):
            raise AdjointTableError("bad staging format")
        if cur.shape[0] != level_rows[lt]:
            raise AdjointTableError(f"launch {gi} stages level {lt} from a buffer of {cur.shape[0]} rows")
        out_rows = plan.nf if init else level_rows[lb]
        out = np.zeros((out_rows, nt), dtype=np.float32)
        hits = np.zeros((out_rows, nt), dtype=np.int32)
        if smem_bytes > 227 * 1024 or s_end < BARRIER or pa_end < s_end or smem_bytes < pa_end + over_read + desc:
            raise AdjointTableError("bad launch layout")
        for tpl in range(tb, tb + tc):
            lb0, lc, _, _, sb, n_st, tx, _ = (int(v) for v in tpls[tpl])
            for tile in range(ntiles):
                T0 = tile * W
                sm = np.full(smem_bytes // 4, np.nan, dtype=np.float32)
                got = 0
                for row, off, xoff, nbox in loads[lb0:lb0 + lc]:
                    row, off, xoff, nbox = int(row), int(off), int(xoff), int(nbox)
                    # row boxes: nbox boxes of one row; row blocks: 2^nbox rows
                    nrows, n = (1, nbox * box) if chunk == 0 else (1 << nbox, kchunks * chunk)
                    if chunk > 0 and (nbox > max_p or (T0 + xoff) % chunk):
                        raise AdjointTableError("bad row block")
                    if off % 16 or (T0 + xoff) % 4 or off < BARRIER or off + 4 * n * nrows > s_end:
                        raise AdjointTableError("staged copy outside S or misaligned")
                    if row < 0 or row + nrows > cur.shape[0]:
                        raise AdjointTableError("staged rows outside level lt")
                    cols = T0 + xoff + np.arange(n)
                    ok = (cols >= 0) & (cols < nt)
                    for r in range(nrows):
                        vals = np.zeros(n, dtype=np.float32)
                        vals[ok] = cur[row + r, cols[ok]]
                        a = off // 4 + r * n
                        sm[a:a + n] = vals
                    got += 4 * n * nrows
                if got != tx:
                    raise AdjointTableError("TMA byte count differs from the copies")
                for s in range(n_st):
                    words = stages[sb + s * STAGE_WORDS:sb + (s + 1) * STAGE_WORDS]
                    kind = int(words[0])
                    starts = [int(v) for v in words[1:]]
                    if any(starts[i] > starts[i + 1] for i in range(WARPS)):
                        raise AdjointTableError("warp ranges out of order")
                    last = s == n_st - 1
                    if kind in (INIT, INITF) and not (init and last):
                        raise AdjointTableError("initialisation transpose not at the end of the last launch")
                    lo_ok = BARRIER if s == 0 else s_end
                    hi_ok = s_end if s == 0 else smem_bytes - over_read - desc
                    writes = []
                    for dst, p0, p1, p2, _, width, flags, col in ops[starts[0]:starts[WARPS]]:
                        dst, p0, p1, p2, width, flags, col = (int(v) for v in (dst, p0, p1, p2, width, flags, col))
                        if not 0 < width <= PIECE or p2 < 1 or p0 % 4 or p1 % 4:
                            raise AdjointTableError("bad op")
                        v = None  # the sum starts from the first term
                        for grp in term_groups(kind, p0, p1, p2, flags):
                            r = None
                            for a in grp:
                                if a * 4 < lo_ok or (a + width) * 4 > hi_ok:
                                    raise AdjointTableError("op reads outside its source region")
                                if (a + PIECE) * 4 > smem_bytes:
                                    raise AdjointTableError("whole-piece read past the end of shared memory")
                                x = sm[a:a + width].astype(np.float32)
                                r = x.copy() if r is None else (r + x).astype(np.float32)
                            v = r if v is None else (v + r).astype(np.float32)
                        if kind in (INIT, INITF) and w is not None:
                            v = (v * w[dst]).astype(np.float32)
                        if last and not (init and kind == GATHER):
                            t = T0 + col + np.arange(width)
                            ok = (t >= 0) & (t < nt)
                            out[dst, t[ok]] = v[ok]
                            hits[dst, t[ok]] += 1
                        else:
                            if dst % 4 or dst < s_end or dst + 4 * width > smem_bytes - over_read - desc:
                                raise AdjointTableError("op writes outside Pa / Pb")
                            writes.append((dst // 4, v))
                    # a stage's writes land after all its reads (a block barrier)
                    for a, v in writes:
                        sm[a:a + len(v)] = v
        if not (hits == 1).all():
            bad = np.argwhere(hits != 1)
            raise AdjointTableError(f"launch {gi}: {len(bad)} outputs written {hits[tuple(bad[0])]} times, "
                                    f"first at {bad[0].tolist()}")
        cur = out
    return cur


def check_adjoint_tables(plan):
    """Static checks of a (possibly full-size) plan's adjoint tables: every
    copy, read, whole-piece over-read and write inside its region, and every
    output row owned by one template whose pieces tile [o, o + W) with
    o <= 0 and o + ntiles W >= Nt (so each output element is written exactly
    once over the tiles).  Returns the number of ops checked."""
    groups, tpls, loads, ops, stages = tables(plan)
    over_read, desc = layout(plan)
    nt = plan.nt
    L = plan.levels
    level_rows = [int(plan.band_rows(l).sum()) for l in range(L + 1)]
    checked = 0
    for gi, grp in enumerate(groups):
        lt, lb, init, W, box, tb, tc, smem_bytes, s_end, pa_end, ntiles, _, chunk, kchunks, max_p = (
            int(v) for v in grp)
        if (box > 0) == (chunk > 0) or (chunk > 0 and (nt % chunk or not 1 <= kchunks <= 256 or max_p > 5)):
            raise AdjointTableError("bad staging format")
        owner = {}
        pieces = {}
        for tpl in range(tb, tb + tc):
            lb0, lc, _, _, sb, n_st, tx, _ = (int(v) for v in tpls[tpl])
            ld = loads[lb0:lb0 + lc]
            if len(ld):
                if chunk == 0:
                    nrows, nbytes = np.ones(len(ld), np.int64), 4 * box * ld[:, 3]
                else:
                    nrows, nbytes = 1 << ld[:, 3].astype(np.int64), 4 * kchunks * chunk * (1 << ld[:, 3].astype(np.int64))
                    if (ld[:, 3] > max_p).any():
                        raise AdjointTableError("row block larger than the maps")
                if (ld[:, 1] % 16).any() or (ld[:, 1] < BARRIER).any() or \
                        (ld[:, 1] + nbytes > s_end).any() or (ld[:, 2] % 4).any():
                    raise AdjointTableError("staged copy outside S or misaligned")
                if (ld[:, 0] < 0).any() or (ld[:, 0] + nrows > level_rows[lt]).any():
                    raise AdjointTableError("staged row outside level lt")
                if int(nbytes.sum()) != tx:
                    raise AdjointTableError("TMA byte count differs from the copies")
            for s in range(n_st):
                words = stages[sb + s * STAGE_WORDS:sb + (s + 1) * STAGE_WORDS]
                kind = int(words[0])
                op = ops[int(words[1]):int(words[WARPS + 1])]
                if np.any(np.diff(words[1:]) < 0):
                    raise AdjointTableError("warp ranges out of order")
                if len(op) == 0:
                    continue
                dst, p0, p1, p2, width, col = op[:, 0], op[:, 1], op[:, 2], op[:, 3], op[:, 5], op[:, 7]
                last = s == n_st - 1
                lo_ok = BARRIER if s == 0 else s_end
                hi_ok = s_end if s == 0 else smem_bytes - over_read - desc
                if (width <= 0).any() or (width > PIECE).any() or (p2 < 1).any():
                    raise AdjointTableError("bad op")
                if kind == INITF:
                    lo_a = np.empty(len(op), np.int64)
                    hi_a = np.empty(len(op), np.int64)
                    for n_, o in enumerate(op):
                        addrs = [a for g in term_groups(INITF, int(o[1]), int(o[2]), int(o[3]), int(o[6]))
                                 for a in g]
                        lo_a[n_], hi_a[n_] = 4 * min(addrs), 4 * max(addrs)
                    first, span = lo_a, hi_a - p0
                    if not (init and last):
                        raise AdjointTableError("folded initialisation transpose outside the end of the last launch")
                else:
                    first, span = p0, (p2 - 1) * p1 + (4 * (p2 - 1) if kind == INIT else 0)
                if (first < lo_ok).any() or (p0 + span + 4 * width > hi_ok).any():
                    raise AdjointTableError("op reads outside its source region")
                if (p0 + span + 4 * PIECE > smem_bytes).any():
                    raise AdjointTableError("whole-piece read past the end of shared memory")
                if last and not (init and kind == GATHER):
                    rows = plan.nf if init else level_rows[lb]
                    if (dst < 0).any() or (dst >= rows).any():
                        raise AdjointTableError("global row out of range")
                    for d, c, wd in zip(dst.tolist(), col.tolist(), width.tolist()):
                        if owner.setdefault(d, tpl) != tpl:
                            raise AdjointTableError(f"row {d} owned by two templates")
                        pieces.setdefault(d, []).append((c, wd))
                else:
                    if (dst < s_end).any() or (dst + 4 * width > smem_bytes - over_read - desc).any():
                        raise AdjointTableError("op writes outside Pa / Pb")
                checked += len(op)
        rows = plan.nf if init else level_rows[lb]
        if len(owner) != rows:
            raise AdjointTableError(f"launch {gi}: {rows - len(owner)} output rows have no owner")
        for d, ps in pieces.items():
            ps.sort()
            o = ps[0][0]
            end = o
            for c, wd in ps:
                if c != end:
                    raise AdjointTableError(f"row {d}: pieces do not tile the tile")
                end = c + wd
            if end - o != W or o > 0 or o + ntiles * W < nt:
                raise AdjointTableError(f"row {d}: window [{o}, {end}) does not cover time with {ntiles} tiles")
    return checked
