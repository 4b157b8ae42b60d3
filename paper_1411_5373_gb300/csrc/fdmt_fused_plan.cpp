// Host planner of the fused schedule (see fdmt_fused.h).
//
// For one group of levels (lb, lt] and one tile width W, every band of level
// lt is split into the fewest row ranges whose cones fit the shared-memory
// budget.  A cone is unrolled top-down with the addition rule of section 4:
// parent rows [a, e] with window offset o and spread s have
//   lower half rows [dl(a), dl(e)], offset o,          spread s
//   upper half rows [a - dl(a), e - dl(e)], offset o + dl(e), spread s + dl(e) - dl(a)
// and parent row Dt reads the upper half at column tau + dl(e) - dl(Dt).
//
// Staged rows reach shared memory by TMA in one of two formats per launch:
// row boxes (a 2-D [rows][nt] map; each row window is copied by whole boxes
// of up to 256 elements) or row blocks (a 3-D [rows][nt / C][C] map, C
// elements = 128 bytes or 64; one copy brings 2^p consecutive rows of K
// chunks, landing with row pitch K * C, so a node of R rows takes popcount(R)
// copies).  Row blocks need nt to be a multiple of C and windows that start
// on a chunk boundary; the input channels of a from-input cone share one
// window (the union of theirs) so they form one block.
//
// The level grouping and W are chosen by a cost model (dynamic programming
// over group boundaries).  A launch takes the larger of its HBM time (staged
// plus written bytes) and its on-chip time: a cost per column of every
// shared-memory op and Option-1 step, plus, per block slot of the GPU
// (SMs x resident blocks), a latency per work item and per op.  The
// constants are a least-squares fit to per-launch device times measured on a
// GB300 over 907 launches of 5 shapes x 4-7 level groupings x 4 tiles x 3
// budgets (mean absolute error 5 %).
#include "fdmt_fused.h"

#include <algorithm>
#include <cmath>
#include <limits>

namespace fdmt {
namespace {

constexpr int32_t kBarrierBytes = 128;  // mbarrier slot, keeps regions 128-byte aligned
constexpr double kHbmRate = 6.0e12;          // bytes/s of unique rows in and out
constexpr double kL2Rate = 14.0e12;          // bytes/s of staged rows (halos and overlaps come from L2)
constexpr double kSlotSeconds = 7.0e-12;     // per shared-memory pipe slot (GPU-wide)
constexpr double kItemSeconds = 0.3e-6;      // per work item, per block slot
constexpr double kOpSeconds = 0;             // per op, per block slot
constexpr double kLaunchSeconds = 8e-6;
constexpr double kSms = 152;
constexpr double kMaxBlocksPerSm = 4;        // the fused kernel's register limit

int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }
int64_t ceil_to(int64_t v, int64_t a) { return round_up(v, a); }

struct Node {
  int32_t band, a, e;  // band index at its level, first and last row
  int32_t o, s;        // window [T0 - o, T0 - o + W + s)
  int32_t smem = 0;    // byte offset of row a
  int32_t stride = 0;  // elements per row in shared memory
  int32_t delta = 0;   // column of time T0 - o within the stored row
  int32_t xsmem = 0, xstride = 0, xdelta = 0;  // staged input (level 0 of an input cone)
  int32_t klo = -1, khi = -1;  // the halves in the level below (khi < 0: none, rows pass up)
};

struct ConeOut {
  FusedTemplate tpl{};
  std::vector<FusedLoad> loads;
  std::vector<FusedWalk> walks;                 // the first stage of a launch from the input
  std::vector<std::vector<FusedOp>> stage_ops;  // single / pair stages, in row order (before the warp split)
  std::vector<int32_t> kinds;                   // stage kinds
  double hbm = 0;
  double slots = 0;  // cost model: shared-memory pipe slots of one tile (warp instructions)
  double nops = 0;   // ops and walks of one tile
};

// Region sizes of one cone: S = staged source rows (input channels or the
// base level), Pa / Pb = computed levels, alternating.  A group lays all its
// cones out at the same region bases (the maxima over its cones) so that a
// block can stage the next cone into S while it still computes in Pa / Pb.
struct ConeShape {
  std::vector<std::vector<Node>> nodes;  // [level - lb]
  int64_t s_bytes = 0, pa_bytes = 0, pb_bytes = 0;
  int64_t pt_bytes = 0;  // search: the top level in the search layout
  int32_t top_rows = 0;  // rows of the top node
  std::vector<std::pair<int32_t, int32_t>> needs;  // (window elements from the aligned start, rows) per staged node
  int32_t x_o = 0;  // row blocks, from input: the channels' common window starts at T0 - x_o
};

// Staging format of a launch.  chunk == 0: row boxes of `box` elements.
// chunk > 0: row blocks of kchunks chunks (kchunks == 0 while the windows
// are being measured: each cone then uses its own widest window).
struct StageFmt {
  int32_t box = 0;
  int32_t chunk = 0, kchunks = 0;
  int32_t max_p = 0;  // copies bring at most 2^max_p rows
  int32_t search_k = 0;  // > 0: the launch ends with the boxcar search of this many widths
};

}  // namespace

// The levels a group (lb, lt] stores: lb (staged, or the input when lb = 0),
// then every level a stage ends on.  From the input the first stage ends on
// level 1; an odd number of levels left takes one single-level stage first;
// the rest are pairs.
std::vector<int32_t> stored_levels(int32_t lb, int32_t lt) {
  std::vector<int32_t> v{lb};
  int32_t cur = lb;
  if (lb == 0) {
    v.push_back(1);
    cur = 1;
  }
  if (((lt - cur) & 1) != 0) v.push_back(++cur);
  while (cur < lt) {
    cur += 2;
    v.push_back(cur);
  }
  return v;
}

namespace {

void shape_cone(const Tables &t, int32_t lb, int32_t lt, int32_t band, int32_t r0, int32_t r1,
                int32_t W, const FusedPlan &fp, const StageFmt &f, ConeShape &cs) {
  const bool from_input = (lb == 0);
  const int32_t sA = fp.acc_size, sB = fp.level_size[lb], sI = fp.input_size;
  const int32_t alignB = f.chunk > 0 ? f.chunk : 16 / sB, alignI = f.chunk > 0 ? f.chunk : 16 / sI;
  const int32_t m = lt - lb;
  cs = ConeShape();
  std::vector<std::vector<Node>> &nodes = cs.nodes;
  nodes.assign(m + 1, {});
  const int32_t hist = f.search_k > 0 ? search_hist(f.search_k) : 0;
  nodes[m].push_back(Node{band, r0, r1, hist, hist});
  for (int32_t l = lt; l > lb; --l) {
    std::vector<Node> &kids = nodes[l - 1 - lb];
    for (Node &p : nodes[l - lb]) {
      p.klo = (int32_t)kids.size();
      if (!has_upper(t, l, p.band)) {
        // Nf not a power of two: a band with no channel above its border
        // passes its lower half's rows up unchanged (same rows, same window).
        kids.push_back(Node{2 * p.band, p.a, p.e, p.o, p.s});
        continue;
      }
      const std::vector<int32_t> &dl = t.dl[l][p.band];
      const int32_t da = dl[p.a], de = dl[p.e];
      kids.push_back(Node{2 * p.band, da, de, p.o, p.s});
      p.khi = (int32_t)kids.size();
      kids.push_back(Node{2 * p.band + 1, p.a - da, p.e - de, p.o + de, p.s + de - da});
    }
  }
  // Row pitch of a staged row whose window needs `need` elements.
  auto pitch = [&](int32_t need, int32_t own_max) -> int32_t {
    if (f.chunk == 0) return (int32_t)round_up(need, f.box);
    return f.kchunks > 0 ? f.kchunks * f.chunk : (int32_t)round_up(own_max, f.chunk);
  };
  int32_t own_max = 0;  // widest staged window of this cone (row blocks, measuring)
  if (from_input && f.chunk > 0) {
    for (const Node &n : nodes[0]) cs.x_o = std::max(cs.x_o, n.o + n.e);
    cs.x_o = (int32_t)ceil_to(cs.x_o, alignI);
    for (const Node &n : nodes[0]) own_max = std::max(own_max, W + n.s + cs.x_o - n.o);
  } else if (!from_input) {
    for (const Node &n : nodes[0]) own_max = std::max(own_max, W + n.s + (int32_t)ceil_to(n.o, alignB) - n.o);
  }
  // Level index i = l - lb for l in [lb, lt).  Only the stored levels of
  // the group's stage sequence take shared memory: the staged base level
  // (S), then the stored computed levels alternately in Pa and Pb.  In a
  // launch from the input, level 0 is never stored (the first stage walks
  // the staged input samples).
  const std::vector<int32_t> st = stored_levels(lb, lt);
  int64_t pa = 0, pb = 0;
  int32_t k = 0;  // index among stored computed levels
  for (int32_t i = 0; i < m; ++i) {
    int64_t off = 0;
    const bool staged = (i == 0 && !from_input);
    const bool stored = !(i == 0 && from_input) &&
                        std::find(st.begin(), st.end(), lb + i) != st.end();
    for (Node &n : nodes[i]) {
      const int32_t rows = n.e - n.a + 1;
      n.delta = 0;
      n.smem = -1;
      if (staged) {
        const int32_t ceil_o = (int32_t)ceil_to(n.o, alignB);
        n.delta = ceil_o - n.o;
        cs.needs.emplace_back(W + n.s + n.delta, n.e - n.a + 1);
        n.stride = pitch(W + n.s + n.delta, own_max);
        n.smem = (int32_t)off;
        off += round_up((int64_t)rows * n.stride * sB, 128);
      } else if (stored) {
        n.stride = (int32_t)round_up(W + n.s, 4);
        n.smem = (int32_t)off;
        off += round_up((int64_t)rows * n.stride * sA, 128);
      }
      if (i == 0 && from_input) {
        if (f.chunk > 0) {
          // One block of consecutive channels, one common window.
          n.xdelta = cs.x_o - n.o;
          n.xstride = pitch(W + n.s + n.xdelta, own_max);
          n.xsmem = (int32_t)cs.s_bytes;
          cs.s_bytes += (int64_t)n.xstride * sI;
        } else {
          const int32_t ceil_oe = (int32_t)ceil_to(n.o + n.e, alignI);
          n.xdelta = ceil_oe - n.o;
          n.xstride = pitch(W + n.s + n.xdelta, 0);
          n.xsmem = (int32_t)cs.s_bytes;
          cs.s_bytes += round_up((int64_t)n.xstride * sI, 128);
        }
        cs.needs.emplace_back(W + n.s + n.xdelta, 1);
      }
    }
    if (i == 0 && from_input) cs.s_bytes = round_up(cs.s_bytes, 128);
    if (staged) {
      cs.s_bytes = off;
    } else if (stored) {
      if ((k & 1) == 0) pa = std::max(pa, off);
      else pb = std::max(pb, off);
      ++k;
    }
  }
  cs.pa_bytes = pa;
  cs.pb_bytes = pb;
  if (f.search_k > 0) {
    // The top rows, W + hist columns each in the search layout (region Pt).
    Node &n = nodes[m].front();
    n.delta = 0;
    n.smem = 0;
    // rows 4 words apart modulo the 32 banks: 16-byte loads of eight rows
    // at the same column hit distinct banks
    n.stride = (int32_t)round_up(search_pidx(W + n.s), 4);
    n.stride += (4 - n.stride % 32 + 32) % 32;
    cs.pt_bytes = round_up((int64_t)(n.e - n.a + 1) * n.stride * sA, 128);
    cs.top_rows = n.e - n.a + 1;
  }
}

// The search's per (row, width) bests of a work item with `rows` top rows
// (one 64-bit word each).
int64_t search_q_bytes(const StageFmt &f, int64_t rows) {
  if (f.search_k <= 0) return 0;
  return round_up(rows * f.search_k * 8, 128);
}

int64_t cone_bytes(const ConeShape &cs) {
  return kBarrierBytes + cs.s_bytes + cs.pa_bytes + cs.pb_bytes + cs.pt_bytes + kDescBytes + kOverRead;
}

// Emits the loads, inits and ops of a shaped cone at the given region bases.
// Row blocks: copies of 2^p rows (p <= max_p) covering rows [0, rows) of a
// block, largest first; calls emit(first row, p).
template <class F>
void row_pieces(int32_t rows, int32_t max_p, F emit) {
  for (int32_t r = 0; r < rows;) {
    int32_t p = max_p;
    while ((1 << p) > rows - r) --p;
    emit(r, p);
    r += 1 << p;
  }
}

// Shared-memory pipe slots (warp instructions, 32 columns each) of one op
// per 32 columns: its loads, the shuffle of a shifted upper half, the store.
double op_slots(int32_t kind, int32_t flags) {
  const double hi = (flags & kOpNoHi) ? 0 : 1;
  if (kind == kStageSingle) return ((flags & kOpLoSame) ? 0 : 1) + hi + 1;
  const double lo = (flags & kOpLoSame) ? 0 : ((flags & kOpLoOne) ? 1 : 2);
  const double up = (flags & kOpNoHi) ? 0 : ((flags & kOpHiShift) ? 1 : ((flags & kOpHiOne) ? 1 : 2));
  return lo + up + 1;
}

// Emits the loads, walks and stage ops of a shaped cone at the given region
// bases.
void emit_cone(const Tables &t, int32_t lb, int32_t lt, int32_t W, const FusedPlan &fp, const StageFmt &f,
               ConeShape &cs, int64_t base_s, int64_t base_a, int64_t base_b, int64_t base_t, ConeOut &c) {
  const bool search = f.search_k > 0;
  const bool from_input = (lb == 0);
  const int32_t sA = fp.acc_size, sB = fp.level_size[lb], sI = fp.input_size;
  const int32_t m = lt - lb;
  std::vector<std::vector<Node>> &nodes = cs.nodes;
  const std::vector<int32_t> st = stored_levels(lb, lt);
  {
    int32_t k = 0;
    for (int32_t i = 0; i < m; ++i) {
      const bool staged = (i == 0 && !from_input);
      bool any = false;
      for (Node &n : nodes[i]) {
        if (n.smem >= 0) {
          any = true;
          n.smem += (int32_t)(staged ? base_s : ((k & 1) == 0 ? base_a : base_b));
        }
        n.xsmem += (int32_t)base_s;
      }
      if (any && !staged) ++k;
    }
    if (search) nodes[m].front().smem += (int32_t)base_t;
  }
  c = ConeOut();
  int64_t tx = 0;
  if (from_input && f.chunk > 0) {
    const Node &n0 = nodes[0].front();
    row_pieces((int32_t)nodes[0].size(), f.max_p, [&](int32_t r, int32_t p) {
      c.loads.push_back(FusedLoad{n0.band + r, n0.xsmem + r * n0.xstride * sI, -cs.x_o, p});
      tx += ((int64_t)n0.xstride * sI) << p;
    });
  }
  if (from_input) {
    if (f.chunk == 0)
      for (const Node &n : nodes[0]) {
        c.loads.push_back(FusedLoad{n.band, n.xsmem, -(int32_t)ceil_to(n.o + n.e, 16 / sI), n.xstride / f.box});
        tx += (int64_t)n.xstride * sI;
      }
  } else {
    for (const Node &n : nodes[0]) {
      const int32_t row0 = t.band_row0[lb][n.band];
      const int32_t xoff = -(int32_t)ceil_to(n.o, f.chunk > 0 ? f.chunk : 16 / sB);
      if (f.chunk > 0) {
        row_pieces(n.e - n.a + 1, f.max_p, [&](int32_t r, int32_t p) {
          c.loads.push_back(FusedLoad{row0 + n.a + r, n.smem + r * n.stride * sB, xoff, p});
          tx += ((int64_t)n.stride * sB) << p;
        });
        continue;
      }
      for (int32_t j = n.a; j <= n.e; ++j) {
        c.loads.push_back(FusedLoad{row0 + j, n.smem + (j - n.a) * n.stride * sB, xoff, n.stride / f.box});
        tx += (int64_t)n.stride * sB;
      }
    }
  }
  c.tpl.tx_bytes = (int32_t)tx;
  c.hbm += (double)tx;
  c.slots += (double)tx / 128.0;  // the copies' writes into shared memory

  // Byte offset of row r, column col (relative to the window start) of a
  // stored node at level index i.
  auto leaf = [&](int32_t i, const Node &n, int32_t r, int32_t col) -> int32_t {
    const int32_t es = (i == 0 && !from_input) ? sB : sA;
    return n.smem + ((r - n.a) * n.stride + n.delta + col) * es;
  };
  auto dlv = [&](int32_t l, int32_t band, int32_t r) { return t.dl[l][band][r]; };

  for (size_t si = 0; si + 1 < st.size(); ++si) {
    const int32_t l1 = st[si + 1];          // level the stage ends on
    const int32_t io = l1 - lb;             // its level index
    const bool top = (l1 == lt);
    const std::vector<Node> &par = nodes[io];
    if (from_input && si == 0) {
      // Level 1 from the staged input: one walk per node, row run and piece.
      c.kinds.push_back(kStageWalk);
      const std::vector<Node> &ch = nodes[0];
      for (size_t pi = 0; pi < par.size(); ++pi) {
        const Node &p = par[pi];
        const bool upper = p.khi >= 0;
        const Node &clo = ch[p.klo], &chi = upper ? ch[p.khi] : ch[p.klo];
        const int32_t de = upper ? dlv(1, p.band, p.e) : 0;
        const int32_t wp = top ? W : W + p.s;
        for (int32_t c0 = 0; c0 < wp; c0 += kPieceCols) {
          for (int32_t ra = p.a; ra <= p.e; ra += 32) {
            const int32_t re = std::min(p.e, ra + 31);
            FusedWalk wk{};
            wk.dst = top ? (t.band_row0[lt][p.band] + ra) : leaf(io, p, ra, c0);
            wk.dst_row = top ? 0 : p.stride * sA;
            wk.x_lo = clo.xsmem + (clo.xdelta + c0) * sI;
            wk.x_hi = chi.xsmem + (chi.xdelta + c0 + de) * sI;
            wk.width = std::min(kPieceCols, wp - c0);
            wk.col = c0;
            wk.a = ra;
            wk.e = re;
            wk.dl0 = dlv(1, p.band, ra);
            wk.bits = 0;
            double sl = (wk.dl0 + 1) + (ra - wk.dl0 + 1) + 1;
            for (int32_t r = ra + 1; r <= re; ++r) {
              const int32_t inc = dlv(1, p.band, r) - dlv(1, p.band, r - 1);
              if (inc) wk.bits |= 1 << (r - ra - 1);
              sl += 1 + inc + 1;
            }
            wk.chan = clo.band;
            wk.flags = upper ? 0 : kWalkNoUpper;
            c.walks.push_back(wk);
            c.slots += sl * kLaneCols;
            c.nops += 1;
            if (top) c.hbm += (double)std::min(kPieceCols, W - c0) * (re - ra + 1) * fp.level_size[lt];
          }
        }
      }
      continue;
    }
    const bool pair = (l1 - st[si] == 2);
    const int32_t kind = pair ? kStagePair : kStageSingle;
    // With a search the top level goes to Pt (search layout), all W + hist
    // columns; otherwise to global memory, W columns.
    const bool to_global = top && !search;
    c.kinds.push_back(kind | (top && search ? kStagePadded : 0));
    std::vector<FusedOp> ops;
    const int32_t wmax = to_global ? W : [&] {
      int32_t v = 0;
      for (const Node &p : par) v = std::max(v, W + p.s);
      return v;
    }();
    for (int32_t c0 = 0; c0 < wmax; c0 += kPieceCols) {
      for (size_t pi = 0; pi < par.size(); ++pi) {
        const Node &p = par[pi];
        const int32_t wp = to_global ? W : W + p.s;
        if (c0 >= wp) continue;
        const int32_t width = std::min(kPieceCols, wp - c0);
        const bool upper = p.khi >= 0;
        const int32_t de = dlv(l1, p.band, p.e);
        const std::vector<Node> &kid = nodes[io - 1];
        const Node &klo = kid[p.klo], &khi = upper ? kid[p.khi] : kid[p.klo];
        int32_t pj = -1, pm = -1;
        for (int32_t dt = p.a; dt <= p.e; ++dt) {
          // (a band without an upper half has dl = dt: row dt is its lower row dt)
          const int32_t j = dlv(l1, p.band, dt), mrow = dt - j, q = de - j;
          FusedOp op{};
          if (to_global)
            op.dst = t.band_row0[lt][p.band] + dt;
          else if (top)  // Pt: the row's base plus the piece's first column in the search layout
            op.dst = p.smem + ((dt - p.a) * p.stride + search_pidx(c0)) * sA;
          else
            op.dst = leaf(io, p, dt, c0);
          op.width = width;
          op.col = c0;
          op.flags = 0;
          if (!pair) {
            op.p0 = leaf(io - 1, klo, j, c0);
            if (upper) op.p1 = leaf(io - 1, khi, mrow, c0 + q);
            else op.flags |= kOpNoHi;
          } else {
            // klo / khi are not stored: expand them into their halves (one
            // term where a half passes its lower rows up).
            const std::vector<Node> &g = nodes[io - 2];
            const int32_t l0 = l1 - 1;
            if (klo.khi >= 0) {
              const int32_t j1 = dlv(l0, klo.band, j), q1 = dlv(l0, klo.band, klo.e) - j1;
              op.p0 = leaf(io - 2, g[klo.klo], j1, c0);
              op.p1 = leaf(io - 2, g[klo.khi], j - j1, c0 + q1);
            } else {
              op.p0 = leaf(io - 2, g[klo.klo], j, c0);
              op.flags |= kOpLoOne;
            }
            if (!upper) {
              op.flags |= kOpNoHi;
            } else if (khi.khi >= 0) {
              const int32_t j2 = dlv(l0, khi.band, mrow), q2 = dlv(l0, khi.band, khi.e) - j2;
              op.p2 = leaf(io - 2, g[khi.klo], j2, c0 + q);
              op.p3 = leaf(io - 2, g[khi.khi], mrow - j2, c0 + q + q2);
            } else {
              op.p2 = leaf(io - 2, g[khi.klo], mrow, c0 + q);
              op.flags |= kOpHiOne;
            }
          }
          if (dt > p.a && j == pj) op.flags |= kOpLoSame;
          if (pair && upper && dt > p.a && mrow == pm && j == pj + 1) op.flags |= kOpHiShift;
          pj = j;
          pm = mrow;
          ops.push_back(op);
          c.slots += op_slots(kind, op.flags) * kLaneCols;
          c.nops += 1;
          if (to_global) c.hbm += (double)width * fp.level_size[lt];
        }
      }
    }
    c.stage_ops.push_back(std::move(ops));
  }
  if (search) {
    // One search op per top row: the row in Pt, its global row, the W
    // owned columns after hist columns of history.
    c.kinds.push_back(kStageSearch);
    std::vector<FusedOp> ops;
    const Node &p = nodes[m].front();
    for (int32_t dt = p.a; dt <= p.e; ++dt) {
      FusedOp op{};
      op.dst = t.band_row0[lt][p.band] + dt;
      op.p0 = p.smem + (dt - p.a) * p.stride * sA;
      op.width = W;
      op.col = p.s;
      ops.push_back(op);
      c.slots += 6.0 * (W + p.s) / 32;
      c.nops += 1;
      c.hbm += (double)W * fp.level_size[lt];
    }
    c.stage_ops.push_back(std::move(ops));
  }
  c.tpl.n_stages = (int32_t)c.kinds.size();
}

// Splits a stage's ops (or walks) into kFusedBlockWarps contiguous runs of
// about equal cost; returns the first index of each run and the end.
std::vector<int32_t> split_warps(const std::vector<double> &cost) {
  double total = 0;
  for (double v : cost) total += v;
  std::vector<int32_t> b(kFusedBlockWarps + 1, (int32_t)cost.size());
  b[0] = 0;
  double acc = 0;
  int32_t w = 1;
  for (int32_t i = 0; i < (int32_t)cost.size() && w < kFusedBlockWarps; ++i) {
    acc += cost[i];
    while (w < kFusedBlockWarps && acc >= total * w / kFusedBlockWarps) b[w++] = i + 1;
  }
  for (; w < kFusedBlockWarps; ++w) b[w] = (int32_t)cost.size();
  return b;
}

// One work item (template): the cones of a bundle, their stage ops merged
// and split over the warps.  Stage offsets are relative to the item's walks
// and ops until the group is appended to the plan.
struct ItemOut {
  FusedTemplate tpl{};
  std::vector<FusedLoad> loads;
  std::vector<FusedWalk> walks;
  std::vector<FusedOp> ops;
  std::vector<int32_t> stages;  // kStageWords per stage
  double hbm = 0, slots = 0, nops = 0;
};

struct GroupBuild {
  bool ok = false;
  FusedGroup g;
  std::vector<ItemOut> cones;
  double seconds = 0;
};

// All cones of group (lb, lt] for tile W: each band of level lt is split
// into the fewest equal row ranges whose cones fit `budget`; the cones are
// then laid out at the group's region bases.  The group total can exceed the
// per-cone budget slightly (maxima of different cones); the budget is
// lowered until the total fits.
// TMA box width for staged rows with the given (window, rows) needs, of
// `es`-byte elements: a multiple of 128 bytes (every copy lands 128-byte
// aligned in shared memory) and at most 256 elements, chosen to minimise
// the copied bytes plus a fixed cost per copy (a copy's issue and
// completion cost about as much as moving kCopyBytes more).
constexpr int64_t kCopyBytes = 1024;
int32_t choose_box(const std::vector<std::pair<int32_t, int32_t>> &needs, int32_t es) {
  const int32_t q = 128 / es;
  int32_t best = 0;
  int64_t best_cost = std::numeric_limits<int64_t>::max();
  for (int32_t box = q; box <= 256; box += q) {
    int64_t cost = 0;
    for (const auto &nr : needs) {
      const int64_t nbox = (nr.first + box - 1) / box;
      cost += nr.second * nbox * ((int64_t)box * es + kCopyBytes);
    }
    if (cost < best_cost) {
      best_cost = cost;
      best = box;
    }
  }
  return best;
}

GroupBuild build_group_fmt(const Tables &t, int64_t nt, int32_t lb, int32_t lt, int32_t W,
                           const FusedPlan &fp, int32_t budget, const StageFmt &f,
                           std::vector<std::pair<int32_t, int32_t>> *needs) {
  GroupBuild gb;
  const int32_t nb = bands_at(t.nf, lt);
  for (int32_t cone_budget = budget; cone_budget >= 4096; cone_budget = cone_budget * 7 / 8) {
    std::vector<ConeShape> shapes;
    bool ok = true;
    for (int32_t b = 0; b < nb && ok; ++b) {
      const int32_t rows = t.band_rows[lt][b];
      auto fits = [&](int32_t per, std::vector<ConeShape> *keep) {
        for (int32_t r0 = 0; r0 < rows; r0 += per) {
          ConeShape cs;
          shape_cone(t, lb, lt, b, r0, std::min(rows, r0 + per) - 1, W, fp, f, cs);
          if (cone_bytes(cs) + search_q_bytes(f, cs.top_rows) > cone_budget) return false;
          if (keep) keep->push_back(std::move(cs));
        }
        return true;
      };
      int32_t lo = 0, hi = rows;
      if (fits(rows, nullptr)) {
        lo = rows;
      } else {
        while (hi - lo > 1) {
          const int32_t mid = lo + (hi - lo) / 2;
          if (fits(std::max(mid, 1), nullptr)) lo = mid; else hi = mid;
        }
      }
      if (lo < 1) {
        ok = false;
        break;
      }
      const int32_t parts = (rows + lo - 1) / lo;
      const int32_t per = (rows + parts - 1) / parts;
      ok = fits(per, &shapes);
    }
    if (!ok) return gb;  // even single rows do not fit
    // Work items: runs of consecutive cones that fit the budget together
    // (their regions stacked), so that small cones share the per-item cost;
    // at most as many per item as leaves two items per block slot.
    const int64_t ntiles = (nt + W - 1) / W;
    const int64_t cap = std::max<int64_t>(
        1, (int64_t)shapes.size() * ntiles / (int64_t)(2 * kSms * kMaxBlocksPerSm));
    std::vector<std::vector<int32_t>> bundles;
    int64_t bs = 0, ba = 0, bb = 0, bt = 0, br = 0;
    for (int32_t i = 0; i < (int32_t)shapes.size(); ++i) {
      const ConeShape &cs = shapes[i];
      if (!bundles.empty() && (int64_t)bundles.back().size() < cap &&
          kBarrierBytes + bs + cs.s_bytes + ba + cs.pa_bytes + bb + cs.pb_bytes + bt + cs.pt_bytes +
                  search_q_bytes(f, br + cs.top_rows) + kDescBytes + kOverRead <= cone_budget) {
        bundles.back().push_back(i);
        bs += cs.s_bytes;
        ba += cs.pa_bytes;
        bb += cs.pb_bytes;
        bt += cs.pt_bytes;
        br += cs.top_rows;
      } else {
        bundles.push_back({i});
        bs = cs.s_bytes;
        ba = cs.pa_bytes;
        bb = cs.pb_bytes;
        bt = cs.pt_bytes;
        br = cs.top_rows;
      }
    }
    int64_t ms = 0, ma = 0, mb = 0, mt = 0, mr = 0;
    for (const std::vector<int32_t> &bu : bundles) {
      int64_t s1 = 0, a1 = 0, b1 = 0, t1 = 0, r1 = 0;
      for (int32_t i : bu) {
        s1 += shapes[i].s_bytes;
        a1 += shapes[i].pa_bytes;
        b1 += shapes[i].pb_bytes;
        t1 += shapes[i].pt_bytes;
        r1 += shapes[i].top_rows;
      }
      ms = std::max(ms, s1);
      ma = std::max(ma, a1);
      mb = std::max(mb, b1);
      mt = std::max(mt, t1);
      mr = std::max(mr, r1);
    }
    const int64_t qb = search_q_bytes(f, mr);
    const int64_t total = kBarrierBytes + ms + ma + mb + mt + qb + kDescBytes + kOverRead;
    if (total > budget && total > 227 * 1024 - 1024) continue;
    if (total > budget && cone_budget > 4096) continue;
    gb = GroupBuild();
    gb.g.lb = lb;
    gb.g.lt = lt;
    gb.g.W = W;
    gb.g.in_size = (lb == 0) ? fp.input_size : fp.level_size[lb];
    gb.g.out_size = fp.level_size[lt];
    gb.g.box = f.box;
    gb.g.chunk = f.chunk;
    gb.g.kchunks = f.kchunks;
    gb.g.max_p = f.max_p;
    gb.g.from_input = (lb == 0);
    gb.g.search_k = f.search_k;
    gb.g.hist = f.search_k > 0 ? search_hist(f.search_k) : 0;
    gb.g.q_off = (int32_t)(kBarrierBytes + ms + ma + mb + mt);
    gb.g.q_row = (int32_t)qb;
    gb.g.ntiles = (nt + W - 1) / W;
    gb.g.smem_bytes = (int32_t)total;
    gb.g.s_end = (int32_t)(kBarrierBytes + ms);
    gb.g.pa_end = (int32_t)(kBarrierBytes + ms + ma);
    double hbm = 0, sl = 0, nops = 0;
    for (const std::vector<int32_t> &bu : bundles) {
      // Each cone of the item gets its own slice of S, Pa and Pb; the item's
      // stage ops are merged stage by stage, then split over the warps.
      ItemOut item;
      int64_t so = 0, ao = 0, bo = 0, to = 0;
      std::vector<ConeOut> cos;
      for (int32_t i : bu) {
        ConeShape &cs = shapes[i];
        if (needs) needs->insert(needs->end(), cs.needs.begin(), cs.needs.end());
        ConeOut c;
        emit_cone(t, lb, lt, W, fp, f, cs, kBarrierBytes + so, kBarrierBytes + ms + ao,
                  kBarrierBytes + ms + ma + bo, kBarrierBytes + ms + ma + mb + to, c);
        so += cs.s_bytes;
        ao += cs.pa_bytes;
        bo += cs.pb_bytes;
        to += cs.pt_bytes;
        item.loads.insert(item.loads.end(), c.loads.begin(), c.loads.end());
        item.tpl.tx_bytes += c.tpl.tx_bytes;
        item.hbm += c.hbm;
        item.slots += c.slots;
        item.nops += c.nops;
        cos.push_back(std::move(c));
      }
      const std::vector<int32_t> &kinds = cos.front().kinds;
      for (size_t si = 0; si < kinds.size(); ++si) {
        std::vector<double> cost;
        int32_t base;
        if ((kinds[si] & kStageKindMask) == kStageWalk) {
          base = (int32_t)item.walks.size();
          for (const ConeOut &c : cos)
            for (const FusedWalk &wk : c.walks) {
              item.walks.push_back(wk);
              cost.push_back(3.0 * (wk.e - wk.a + 1 + wk.dl0) * kLaneCols + 2.0);
            }
        } else {
          base = (int32_t)item.ops.size();
          const size_t k = (lb == 0) ? si - 1 : si;
          const int32_t kind = kinds[si] & kStageKindMask;
          for (const ConeOut &c : cos)
            for (const FusedOp &op : c.stage_ops[k]) {
              item.ops.push_back(op);
              // an op loads and stores whole pieces whatever its width
              cost.push_back(kind == kStageSearch ? 1.0 : op_slots(kind, op.flags) * kLaneCols + 2.0);
            }
        }
        const std::vector<int32_t> b = split_warps(cost);
        bool general = false;
        if ((kinds[si] & kStageKindMask) == kStageWalk) {
          for (size_t i = (size_t)base; i < item.walks.size(); ++i) general |= (item.walks[i].flags & kWalkNoUpper) != 0;
        } else {
          for (size_t i = (size_t)base; i < item.ops.size(); ++i)
            general |= (item.ops[i].flags & (kOpLoOne | kOpHiOne | kOpNoHi)) != 0;
        }
        item.stages.push_back(kinds[si] | (general ? kStageGeneral : 0));
        for (int32_t w = 0; w <= kFusedBlockWarps; ++w) {
          item.stages.push_back(base + b[w]);
          // A warp's first op has nothing earlier to reuse.
          if ((kinds[si] & kStageKindMask) != kStageWalk && w < kFusedBlockWarps && b[w] < b[w + 1])
            item.ops[base + b[w]].flags &= ~(kOpLoSame | kOpHiShift);
        }
      }
      item.tpl.n_stages = (int32_t)kinds.size();
      item.tpl.smem_bytes = (int32_t)total;
      hbm += item.hbm;
      sl += item.slots;
      nops += item.nops;
      gb.cones.push_back(std::move(item));
    }
    gb.g.hbm_bytes = hbm * (double)gb.g.ntiles;
    gb.g.smem_traffic = sl * 128.0 * (double)gb.g.ntiles;
    const double tiles = (double)gb.g.ntiles;
    const double items = (double)gb.cones.size() * tiles;
    const double slots =
        kSms * std::min(kMaxBlocksPerSm, std::max(1.0, std::floor((228.0 * 1024) / (total + 1024.0))));
    const double on_chip = sl * tiles * kSlotSeconds +
                           (items * kItemSeconds + nops * tiles * kOpSeconds) / slots + kLaunchSeconds;
    // DRAM sees each base row and each output row once (neighbouring cones'
    // halos and overlaps are L2 hits); the staged bytes go through L2.
    const double unique = (double)nt * ((lb == 0 ? (double)t.nf * fp.input_size
                                                  : (double)t.level_rows[lb] * fp.level_size[lb]) +
                                        (double)t.level_rows[lt] * fp.level_size[lt]);
    gb.seconds = std::max({unique / kHbmRate, gb.g.hbm_bytes / kL2Rate, on_chip});
    gb.g.ops = nops * tiles;
    gb.g.block_slots = slots;
    gb.g.seconds = gb.seconds;
    gb.ok = true;
    return gb;
  }
  return gb;
}

// Group (lb, lt] for tile W.  The staging format follows the windows of
// the group's own cones: a first build with provisional boxes measures
// them, the second uses the chosen box or block width.
GroupBuild build_group(const Tables &t, int64_t nt, int32_t lb, int32_t lt, int32_t W,
                       const FusedPlan &fp, int32_t budget, int32_t staging, int32_t search_k) {
  const int32_t es = (lb == 0) ? fp.input_size : fp.level_size[lb];
  const int64_t rows = (lb == 0) ? t.nf : t.level_rows[lb];
  // Row blocks: chunks of 128 bytes (64 for 1-byte samples, so that a tile
  // start, a multiple of 64 samples, is a chunk boundary).
  const int32_t chunk = std::min(128 / es, 64);
  const bool blocks = staging != 1 && nt % chunk == 0;
  if (staging == 2 && !blocks) return GroupBuild();
  StageFmt f;
  f.search_k = search_k;
  if (blocks) {
    f.chunk = chunk;
    f.max_p = 0;
    while (f.max_p < 5 && (int64_t(2) << f.max_p) <= rows) ++f.max_p;
  } else {
    f.box = 128 / es;
  }
  std::vector<std::pair<int32_t, int32_t>> needs;
  GroupBuild gb = build_group_fmt(t, nt, lb, lt, W, fp, budget, f, &needs);
  if (!gb.ok) return gb;
  int32_t widest = 0;
  for (const auto &nr : needs) widest = std::max(widest, nr.first);
  if (blocks) {
    // Every staged row of the launch gets the widest window; a copy's row
    // pitch stays a multiple of 128 bytes.  The cones of the rebuilt group
    // can differ (other row splits, other window alignments), so the width
    // is checked again and widened until it covers all of them.
    for (int iter = 0; iter < 4; ++iter) {
      int32_t k = (widest + chunk - 1) / chunk;
      while ((k * chunk * es) % 128 != 0) ++k;
      if (k > 256 || (int64_t)k * chunk > nt) break;
      f.kchunks = std::max(f.kchunks, k);
      std::vector<std::pair<int32_t, int32_t>> got;
      GroupBuild g2 = build_group_fmt(t, nt, lb, lt, W, fp, budget, f, &got);
      if (!g2.ok) break;
      widest = 0;
      for (const auto &nr : got) widest = std::max(widest, nr.first);
      if (widest <= f.kchunks * chunk) return g2;
    }
    if (staging == 2) return GroupBuild();
    f = StageFmt();  // fall back to row boxes
    f.search_k = search_k;
    f.box = 128 / es;
    needs.clear();
    gb = build_group_fmt(t, nt, lb, lt, W, fp, budget, f, &needs);
    if (!gb.ok) return gb;
  }
  f.box = choose_box(needs, es);
  return build_group_fmt(t, nt, lb, lt, W, fp, budget, f, nullptr);
}

void append_group(FusedPlan &fp, GroupBuild &gb) {
  FusedGroup g = gb.g;
  g.tpl_begin = (int32_t)fp.tpls.size();
  g.tpl_count = (int32_t)gb.cones.size();
  for (ItemOut &c : gb.cones) {
    FusedTemplate tp = c.tpl;
    tp.load_begin = (int32_t)fp.loads.size();
    tp.load_count = (int32_t)c.loads.size();
    tp.walk_begin = (int32_t)fp.walks.size();
    tp.walk_count = (int32_t)c.walks.size();
    tp.stage_begin = (int32_t)fp.stages.size();
    const int32_t w0 = (int32_t)fp.walks.size(), o0 = (int32_t)fp.ops.size();
    for (size_t i = 0; i < c.stages.size(); i += kStageWords) {
      const int32_t off = (c.stages[i] & kStageKindMask) == kStageWalk ? w0 : o0;
      fp.general |= (c.stages[i] & kStageGeneral) != 0;
      fp.stages.push_back(c.stages[i]);
      for (int32_t w = 1; w < kStageWords; ++w) fp.stages.push_back(c.stages[i + w] + off);
    }
    fp.loads.insert(fp.loads.end(), c.loads.begin(), c.loads.end());
    fp.walks.insert(fp.walks.end(), c.walks.begin(), c.walks.end());
    fp.ops.insert(fp.ops.end(), c.ops.begin(), c.ops.end());
    fp.tpls.push_back(tp);
  }
  fp.groups.push_back(g);
}

}  // namespace

std::string plan_fused(const Tables &t, int64_t nt, int32_t state_size, int32_t input_size,
                       const FusedParams &p, FusedPlan &out) {
  const int32_t L = t.levels;
  std::vector<int32_t> widths;
  if (p.W > 0) {
    if (p.W % 64 != 0) return "tile width must be a multiple of 64";
    widths.push_back(p.W);
  } else {
    widths = {128, 256, 384, 448, 512, 960, 1024};
  }
  if (p.search_k < 0 || p.search_k > kSearchMaxWidths || (p.search_k > 0 && L < 2))
    return "the search in the last launch takes 1 .. 9 widths and at least two merge levels";
  if (p.search_k > 0 && p.W > 0 && p.W + search_hist(p.search_k) > 16 * kFusedBlockWarps * 32)
    return "the searched window must fit one wave of the block";
  FusedPlan fp;
  fp.state_size = state_size;
  fp.input_size = input_size;
  fp.acc_size = 4;
  // Stored element size of each level at a launch boundary; the output
  // (level L) is 4 bytes.  With p.narrow (integer sums of uint8 samples), a
  // level whose sums stay below 2^16 is stored as uint16: row Dt of a band
  // of 2^l channels sums 2^l + Dt samples (the path's sample counts
  // telescope, section 4), each at most 255.
  fp.level_size.assign(L + 1, state_size);
  fp.level_size[L] = 4;
  if (p.narrow) {
    for (int32_t l = 1; l < L; ++l) {
      int32_t rmax = 0;
      for (int32_t r : t.band_rows[l]) rmax = std::max(rmax, r);
      if (255LL * ((1LL << l) + rmax - 1) <= 65535 && (nt * 2) % 16 == 0) fp.level_size[l] = 2;
    }
  }
  // Best tile for one group (lb, lt] (optionally a given tile and budget).
  auto best_segment = [&](int32_t lb, int32_t lt, int32_t forced_W = 0, int32_t budget = 0) {
    GroupBuild best;
    const std::vector<int32_t> ws = forced_W > 0 ? std::vector<int32_t>{forced_W} : widths;
    for (int32_t W : ws) {
      GroupBuild gb = build_group(t, nt, lb, lt, W, fp, budget > 0 ? budget : p.smem_budget, p.staging,
                                  lt == L ? p.search_k : 0);
      if (gb.ok && (!best.ok || gb.seconds < best.seconds)) best = std::move(gb);
    }
    return best;
  };
  std::vector<int32_t> bounds = p.bounds;
  if (bounds.empty()) {
    // Dynamic programming over boundaries: cost[j] = best time to reach level j.
    std::vector<double> cost(L + 1, std::numeric_limits<double>::infinity());
    std::vector<int32_t> from(L + 1, -1);
    cost[0] = 0;
    for (int32_t j = 1; j <= L; ++j)
      for (int32_t i = std::max(0, j - 6); i < j; ++i) {
        if (!std::isfinite(cost[i])) continue;
        GroupBuild gb = best_segment(i, j);
        if (!gb.ok) continue;
        if (cost[i] + gb.seconds < cost[j]) {
          cost[j] = cost[i] + gb.seconds;
          from[j] = i;
        }
      }
    if (!std::isfinite(cost[L])) return "no fused schedule fits the shared-memory budget";
    std::vector<int32_t> rev;
    for (int32_t j = L; j > 0; j = from[j]) rev.push_back(j);
    bounds = {0};
    for (auto it = rev.rbegin(); it != rev.rend(); ++it) bounds.push_back(*it);
  }
  if (bounds.size() < 2 || bounds.front() != 0 || bounds.back() != L)
    return "level boundaries must run from 0 to L";
  double secs = 0;
  for (size_t i = 0; i + 1 < bounds.size(); ++i) {
    if (bounds[i + 1] <= bounds[i]) return "level boundaries must increase";
    const int32_t gw = i < p.group_W.size() ? p.group_W[i] : 0;
    const int32_t gbud = i < p.group_budget.size() ? p.group_budget[i] : 0;
    if (gw < 0 || gw % 64 != 0 || gbud < 0 || gbud > 227 * 1024) return "bad per-group parameters";
    GroupBuild gb = best_segment(bounds[i], bounds[i + 1], gw, gbud);
    if (!gb.ok) return "a level group does not fit the shared-memory budget";
    secs += gb.seconds;
    append_group(fp, gb);
  }
  fp.W = fp.groups.front().W;
  fp.model_seconds = secs;
  // Intermediate states between groups: group g writes buffer g % 2.
  size_t even = 0, odd = 0;
  for (size_t g = 0; g + 1 < fp.groups.size(); ++g) {
    const size_t bytes = (size_t)t.level_rows[fp.groups[g].lt] * (size_t)nt * (size_t)fp.level_size[fp.groups[g].lt];
    if (g & 1) odd = std::max(odd, bytes); else even = std::max(even, bytes);
  }
  fp.ws_split = (size_t)round_up((int64_t)even, 256);
  fp.ws_bytes = fp.ws_split + (size_t)round_up((int64_t)odd, 256);
  out = std::move(fp);
  return "";
}

}  // namespace fdmt
