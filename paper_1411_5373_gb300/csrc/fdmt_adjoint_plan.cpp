// Planner of the fused adjoint schedule (pull cones, see
// fdmt_adjoint_fused.h): which levels each launch covers, the row ranges of
// its work items, and for every item its TMA copies and gather ops.
#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "fdmt_adjoint_fused.h"

namespace fdmt {

namespace {

constexpr int32_t kAdjBarrierBytes = 128;  // mbarrier slot; regions stay 128-byte aligned
constexpr int32_t kAdjBox = 64;            // TMA box width of the staged rows (elements)
constexpr int64_t kAdjMaxSmem = 227 * 1024;
constexpr int32_t kAdjChunk = 32;          // row blocks: chunks of 128 bytes

int64_t rup(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// A band of the subtree under one band B of level lt.  Index i = lt - level.
struct SubBand {
  int32_t band = 0;   // band index at its level
  int32_t kind = 0;   // below the top: 0 lower half, 1 upper half, 2 passed down (no upper half)
  int32_t parent = -1;
  int32_t lo = -1, hi = -1;  // children at the level below (hi < 0: none)
  std::vector<int32_t> rs, re;  // below the top: the run of parent rows each row reads
  std::vector<int32_t> ts, te;  // the run of level-lt rows (composed down the levels)
};

using Subtree = std::vector<std::vector<SubBand>>;

std::string build_subtree(const Tables &t, int32_t lt, int32_t lb, int32_t B, Subtree &st) {
  const int32_t m = lt - lb;
  st.assign(m + 1, {});
  SubBand top;
  top.band = B;
  const int32_t R = t.band_rows[lt][B];
  top.ts.resize(R);
  top.te.resize(R);
  for (int32_t r = 0; r < R; ++r) top.ts[r] = top.te[r] = r;
  st[0].push_back(top);
  for (int32_t i = 0; i < m; ++i) {
    const int32_t l = lt - i;
    for (int32_t k = 0; k < (int32_t)st[i].size(); ++k) {
      const int32_t b = st[i][k].band;
      const int32_t rows = t.band_rows[l][b];
      const std::vector<int32_t> &dl = t.dl[l][b];
      auto add = [&](int32_t kind, int32_t cband, int32_t crows) {
        SubBand c;
        c.band = cband;
        c.kind = kind;
        c.parent = k;
        c.rs.assign(crows, -1);
        c.re.assign(crows, -1);
        for (int32_t d = 0; d < rows; ++d) {
          const int32_t x = kind == 0 ? dl[d] : kind == 1 ? d - dl[d] : d;
          if (x < 0 || x >= crows) return std::string("internal: child row out of range");
          if (c.rs[x] < 0) c.rs[x] = d;
          c.re[x] = d;
        }
        for (int32_t x = 0; x < crows; ++x)
          if (c.rs[x] < 0) return std::string("internal: child row never read");
        c.ts.resize(crows);
        c.te.resize(crows);
        const SubBand &p = st[i][k];
        for (int32_t x = 0; x < crows; ++x) {
          c.ts[x] = p.ts[c.rs[x]];
          c.te[x] = p.te[c.re[x]];
        }
        st[i + 1].push_back(std::move(c));
        return std::string();
      };
      std::string err;
      if (has_upper(t, l, b)) {
        st[i][k].lo = (int32_t)st[i + 1].size();
        err = add(0, 2 * b, t.band_rows[l - 1][2 * b]);
        if (!err.empty()) return err;
        st[i][k].hi = (int32_t)st[i + 1].size();
        err = add(1, 2 * b + 1, t.band_rows[l - 1][2 * b + 1]);
      } else {
        st[i][k].lo = (int32_t)st[i + 1].size();
        if (t.band_rows[l - 1][2 * b] != rows) return "internal: passed-down band changes its rows";
        err = add(2, 2 * b, rows);
      }
      if (!err.empty()) return err;
    }
  }
  return "";
}

// One node of a shaped cone: the rows [a, e] of its band that the item
// needs, its window [T0 + o, T0 + o + need), where it lives in shared memory.
struct TNode {
  int32_t a = 0, e = -1;
  int32_t o = 0, need = 0;
  int32_t dls = 0;     // upper half: dl of the first parent row its runs read
  int32_t smem = 0, stride = 0;
  bool empty() const { return e < a; }
};

struct Shape {
  std::vector<std::vector<TNode>> nodes;  // [i][k] as the subtree
  int64_t s_bytes = 0, pa_bytes = 0, pb_bytes = 0;
  bool any = false;  // the item owns something
};

// Shapes the cone of top rows [r0, r1] (region-relative offsets).
// fuse: the launch folds the level 1 -> 0 gather into the initialisation
// transpose (level 0 is never stored).
void shape(const Tables &t, const Subtree &st, int32_t lt, int32_t lb, bool init, bool fuse, int32_t r0,
           int32_t r1, int32_t W, int32_t pitch, Shape &sh) {
  const int32_t m = lt - lb;
  sh = Shape();
  sh.nodes.resize(m + 1);
  for (int32_t i = 0; i <= m; ++i) sh.nodes[i].resize(st[i].size());
  // Owned rows of level lb.
  for (size_t k = 0; k < st[m].size(); ++k) {
    const SubBand &s = st[m][k];
    TNode &n = sh.nodes[m][k];
    if (init) {
      // a channel: all its level-0 rows, owned with its row 0
      if (s.ts[0] >= r0 && s.ts[0] <= r1) {
        n.a = 0;
        n.e = (int32_t)s.ts.size() - 1;
        n.need = W + n.e;  // the transpose reads rows j at tau + i, i <= j
      }
    } else {
      n.a = (int32_t)(std::lower_bound(s.ts.begin(), s.ts.end(), r0) - s.ts.begin());
      n.e = (int32_t)(std::upper_bound(s.ts.begin(), s.ts.end(), r1) - s.ts.begin()) - 1;
      n.need = W;
    }
    if (!n.empty()) sh.any = true;
  }
  // Needed rows and widths, bottom-up.
  for (int32_t i = m - 1; i >= 0; --i) {
    const int32_t l = lt - i;
    for (size_t k = 0; k < st[i].size(); ++k) {
      const SubBand &s = st[i][k];
      TNode &n = sh.nodes[i][k];
      n.a = INT32_MAX;
      n.e = -1;
      n.need = 0;
      for (int32_t c : {s.lo, s.hi}) {
        if (c < 0) continue;
        const SubBand &cs = st[i + 1][c];
        TNode &cn = sh.nodes[i + 1][c];
        if (cn.empty()) continue;
        const int32_t pa = cs.rs[cn.a], pe = cs.re[cn.e];
        n.a = std::min(n.a, pa);
        n.e = std::max(n.e, pe);
        int32_t w = cn.need;
        if (cs.kind == 1) {
          cn.dls = t.dl[l][s.band][pa];
          w += t.dl[l][s.band][pe] - cn.dls;
        }
        n.need = std::max(n.need, w);
      }
      if (n.e < 0) n.a = 0;
    }
  }
  // Window starts, top-down.
  for (int32_t i = 0; i < m; ++i)
    for (size_t k = 0; k < st[i].size(); ++k) {
      const SubBand &s = st[i][k];
      for (int32_t c : {s.lo, s.hi}) {
        if (c < 0) continue;
        TNode &cn = sh.nodes[i + 1][c];
        cn.o = sh.nodes[i][k].o - (st[i + 1][c].kind == 1 ? cn.dls : 0);
      }
    }
  // Shared memory: the staged top rows in S; the stored levels (every level
  // between, and level 0 of a launch that applies the initialisation
  // transpose) alternately in Pa and Pb.
  // (row blocks: every staged row has the launch's pitch; a cone wider
  // than it does not fit)
  TNode &top = sh.nodes[0][0];
  if (!top.empty()) {
    top.stride = pitch > 0 ? pitch : (int32_t)rup(top.need, kAdjBox);
    top.smem = 0;
    sh.s_bytes = top.need > top.stride ? (int64_t)1 << 40
                                       : rup((int64_t)(top.e - top.a + 1) * top.stride * 4, 128);
  }
  for (int32_t i = 1; i <= m; ++i) {
    if (i == m && (!init || fuse)) break;
    int64_t off = 0;
    for (TNode &n : sh.nodes[i]) {
      if (n.empty()) continue;
      n.stride = (int32_t)rup(n.need, 4);
      n.smem = (int32_t)off;
      off += rup((int64_t)(n.e - n.a + 1) * n.stride * 4, 128);
    }
    int64_t &region = ((i - 1) & 1) == 0 ? sh.pa_bytes : sh.pb_bytes;
    region = std::max(region, off);
  }
}

int64_t shape_bytes(const Shape &sh) {
  return kAdjBarrierBytes + sh.s_bytes + sh.pa_bytes + sh.pb_bytes + kDescBytes + kOverRead;
}

// The wait of an init op for its input samples, in the cost's units
// (shared-memory slots per lane group), for the warp split only.
constexpr double kInitOpWait = 64.0;

// The folded init op (kAdjInitF) describes a channel's level-0 rows by the
// lengths of their level-1 runs, 4 bits each in the op's flags.
constexpr int32_t kInitFMaxRows = 7, kInitFMaxRun = 15;

// Whether every channel's level-0 rows fit the folded op: the runs of
// level-1 rows its rows read (dl for a lower half, row - dl for an upper
// half, one row each for a band passed down).
bool init_fusable(const Tables &t) {
  if (t.levels < 1) return false;
  for (int32_t b = 0; b < (int32_t)t.band_rows[1].size(); ++b) {
    const int32_t rows = t.band_rows[1][b];
    const std::vector<int32_t> &dl = t.dl[1][b];
    const bool up = has_upper(t, 1, b);
    for (int32_t half = 0; half < (up ? 2 : 1); ++half) {
      const int32_t crows = !up ? rows : t.band_rows[0][2 * b + half];
      if (crows > kInitFMaxRows) return false;
      std::vector<int32_t> cnt(crows, 0);
      for (int32_t d = 0; d < rows; ++d) {
        const int32_t x = !up ? d : half == 0 ? dl[d] : d - dl[d];
        if (x < 0 || x >= crows) return false;
        if (++cnt[x] > kInitFMaxRun) return false;
      }
    }
  }
  return true;
}

std::vector<int32_t> balance_warps(const std::vector<double> &cost) {
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

// Appends the template of a shaped cone (offsets rebased on the group's
// regions) to the plan.
void emit(const Tables &t, const Subtree &st, int32_t lt, int32_t lb, bool init, bool fuse, int32_t W, Shape sh,
          int32_t s_base, int32_t pa_base, int32_t pb_base, AdjFusedPlan &out, AdjGroup &g) {
  const int32_t m = lt - lb;
  auto base_of = [&](int32_t i) { return i == 0 ? s_base : (((i - 1) & 1) == 0 ? pa_base : pb_base); };
  for (int32_t i = 0; i <= m; ++i)
    for (TNode &n : sh.nodes[i]) n.smem += base_of(i);
  FusedTemplate tp{};
  tp.load_begin = (int32_t)out.loads.size();
  const TNode &top = sh.nodes[0][0];
  const int32_t row0 = t.band_row0[lt][st[0][0].band];
  if (g.chunk > 0) {
    // row blocks: copies of 2^p consecutive rows, largest first
    const int32_t rows = top.e - top.a + 1;
    for (int32_t r = 0; r < rows;) {
      int32_t p = g.max_p;
      while ((1 << p) > rows - r) --p;
      out.loads.push_back(FusedLoad{row0 + top.a + r, top.smem + r * top.stride * 4, 0, p});
      r += 1 << p;
    }
  } else {
    for (int32_t d = top.a; d <= top.e; ++d)
      out.loads.push_back(FusedLoad{row0 + d, top.smem + (d - top.a) * top.stride * 4, 0, top.stride / kAdjBox});
  }
  tp.load_count = (int32_t)out.loads.size() - tp.load_begin;
  tp.tx_bytes = (top.e - top.a + 1) * top.stride * 4;
  tp.walk_begin = tp.walk_count = 0;
  tp.stage_begin = (int32_t)out.stages.size();
  g.hbm_bytes += (double)tp.tx_bytes * g.ntiles;

  // bal: the weights the warp split balances (default: the cost)
  auto push_stage = [&](int32_t kind, std::vector<FusedOp> &ops, std::vector<double> &cost,
                        const std::vector<double> *bal = nullptr) {
    const int32_t base = (int32_t)out.ops.size();
    out.ops.insert(out.ops.end(), ops.begin(), ops.end());
    const std::vector<int32_t> b = balance_warps(bal != nullptr ? *bal : cost);
    out.stages.push_back(kind);
    for (int32_t w = 0; w <= kFusedBlockWarps; ++w) out.stages.push_back(base + b[w]);
    for (double c : cost) g.slots += c * 32.0 * g.ntiles;
    ++tp.n_stages;
  };
  tp.n_stages = 0;
  for (int32_t s = 0; s < (fuse ? m - 1 : m); ++s) {
    const int32_t l = lt - s;
    const bool to_global = (s == m - 1) && !init;
    std::vector<FusedOp> ops;
    std::vector<double> cost;
    for (size_t k = 0; k < st[s].size(); ++k) {
      const SubBand &sb = st[s][k];
      const TNode &n = sh.nodes[s][k];
      if (n.empty()) continue;
      for (int32_t c : {sb.lo, sb.hi}) {
        if (c < 0) continue;
        const SubBand &cs = st[s + 1][c];
        const TNode &cn = sh.nodes[s + 1][c];
        if (cn.empty()) continue;
        const bool upper = cs.kind == 1;
        const int32_t width_all = to_global ? W : cn.need;
        for (int32_t x = cn.a; x <= cn.e; ++x) {
          const int32_t d0 = cs.rs[x], cnt = cs.re[x] - cs.rs[x] + 1;
          const int32_t shift0 = upper ? t.dl[l][sb.band][d0] - cn.dls : 0;
          for (int32_t c0 = 0; c0 < width_all; c0 += kPieceCols) {
            FusedOp op{};
            op.p0 = n.smem + ((d0 - n.a) * n.stride + c0 + shift0) * 4;
            op.p1 = (n.stride + (upper ? 1 : 0)) * 4;
            op.p2 = cnt;
            op.width = std::min(kPieceCols, width_all - c0);
            if (to_global) {
              op.dst = t.band_row0[lb][cs.band] + x;
              op.col = cn.o + c0;
              g.hbm_bytes += (double)op.width * 4 * g.ntiles;
            } else {
              op.dst = cn.smem + ((x - cn.a) * cn.stride + c0) * 4;
              op.col = c0;
            }
            ops.push_back(op);
            cost.push_back(cnt * kLaneCols + 3.0);
          }
        }
      }
    }
    push_stage(kAdjGather, ops, cost);
  }
  if (init && fuse) {
    // the level 1 -> 0 gather folded into the transpose: per channel and
    // piece, the first level-1 row's address (as the gather op of its row
    // 0 would read it) and the run lengths of its level-0 rows
    std::vector<FusedOp> ops;
    std::vector<double> cost;
    for (size_t k = 0; k < st[m].size(); ++k) {
      const SubBand &cs = st[m][k];
      const TNode &cn = sh.nodes[m][k];
      if (cn.empty()) continue;
      const SubBand &sb = st[m - 1][cs.parent];
      const TNode &n = sh.nodes[m - 1][cs.parent];
      const bool upper = cs.kind == 1;
      const int32_t rows = cn.e - cn.a + 1;
      int32_t runs = 0;
      double terms = 0;
      for (int32_t j = 0; j < rows; ++j) {
        const int32_t cnt = cs.re[j] - cs.rs[j] + 1;
        runs |= cnt << (4 * j);
        terms += (j + 1.0) * cnt;
      }
      const int32_t d0 = cs.rs[0];
      const int32_t shift0 = upper ? t.dl[1][sb.band][d0] - cn.dls : 0;
      for (int32_t c0 = 0; c0 < W; c0 += kPieceCols) {
        FusedOp op{};
        op.dst = cs.band;  // the channel
        op.p0 = n.smem + ((d0 - n.a) * n.stride + c0 + shift0) * 4;
        op.p1 = (n.stride + (upper ? 1 : 0)) * 4;
        op.p2 = rows;
        op.p3 = c0 / kPieceCols;
        op.width = std::min(kPieceCols, W - c0);
        op.flags = (upper ? 1 : 0) | (runs << 1);
        op.col = cn.o + c0;
        g.hbm_bytes += (double)op.width * 4 * g.ntiles;
        ops.push_back(op);
        cost.push_back(terms * kLaneCols + 3.0);
      }
    }
    std::vector<double> bal(cost);
    for (double &v : bal) v += kInitOpWait;
    push_stage(kAdjInitF, ops, cost, &bal);
  } else if (init) {
    std::vector<FusedOp> ops;
    std::vector<double> cost;
    for (size_t k = 0; k < st[m].size(); ++k) {
      const TNode &n = sh.nodes[m][k];
      if (n.empty()) continue;
      const int32_t rows = n.e - n.a + 1;
      for (int32_t c0 = 0; c0 < W; c0 += kPieceCols) {
        FusedOp op{};
        op.dst = st[m][k].band;  // the channel
        op.p0 = n.smem + c0 * 4;
        op.p1 = n.stride * 4;
        op.p2 = rows;
        op.p3 = c0 / kPieceCols;
        op.width = std::min(kPieceCols, W - c0);
        op.col = n.o + c0;
        g.hbm_bytes += (double)op.width * 4 * g.ntiles;
        ops.push_back(op);
        cost.push_back(rows * (rows + 1) / 2.0 * kLaneCols + 3.0);
      }
    }
    // With the weight gradient every init op waits once for its input
    // samples from global memory, a latency that dwarfs its sums: the warp
    // split weighs that wait too, so the warps get nearly equal op counts.
    std::vector<double> bal(cost);
    for (double &v : bal) v += kInitOpWait;
    push_stage(kAdjInit, ops, cost, &bal);
  }
  tp.smem_bytes = g.smem_bytes;
  out.tpls.push_back(tp);
  ++g.tpl_count;
}

// pitch > 0: row blocks of `chunk` elements, every staged row `pitch` wide;
// *widest receives the widest staged window of the launch's cones.
std::string plan_group(const Tables &t, int64_t nt, int32_t lt, int32_t lb, int32_t W, int32_t budget, bool grow,
                       int32_t pitch, int32_t chunk, AdjFusedPlan &out, AdjGroup &g, int32_t *widest) {
  const bool init = (lb == 0);
  const bool fuse = init && lt - lb >= 2 && init_fusable(t);
  g = AdjGroup();
  g.lt = lt;
  g.lb = lb;
  g.init = init;
  g.W = W;
  g.box = kAdjBox;
  if (pitch > 0) {
    g.box = 0;
    g.chunk = chunk;
    g.kchunks = pitch / chunk;
    // (one copy stays within 64 KiB of shared memory)
    g.max_p = 0;
    while (g.max_p < kMaxBlockP && (int64_t(2) << g.max_p) <= t.level_rows[lt] &&
           (int64_t(2) << g.max_p) * pitch * 4 <= 64 * 1024)
      ++g.max_p;
  }
  *widest = 0;
  g.tpl_begin = (int32_t)out.tpls.size();
  struct Piece {
    int32_t band, r0, r1;
    Shape sh;
  };
  std::vector<Subtree> subs;
  std::vector<Piece> pieces;
  const int32_t nb = (int32_t)t.band_rows[lt].size();
  for (int32_t B = 0; B < nb; ++B) {
    Subtree st;
    const std::string err = build_subtree(t, lt, lb, B, st);
    if (!err.empty()) return err;
    subs.push_back(std::move(st));
    const Subtree &s = subs.back();
    const int32_t R = t.band_rows[lt][B];
    // Split the top rows into ranges that fit the budget: the longest
    // range from r0 whose cone fits (binary search; the size grows with r1).
    for (int32_t r0 = 0; r0 < R;) {
      Shape sh;
      shape(t, s, lt, lb, init, fuse, r0, r0, W, pitch, sh);
      if (shape_bytes(sh) > budget) {
        // One row's cone can need most of its band (a band whose upper half
        // is one channel: that channel's row reads every parent row); the
        // launch then takes the shared memory it needs, if allowed.
        if (!grow || shape_bytes(sh) > kAdjMaxSmem)
          return "unsupported: one row of level " + std::to_string(lt) + " does not fit";
        budget = (int32_t)shape_bytes(sh);
      }
      int32_t lo = r0, hi = R - 1;
      while (lo < hi) {
        const int32_t mid = (lo + hi + 1) / 2;
        shape(t, s, lt, lb, init, fuse, r0, mid, W, pitch, sh);
        if (shape_bytes(sh) <= budget) lo = mid;
        else hi = mid - 1;
      }
      shape(t, s, lt, lb, init, fuse, r0, lo, W, pitch, sh);
      if (sh.any) {
        *widest = std::max(*widest, sh.nodes[0][0].need);
        pieces.push_back(Piece{B, r0, lo, sh});
      }
      r0 = lo + 1;
    }
  }
  // Group-wide regions, tiles.
  int64_t S = 0, Pa = 0, Pb = 0;
  int32_t omin = 0;
  for (const Piece &p : pieces) {
    S = std::max(S, p.sh.s_bytes);
    Pa = std::max(Pa, p.sh.pa_bytes);
    Pb = std::max(Pb, p.sh.pb_bytes);
    for (const TNode &n : p.sh.nodes.back())
      if (!n.empty()) omin = std::min(omin, n.o);
  }
  const int64_t total = kAdjBarrierBytes + S + Pa + Pb + kDescBytes + kOverRead;
  if (total > kAdjMaxSmem) return "unsupported: shared memory";
  g.smem_bytes = (int32_t)total;
  g.s_end = (int32_t)(kAdjBarrierBytes + S);
  g.pa_end = (int32_t)(g.s_end + Pa);
  g.ntiles = (nt - omin + W - 1) / W;
  for (const Piece &p : pieces)
    emit(t, subs[p.band], lt, lb, init, fuse, W, p.sh, kAdjBarrierBytes, g.s_end, g.pa_end, out, g);
  return "";
}

}  // namespace

std::string plan_adjoint_fused(const Tables &t, int64_t nt, const AdjParams &p, AdjFusedPlan &out) {
  out = AdjFusedPlan();
  const int32_t L = t.levels;
  if (L < 1) return "unsupported: no merge level";
  if (p.W < 64 || p.W % 64 != 0) return "tile must be a positive multiple of 64";
  if (p.smem_budget < 8 * 1024 || p.smem_budget > 227 * 1024) return "shared-memory budget out of range";
  auto try_bounds = [&](const std::vector<int32_t> &bounds) -> std::string {
    out = AdjFusedPlan();
    if (bounds.size() < 2 || bounds.front() != 0 || bounds.back() != L) return "bounds must run from 0 to L";
    for (size_t i = 1; i < bounds.size(); ++i)
      if (bounds[i] <= bounds[i - 1]) return "bounds must increase";
    for (size_t i = bounds.size() - 1; i >= 1; --i) {
      AdjGroup g;
      std::string err;
      const size_t tpls = out.tpls.size(), loads = out.loads.size(), ops = out.ops.size(),
                   stages = out.stages.size();
      auto rollback = [&]() {
        out.tpls.resize(tpls);
        out.loads.resize(loads);
        out.ops.resize(ops);
        out.stages.resize(stages);
      };
      // With the default budget a launch whose one-row cone does not fit
      // also tries narrower tiles (its window grows with the tile).
      int32_t widest = 0;
      const bool own = !p.bounds.empty() && i - 1 < p.group_W.size() && p.group_W[i - 1] > 0;
      // (the launch that ends at level 0 takes a wider tile unless told
      // otherwise: its items are small; three times the tile when it folds
      // the level 1 -> 0 gather into the transpose and so stores no level
      // 0, else twice; measured best on GB300)
      const bool fold = bounds[i - 1] == 0 && bounds[i] >= 2 && init_fusable(t);
      int32_t W = own ? p.group_W[i - 1]
                      : (bounds[i - 1] == 0 && p.init_wide ? std::min((fold ? 3 : 2) * p.W, 2048) : p.W);
      const int32_t budget =
          !p.bounds.empty() && i - 1 < p.group_budget.size() && p.group_budget[i - 1] > 0 ? p.group_budget[i - 1]
                                                                                          : p.smem_budget;
      if (W < 64 || W % 64 != 0 || budget < 8 * 1024 || budget > 227 * 1024) return "bad launch parameters";
      for (;; W /= 2) {
        err = plan_group(t, nt, bounds[i], bounds[i - 1], W, budget, p.grow_budget, 0, 0, out, g, &widest);
        if (err.empty() || !p.grow_budget || W / 2 < 64 || (W / 2) % 64 != 0) break;
        rollback();
      }
      if (!err.empty()) return err;
      if (nt % kAdjChunk == 0) {
        // Row blocks: one TMA copy per 2^p staged rows, every row as wide as
        // the launch's widest window (rebuilt until the pitch covers all).
        AdjGroup gb;
        for (int iter = 0; iter < 4; ++iter) {
          const int32_t k = (widest + kAdjChunk - 1) / kAdjChunk;
          if (k > 256 || (int64_t)k * kAdjChunk > nt) break;
          rollback();
          int32_t w2 = 0;
          const std::string e2 = plan_group(t, nt, bounds[i], bounds[i - 1], W, budget, p.grow_budget,
                                            k * kAdjChunk, kAdjChunk, out, gb, &w2);
          if (!e2.empty()) break;
          if (w2 <= k * kAdjChunk) {
            g = gb;
            widest = -1;
            break;
          }
          widest = w2;
        }
        if (widest >= 0) {  // keep row boxes
          rollback();
          err = plan_group(t, nt, bounds[i], bounds[i - 1], W, budget, p.grow_budget, 0, 0, out, g, &widest);
          if (!err.empty()) return err;
        }
      }
      out.groups.push_back(g);
    }
    return "";
  };
  std::string err;
  if (!p.bounds.empty()) {
    err = try_bounds(p.bounds);
  } else {
    // The launch that ends with the initialisation transpose covers d
    // levels (a channel's level-0 rows are needed whole, so it stays
    // shallow), those above it s levels each; a one-level remainder at the
    // top joins the launch below it.  Two levels per launch measured best
    // on GB300 (a cone's staged row halo doubles with every level); the
    // first grouping that fits wins.
    err = "unsupported: no grouping fits";
    for (int32_t s : {2, 3, 1}) {
      for (int32_t d : {2, 1, 3}) {
        std::vector<int32_t> b{0};
        for (int32_t v = std::min(L, d); ; v = std::min(L, v + s)) {
          b.push_back(v);
          if (v == L) break;
        }
        if (b.size() > 3 && b[b.size() - 1] - b[b.size() - 2] == 1) b.erase(b.end() - 2);
        if ((err = try_bounds(b)).empty()) break;
      }
      if (err.empty()) break;
    }
  }
  if (!err.empty()) {
    out = AdjFusedPlan();
    return err;
  }
  {
    AdjGroup &gl = out.groups.back();
    gl.pieces = (gl.W + kPieceCols - 1) / kPieceCols;
    out.part_slots = (int64_t)t.nf * gl.ntiles * gl.pieces;
  }
  // Group k writes level lb_k into buffer k % 2 (the last writes the input
  // gradient).
  for (size_t k = 0; k + 1 < out.groups.size(); ++k) {
    const size_t b = (size_t)t.level_rows[out.groups[k].lb] * (size_t)nt * sizeof(float);
    out.buf_bytes[k & 1] = std::max(out.buf_bytes[k & 1], b);
  }
  return "";
}

}  // namespace fdmt
