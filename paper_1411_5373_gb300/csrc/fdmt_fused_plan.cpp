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
// The level grouping and W are chosen by a cost model (dynamic programming
// over group boundaries): time = max(HBM bytes / HBM rate, shared-memory
// bytes / shared-memory rate) + a launch overhead per group.
#include "fdmt_fused.h"

#include <algorithm>
#include <cmath>
#include <limits>

namespace fdmt {
namespace {

constexpr int32_t kBarrierBytes = 128;  // mbarrier slot, keeps regions 128-byte aligned
constexpr double kHbmRate = 6.0e12;     // bytes/s, model only
constexpr double kSmemRate = 2.4e13;    // bytes/s, model only
constexpr double kLaunchSeconds = 4e-6;

int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }
int64_t ceil_to(int64_t v, int64_t a) { return round_up(v, a); }

struct Node {
  int32_t band, a, e;  // band index at its level, first and last row
  int32_t o, s;        // window [T0 - o, T0 - o + W + s)
  int32_t smem = 0;    // byte offset of row a
  int32_t stride = 0;  // elements per row in shared memory
  int32_t delta = 0;   // column of time T0 - o within the stored row
  int32_t xsmem = 0, xstride = 0, xdelta = 0;  // staged input (level 0 of an input cone)
};

struct ConeOut {
  FusedTemplate tpl{};
  std::vector<FusedLoad> loads;
  std::vector<FusedInit> inits;
  std::vector<FusedOp> ops;
  std::vector<int32_t> level_ops;  // relative to ops
  double hbm = 0, smem_traffic = 0;
};

// Builds one cone; returns false if it needs more than `budget` bytes.
bool build_cone(const Tables &t, int32_t lb, int32_t lt, int32_t band, int32_t r0, int32_t r1,
                int32_t W, const FusedPlan &fp, int32_t budget, ConeOut &c) {
  const bool from_input = (lb == 0);
  const int32_t sA = fp.acc_size, sB = fp.state_size, sI = fp.input_size;
  const int32_t alignB = 16 / sB, alignI = 16 / sI;
  const int32_t m = lt - lb;
  std::vector<std::vector<Node>> nodes(m + 1);
  nodes[m].push_back(Node{band, r0, r1, 0, 0});
  for (int32_t l = lt; l > lb; --l) {
    std::vector<Node> &kids = nodes[l - 1 - lb];
    for (const Node &p : nodes[l - lb]) {
      const std::vector<int32_t> &dl = t.dl[l][p.band];
      const int32_t da = dl[p.a], de = dl[p.e];
      kids.push_back(Node{2 * p.band, da, de, p.o, p.s});
      kids.push_back(Node{2 * p.band + 1, p.a - da, p.e - de, p.o + de, p.s + de - da});
    }
  }

  // Shared-memory layout: [barrier][X: staged input][P0: even levels][P1: odd levels].
  int64_t x_bytes = 0;
  int64_t level_bytes[2] = {0, 0};
  std::vector<int64_t> lvl_size(m, 0);
  for (int32_t i = 0; i < m; ++i) {  // levels lb .. lt-1
    int64_t off = 0;
    for (Node &n : nodes[i]) {
      const int32_t rows = n.e - n.a + 1;
      int32_t esz;
      if (i == 0 && !from_input) {  // TMA-loaded base rows
        const int32_t ceil_o = (int32_t)ceil_to(n.o, alignB);
        n.delta = ceil_o - n.o;
        n.stride = (int32_t)round_up(W + n.s + n.delta, fp.box_state);
        esz = sB;
      } else {
        n.delta = 0;
        n.stride = (int32_t)round_up(W + n.s, 4);
        esz = sA;
      }
      n.smem = (int32_t)off;  // relative to the region for now
      off += round_up((int64_t)rows * n.stride * esz, 128);
      if (i == 0 && from_input) {
        const int32_t ceil_oe = (int32_t)ceil_to(n.o + n.e, alignI);
        n.xdelta = ceil_oe - n.o;
        n.xstride = (int32_t)round_up(W + n.s + n.xdelta, fp.box_input);
        n.xsmem = (int32_t)x_bytes;
        x_bytes += round_up((int64_t)n.xstride * sI, 128);
      }
    }
    lvl_size[i] = off;
    level_bytes[i & 1] = std::max(level_bytes[i & 1], off);
  }
  const int64_t p0 = kBarrierBytes + x_bytes;
  const int64_t p1 = p0 + level_bytes[0];
  const int64_t total = p1 + level_bytes[1];
  if (total > budget) return false;
  for (int32_t i = 0; i < m; ++i)
    for (Node &n : nodes[i]) {
      n.smem += (int32_t)((i & 1) ? p1 : p0);
      n.xsmem += (int32_t)kBarrierBytes;
    }

  c = ConeOut();
  c.tpl.smem_bytes = (int32_t)total;
  int64_t tx = 0;
  // Loads.
  if (from_input) {
    for (const Node &n : nodes[0]) {
      FusedLoad ld{n.band, n.xsmem, -(int32_t)ceil_to(n.o + n.e, alignI), n.xstride / fp.box_input};
      c.loads.push_back(ld);
      tx += (int64_t)n.xstride * sI;
      FusedInit in{};
      in.x_smem = n.xsmem + n.xdelta * sI;
      in.dst_smem = n.smem;
      in.a = n.a;
      in.e = n.e;
      in.width = W + n.s;
      in.chan = n.band;
      in.dst_stride = n.stride;
      c.inits.push_back(in);
      c.smem_traffic += (double)in.width * ((n.e + 1) * sI + (n.e - n.a + 1) * sA);
    }
  } else {
    for (const Node &n : nodes[0]) {
      const int32_t row0 = t.band_row0[lb][n.band];
      for (int32_t j = n.a; j <= n.e; ++j) {
        FusedLoad ld{row0 + j, n.smem + (j - n.a) * n.stride * sB, -(int32_t)ceil_to(n.o, alignB),
                     n.stride / fp.box_state};
        c.loads.push_back(ld);
        tx += (int64_t)n.stride * sB;
      }
    }
  }
  c.tpl.tx_bytes = (int32_t)tx;
  c.hbm += (double)tx;

  // Ops, level by level (lb+1 .. lt).
  for (int32_t l = lb + 1; l <= lt; ++l) {
    c.level_ops.push_back((int32_t)c.ops.size());
    const bool top = (l == lt);
    const std::vector<Node> &par = nodes[l - lb];
    const std::vector<Node> &kid = nodes[l - 1 - lb];
    const bool kids_base = (l - 1 == lb) && !from_input;
    const int32_t ksz = kids_base ? sB : sA;
    for (size_t pi = 0; pi < par.size(); ++pi) {
      const Node &p = par[pi];
      const Node &lo = kid[2 * pi];
      const Node &hi = kid[2 * pi + 1];
      const std::vector<int32_t> &dl = t.dl[l][p.band];
      const int32_t de = dl[p.e];
      for (int32_t dt = p.a; dt <= p.e; ++dt) {
        const int32_t j = dl[dt];
        const int32_t mrow = dt - j;
        const int32_t q = de - j;
        FusedOp op;
        op.dst = top ? (t.band_row0[lt][p.band] + dt) : (p.smem + (dt - p.a) * p.stride * sA);
        op.lo = lo.smem + ((j - lo.a) * lo.stride + lo.delta) * ksz;
        op.hi = hi.smem + ((mrow - hi.a) * hi.stride + hi.delta + q) * ksz;
        op.width = top ? W : W + p.s;
        c.ops.push_back(op);
        c.smem_traffic += (double)op.width * (2 * ksz + (top ? 0 : sA));
        if (top) c.hbm += (double)W * (lt == t.levels ? 4 : sB);
      }
    }
  }
  c.level_ops.push_back((int32_t)c.ops.size());
  c.tpl.n_levels = m;
  return true;
}

struct GroupBuild {
  bool ok = false;
  FusedGroup g;
  std::vector<ConeOut> cones;
  double seconds = 0;
};

// All cones of group (lb, lt]: each band of level lt split into the fewest
// equal row ranges that fit.
GroupBuild build_group(const Tables &t, int64_t nt, int32_t lb, int32_t lt, int32_t W,
                       const FusedPlan &fp, int32_t budget) {
  GroupBuild gb;
  gb.g.lb = lb;
  gb.g.lt = lt;
  gb.g.from_input = (lb == 0);
  gb.g.ntiles = (nt + W - 1) / W;
  const int32_t nb = t.nf >> lt;
  for (int32_t b = 0; b < nb; ++b) {
    const int32_t rows = t.band_rows[lt][b];
    // Largest rows-per-cone `per` whose cones all fit (binary search: smaller
    // row ranges give smaller cones).
    auto try_split = [&](int32_t per, std::vector<ConeOut> *keep) {
      for (int32_t r0 = 0; r0 < rows; r0 += per) {
        ConeOut c;
        if (!build_cone(t, lb, lt, b, r0, std::min(rows, r0 + per) - 1, W, fp, budget, c)) return false;
        if (keep) keep->push_back(std::move(c));
      }
      return true;
    };
    int32_t lo = 0, hi = rows;  // lo fits (0 = none yet), hi is the candidate upper bound
    if (try_split(rows, nullptr)) {
      lo = rows;
    } else {
      while (hi - lo > 1) {
        const int32_t mid = lo + (hi - lo) / 2;
        if (try_split(std::max(mid, 1), nullptr)) lo = mid; else hi = mid;
      }
    }
    if (lo < 1) return gb;  // even single rows do not fit
    // Balance: the fewest parts of size <= lo, spread evenly.
    const int32_t parts = (rows + lo - 1) / lo;
    const int32_t per = (rows + parts - 1) / parts;
    std::vector<ConeOut> cs;
    if (!try_split(per, &cs)) return gb;
    for (ConeOut &c : cs) gb.cones.push_back(std::move(c));
  }
  double hbm = 0, sm = 0;
  int32_t smem = 0;
  for (const ConeOut &c : gb.cones) {
    hbm += c.hbm;
    sm += c.smem_traffic;
    smem = std::max(smem, c.tpl.smem_bytes);
  }
  gb.g.hbm_bytes = hbm * (double)gb.g.ntiles;
  gb.g.smem_traffic = sm * (double)gb.g.ntiles;
  gb.g.smem_bytes = smem;
  // Two blocks per SM share the shared memory bandwidth when they fit.
  gb.seconds = std::max(gb.g.hbm_bytes / kHbmRate, gb.g.smem_traffic / kSmemRate) + kLaunchSeconds;
  gb.ok = true;
  return gb;
}

void append_group(FusedPlan &fp, GroupBuild &gb) {
  FusedGroup g = gb.g;
  g.tpl_begin = (int32_t)fp.tpls.size();
  g.tpl_count = (int32_t)gb.cones.size();
  for (ConeOut &c : gb.cones) {
    FusedTemplate tp = c.tpl;
    tp.load_begin = (int32_t)fp.loads.size();
    tp.load_count = (int32_t)c.loads.size();
    tp.init_begin = (int32_t)fp.inits.size();
    tp.init_count = (int32_t)c.inits.size();
    tp.level_begin = (int32_t)fp.level_ops.size();
    const int32_t op0 = (int32_t)fp.ops.size();
    for (int32_t v : c.level_ops) fp.level_ops.push_back(op0 + v);
    fp.loads.insert(fp.loads.end(), c.loads.begin(), c.loads.end());
    fp.inits.insert(fp.inits.end(), c.inits.begin(), c.inits.end());
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
    widths = {128, 256, 512};
  }
  FusedPlan best;
  double best_s = std::numeric_limits<double>::infinity();
  for (int32_t W : widths) {
    FusedPlan fp;
    fp.W = W;
    fp.state_size = state_size;
    fp.input_size = input_size;
    fp.acc_size = 4;
    fp.box_state = 256 / state_size;
    fp.box_input = 256 / input_size;
    std::vector<int32_t> bounds = p.bounds;
    std::vector<GroupBuild> chosen;
    if (bounds.empty()) {
      // Dynamic programming over boundaries: cost[j] = best time to reach level j.
      std::vector<double> cost(L + 1, std::numeric_limits<double>::infinity());
      std::vector<int32_t> from(L + 1, -1);
      cost[0] = 0;
      for (int32_t j = 1; j <= L; ++j)
        for (int32_t i = std::max(0, j - 6); i < j; ++i) {
          if (!std::isfinite(cost[i])) continue;
          GroupBuild gb = build_group(t, nt, i, j, W, fp, p.smem_budget);
          if (!gb.ok) continue;
          if (cost[i] + gb.seconds < cost[j]) {
            cost[j] = cost[i] + gb.seconds;
            from[j] = i;
          }
        }
      if (!std::isfinite(cost[L])) continue;
      std::vector<int32_t> rev;
      for (int32_t j = L; j > 0; j = from[j]) rev.push_back(j);
      bounds = {0};
      for (auto it = rev.rbegin(); it != rev.rend(); ++it) bounds.push_back(*it);
    }
    if (bounds.size() < 2 || bounds.front() != 0 || bounds.back() != L)
      return "level boundaries must run from 0 to L";
    double secs = 0;
    bool ok = true;
    for (size_t i = 0; i + 1 < bounds.size() && ok; ++i) {
      if (bounds[i + 1] <= bounds[i]) return "level boundaries must increase";
      GroupBuild gb = build_group(t, nt, bounds[i], bounds[i + 1], W, fp, p.smem_budget);
      if (!gb.ok) ok = false;
      secs += gb.seconds;
      chosen.push_back(std::move(gb));
    }
    if (!ok) continue;
    for (GroupBuild &gb : chosen) append_group(fp, gb);
    fp.model_seconds = secs;
    if (secs < best_s) {
      best_s = secs;
      best = std::move(fp);
    }
  }
  if (!std::isfinite(best_s)) return "no fused schedule fits the shared-memory budget";
  // Intermediate states between groups: group g writes buffer g % 2.
  size_t even = 0, odd = 0;
  for (size_t g = 0; g + 1 < best.groups.size(); ++g) {
    const size_t bytes = (size_t)t.level_rows[best.groups[g].lt] * (size_t)nt * (size_t)state_size;
    if (g & 1) odd = std::max(odd, bytes); else even = std::max(even, bytes);
  }
  best.ws_split = (size_t)round_up((int64_t)even, 256);
  best.ws_bytes = best.ws_split + (size_t)round_up((int64_t)odd, 256);
  out = std::move(best);
  return "";
}

}  // namespace fdmt
