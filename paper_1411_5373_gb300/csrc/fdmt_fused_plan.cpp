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
constexpr double kHbmRate = 7.0e12;          // bytes/s
constexpr double kColumnSeconds = 3.9e-13;   // per column of a shared-memory op (GPU-wide)
constexpr double kInitSeconds = 3.9e-13;     // per column x row of an Option-1 sum
constexpr double kItemSeconds = 1.73e-6;     // per work item, per block slot
constexpr double kOpSeconds = 1.76e-8;       // per op, per block slot
constexpr double kLaunchSeconds = 14e-6;
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
};

struct ConeOut {
  FusedTemplate tpl{};
  std::vector<FusedLoad> loads;
  std::vector<FusedInit> inits;
  std::vector<FusedOp> ops;
  std::vector<int32_t> level_ops;  // relative to ops
  double hbm = 0, smem_traffic = 0;
  double op_cols = 0, init_cols = 0, nops = 0;  // cost-model counts (one tile)
};

// Region sizes of one cone: S = staged source rows (input channels or the
// base level), Pa / Pb = computed levels, alternating.  A group lays all its
// cones out at the same region bases (the maxima over its cones) so that a
// block can stage the next cone into S while it still computes in Pa / Pb.
struct ConeShape {
  std::vector<std::vector<Node>> nodes;  // [level - lb]
  int64_t s_bytes = 0, pa_bytes = 0, pb_bytes = 0;
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
};

void shape_cone(const Tables &t, int32_t lb, int32_t lt, int32_t band, int32_t r0, int32_t r1,
                int32_t W, const FusedPlan &fp, const StageFmt &f, ConeShape &cs) {
  const bool from_input = (lb == 0);
  const int32_t sA = fp.acc_size, sB = fp.level_size[lb], sI = fp.input_size;
  const int32_t alignB = f.chunk > 0 ? f.chunk : 16 / sB, alignI = f.chunk > 0 ? f.chunk : 16 / sI;
  const int32_t m = lt - lb;
  cs = ConeShape();
  std::vector<std::vector<Node>> &nodes = cs.nodes;
  nodes.assign(m + 1, {});
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
  // Level index i = l - lb for l in [lb, lt).  Computed levels take Pa, Pb,
  // Pa, ... in order: for an input cone that starts with level 0 itself,
  // otherwise with level lb + 1.
  int64_t pa = 0, pb = 0;
  for (int32_t i = 0; i < m; ++i) {
    int64_t off = 0;
    const bool staged = (i == 0 && !from_input);
    const int32_t k = from_input ? i : i - 1;  // index among computed levels
    for (Node &n : nodes[i]) {
      const int32_t rows = n.e - n.a + 1;
      if (staged) {
        const int32_t ceil_o = (int32_t)ceil_to(n.o, alignB);
        n.delta = ceil_o - n.o;
        cs.needs.emplace_back(W + n.s + n.delta, n.e - n.a + 1);
        n.stride = pitch(W + n.s + n.delta, own_max);
        n.smem = (int32_t)off;
        off += round_up((int64_t)rows * n.stride * sB, 128);
      } else {
        n.delta = 0;
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
    if (staged) cs.s_bytes = off;
    else if ((k & 1) == 0) pa = std::max(pa, off);
    else pb = std::max(pb, off);
  }
  cs.pa_bytes = pa;
  cs.pb_bytes = pb;
}

int64_t cone_bytes(const ConeShape &cs) {
  return kBarrierBytes + cs.s_bytes + cs.pa_bytes + cs.pb_bytes;
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

// `cones` = cones in the work item (their channels share the warps).
void emit_cone(const Tables &t, int32_t lb, int32_t lt, int32_t W, const FusedPlan &fp, const StageFmt &f,
               ConeShape &cs, int64_t base_s, int64_t base_a, int64_t base_b, int32_t cones, ConeOut &c) {
  const bool from_input = (lb == 0);
  const int32_t sA = fp.acc_size, sB = fp.level_size[lb], sI = fp.input_size;
  const int32_t alignB = f.chunk > 0 ? f.chunk : 16 / sB, alignI = f.chunk > 0 ? f.chunk : 16 / sI;
  const int32_t m = lt - lb;
  std::vector<std::vector<Node>> &nodes = cs.nodes;
  for (int32_t i = 0; i < m; ++i) {
    const bool staged = (i == 0 && !from_input);
    const int32_t k = from_input ? i : i - 1;
    const int64_t region = staged ? base_s : ((k & 1) == 0 ? base_a : base_b);
    for (Node &n : nodes[i]) {
      n.smem += (int32_t)region;
      n.xsmem += (int32_t)base_s;
    }
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
    // With fewer channels in the work item than warps, each channel's
    // columns are split into pieces (multiples of 32 columns) so that every
    // warp has a piece.
    const int32_t nch = (int32_t)nodes[0].size() * cones;
    const int32_t pieces = std::max<int32_t>(1, kFusedBlockWarps / nch);
    for (const Node &n : nodes[0]) {
      if (f.chunk == 0) {
        c.loads.push_back(FusedLoad{n.band, n.xsmem, -(int32_t)ceil_to(n.o + n.e, alignI),
                                    n.xstride / f.box});
        tx += (int64_t)n.xstride * sI;
      }
      const int32_t width = W + n.s;
      const int32_t piece = (int32_t)round_up((width + pieces - 1) / pieces, 32);
      for (int32_t c0 = 0; c0 < width; c0 += piece) {
        FusedInit in{};
        in.x_smem = n.xsmem + (n.xdelta + c0) * sI;
        in.dst_smem = n.smem + c0 * sA;
        in.a = n.a;
        in.e = n.e;
        in.width = std::min(piece, width - c0);
        in.chan = n.band;
        in.dst_stride = n.stride;
        c.inits.push_back(in);
      }
      c.smem_traffic += (double)width * ((n.e + 1) * sI + (n.e - n.a + 1) * sA);
      c.init_cols += (double)width * (n.e + 1);
    }
  } else {
    for (const Node &n : nodes[0]) {
      const int32_t row0 = t.band_row0[lb][n.band];
      const int32_t xoff = -(int32_t)ceil_to(n.o, alignB);
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
        c.nops += 1;
        if (!top) c.op_cols += op.width;
        if (top) c.hbm += (double)W * fp.level_size[lt];
      }
    }
  }
  c.level_ops.push_back((int32_t)c.ops.size());
  c.tpl.n_levels = m;
}

struct GroupBuild {
  bool ok = false;
  FusedGroup g;
  std::vector<ConeOut> cones;
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
  const int32_t nb = t.nf >> lt;
  for (int32_t cone_budget = budget; cone_budget >= 4096; cone_budget = cone_budget * 7 / 8) {
    std::vector<ConeShape> shapes;
    bool ok = true;
    for (int32_t b = 0; b < nb && ok; ++b) {
      const int32_t rows = t.band_rows[lt][b];
      auto fits = [&](int32_t per, std::vector<ConeShape> *keep) {
        for (int32_t r0 = 0; r0 < rows; r0 += per) {
          ConeShape cs;
          shape_cone(t, lb, lt, b, r0, std::min(rows, r0 + per) - 1, W, fp, f, cs);
          if (cone_bytes(cs) > cone_budget) return false;
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
    int64_t bs = 0, ba = 0, bb = 0;
    for (int32_t i = 0; i < (int32_t)shapes.size(); ++i) {
      const ConeShape &cs = shapes[i];
      if (!bundles.empty() && (int64_t)bundles.back().size() < cap &&
          kBarrierBytes + bs + cs.s_bytes + ba + cs.pa_bytes + bb + cs.pb_bytes <= cone_budget) {
        bundles.back().push_back(i);
        bs += cs.s_bytes;
        ba += cs.pa_bytes;
        bb += cs.pb_bytes;
      } else {
        bundles.push_back({i});
        bs = cs.s_bytes;
        ba = cs.pa_bytes;
        bb = cs.pb_bytes;
      }
    }
    int64_t ms = 0, ma = 0, mb = 0;
    for (const std::vector<int32_t> &bu : bundles) {
      int64_t s1 = 0, a1 = 0, b1 = 0;
      for (int32_t i : bu) {
        s1 += shapes[i].s_bytes;
        a1 += shapes[i].pa_bytes;
        b1 += shapes[i].pb_bytes;
      }
      ms = std::max(ms, s1);
      ma = std::max(ma, a1);
      mb = std::max(mb, b1);
    }
    const int64_t total = kBarrierBytes + ms + ma + mb;
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
    gb.g.ntiles = (nt + W - 1) / W;
    gb.g.smem_bytes = (int32_t)total;
    gb.g.s_end = (int32_t)(kBarrierBytes + ms);
    gb.g.pa_end = (int32_t)(kBarrierBytes + ms + ma);
    double hbm = 0, sm = 0, opc = 0, inic = 0, nops = 0;
    for (const std::vector<int32_t> &bu : bundles) {
      // Each cone of the item gets its own slice of S, Pa and Pb; the item's
      // ops are merged level by level.
      ConeOut item;
      int64_t so = 0, ao = 0, bo = 0;
      std::vector<std::vector<FusedOp>> per_level(lt - lb);
      for (int32_t i : bu) {
        ConeShape &cs = shapes[i];
        if (needs) needs->insert(needs->end(), cs.needs.begin(), cs.needs.end());
        ConeOut c;
        emit_cone(t, lb, lt, W, fp, f, cs, kBarrierBytes + so, kBarrierBytes + ms + ao,
                  kBarrierBytes + ms + ma + bo, (int32_t)bu.size(), c);
        so += cs.s_bytes;
        ao += cs.pa_bytes;
        bo += cs.pb_bytes;
        item.loads.insert(item.loads.end(), c.loads.begin(), c.loads.end());
        item.inits.insert(item.inits.end(), c.inits.begin(), c.inits.end());
        for (int32_t lv = 0; lv < lt - lb; ++lv)
          per_level[lv].insert(per_level[lv].end(), c.ops.begin() + c.level_ops[lv],
                               c.ops.begin() + c.level_ops[lv + 1]);
        item.tpl.tx_bytes += c.tpl.tx_bytes;
        item.hbm += c.hbm;
        item.smem_traffic += c.smem_traffic;
        item.op_cols += c.op_cols;
        item.init_cols += c.init_cols;
        item.nops += c.nops;
      }
      for (int32_t lv = 0; lv < lt - lb; ++lv) {
        item.level_ops.push_back((int32_t)item.ops.size());
        item.ops.insert(item.ops.end(), per_level[lv].begin(), per_level[lv].end());
      }
      item.level_ops.push_back((int32_t)item.ops.size());
      item.tpl.n_levels = lt - lb;
      item.tpl.smem_bytes = (int32_t)total;
      hbm += item.hbm;
      sm += item.smem_traffic;
      opc += item.op_cols;
      inic += item.init_cols;
      nops += item.nops;
      gb.cones.push_back(std::move(item));
    }
    gb.g.hbm_bytes = hbm * (double)gb.g.ntiles;
    gb.g.smem_traffic = sm * (double)gb.g.ntiles;
    const double tiles = (double)gb.g.ntiles;
    const double items = (double)gb.cones.size() * tiles;
    const double slots =
        kSms * std::min(kMaxBlocksPerSm, std::max(1.0, std::floor((228.0 * 1024) / (total + 1024.0))));
    const double on_chip = (opc * kColumnSeconds + inic * kInitSeconds) * tiles +
                           (items * kItemSeconds + nops * tiles * kOpSeconds) / slots + kLaunchSeconds;
    gb.seconds = std::max(gb.g.hbm_bytes / kHbmRate, on_chip);
    gb.ok = true;
    return gb;
  }
  return gb;
}

// Group (lb, lt] for tile W.  The staging format follows the windows of
// the group's own cones: a first build with provisional boxes measures
// them, the second uses the chosen box or block width.
GroupBuild build_group(const Tables &t, int64_t nt, int32_t lb, int32_t lt, int32_t W,
                       const FusedPlan &fp, int32_t budget, int32_t staging) {
  const int32_t es = (lb == 0) ? fp.input_size : fp.level_size[lb];
  const int64_t rows = (lb == 0) ? t.nf : t.level_rows[lb];
  // Row blocks: chunks of 128 bytes (64 for 1-byte samples, so that a tile
  // start, a multiple of 64 samples, is a chunk boundary).
  const int32_t chunk = std::min(128 / es, 64);
  const bool blocks = staging != 1 && nt % chunk == 0;
  if (staging == 2 && !blocks) return GroupBuild();
  StageFmt f;
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
    widths = {128, 256, 512, 1024};
  }
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
      GroupBuild gb = build_group(t, nt, lb, lt, W, fp, budget > 0 ? budget : p.smem_budget, p.staging);
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
