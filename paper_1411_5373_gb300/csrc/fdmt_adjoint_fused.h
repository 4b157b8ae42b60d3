// Fused schedule of the FDMT adjoint: several transposed levels per launch.
//
// The adjoint of the addition rule (section 4 of arXiv:1411.5373; the
// transpose is derived, the paper does not state it) runs from level L down.
// For a band b of level l with lower half lo and upper half hi:
//   g_lo[j][u] = sum over rows Dt with dl(Dt) = j       of g[Dt][u]
//   g_hi[m][u] = sum over rows Dt with Dt - dl(Dt) = m  of g[Dt][u + dl(Dt)]
// (g = 0 at times >= Nt); a band without an upper half passes its rows down.
// Because dl grows by 0 or 1 from one row to the next, the rows read by one
// child row form a run of consecutive parent rows, and for the upper half
// the shift grows by one along the run.
//
// A launch covers the levels lt -> lb.  Its work items are "pull cones": a
// band B of level lt, a range [r0, r1] of its rows, and a time tile.  The
// item owns the level-lb rows whose run of level-lt rows (the composition
// of the runs down the levels) starts in [r0, r1]; every row of level lb is
// owned by exactly one item.  The rows each level of the cone needs are the
// hull of the runs of the rows the level below needs, so the staged level-lt
// rows extend past r1 by the last owned run.  Windows: a node of the cone
// holds the times [T0 + o, T0 + o + w); the lower half keeps its parent's
// start, the upper half starts dl(first row of its runs) earlier, and a
// parent is as wide as its widest child plus that child's dl range.  The
// owned level-lb rows are written for [T0 + o, T0 + o + W), so each band
// tiles time with its own offset (o <= 0).  The level-lt rows are staged in
// shared memory by TMA (zero past Nt: the gradient of outputs that do not
// exist), the levels in between are computed in shared memory, and level lb
// is written to global memory.  The launch that ends at level 0 also applies
// the transpose of the Option-1 initialisation and writes the input
// gradient (level 0 never reaches global memory); when it covers two levels
// or more, the level 1 -> 0 gather is folded into that transpose and level
// 0 is not stored in shared memory either.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "fdmt_fused.h"
#include "fdmt_tables.h"

namespace fdmt {

// Stage kinds of an adjoint item (stage words as in the forward schedule:
// kind, the first op of each warp, the end of the stage's ops).  Ops reuse
// the FusedOp layout:
//   kAdjGather  out[tau] = sum_{i < p2} s[p0 + i p1 + 4 tau]    (one level)
//   kAdjInit    out[tau] = sum_{j < p2} sum_{i <= j} s[p0 + j p1 + 4 (tau + i)]
//               (the Option-1 transpose: rows j of one channel at level 0;
//               p3 = the op's piece within the tile)
//   kAdjInitF   the same with the level 1 -> 0 gather folded in: level-0 row
//               j of the channel is never stored; each of its values is
//               re-formed from its run of cnt_j level-1 rows, term (j, i) =
//               sum_{q < cnt_j} s[P_j + 4 (tau + i) + q p1], P_0 = p0,
//               P_{j+1} = P_j + cnt_j p1 - 4 u (u = flags & 1: the channel
//               is its band's upper half), cnt_j = (flags >> (1 + 4 j)) & 15;
//               the same additions in the same order as kAdjGather then
//               kAdjInit
// p0 and p1 are byte offsets and strides in shared memory, p2 the number of
// terms (rows).  dst is a byte offset in shared memory, or for the stage
// that writes global memory the global row (level-lb row, or the channel),
// written at times T0 + col + tau for tau < width inside [0, Nt).
enum : int32_t { kAdjGather = 1, kAdjInit = 2, kAdjInitF = 3 };

struct AdjGroup {
  int32_t lt = 0, lb = 0;     // levels lt -> lb
  bool init = false;          // lb == 0: ends with the initialisation transpose
  int32_t W = 0;              // time tile of this launch
  int32_t box = 0;            // row boxes: TMA box width (elements) of the staged rows
  int32_t chunk = 0;          // row blocks (chunk > 0): chunk elements, chunks per row
  int32_t kchunks = 0;        //   (the row pitch), and the largest copy (2^max_p rows)
  int32_t max_p = 0;
  int32_t tpl_begin = 0, tpl_count = 0;
  int32_t smem_bytes = 0;     // barrier + S + Pa + Pb + over-read slack
  int32_t s_end = 0, pa_end = 0;
  int64_t ntiles = 0;         // tiles per template (time covered with the bands' offsets)
  int32_t pieces = 0;         // init launch: op pieces per channel and tile (weight-gradient partials)
  double hbm_bytes = 0;       // model: staged + written bytes per launch
  double slots = 0;           // model: shared-memory accesses per launch
};

struct AdjParams {
  int32_t W = 512;                // time tile (multiple of 64)
  int32_t smem_budget = 112 * 1024;
  std::vector<int32_t> bounds;    // level boundaries 0 = b0 < ... < bk = L; empty = choose
  std::vector<int32_t> group_W;       // with bounds: tile of the launch b_{i+1} -> b_i (0 = W)
  std::vector<int32_t> group_budget;  // with bounds: its budget (0 = smem_budget)
  bool grow_budget = true;        // a launch whose single-row cone exceeds the budget takes what it needs
  bool init_wide = true;          // the launch ending at level 0 takes a wider tile (no explicit tile):
                                  // 3x when it folds the level 1 -> 0 gather, else 2x
};

struct AdjFusedPlan {
  std::vector<AdjGroup> groups;   // in launch order (from level L down)
  std::vector<FusedTemplate> tpls;
  std::vector<FusedLoad> loads;
  std::vector<FusedOp> ops;
  std::vector<int32_t> stages;
  // Workspace: the level between two launches, ping-pong (group g writes
  // buffer g % 2); bytes each buffer needs.
  size_t buf_bytes[2] = {0, 0};
  // Weight-gradient partials of the init launch: one float per (channel,
  // tile, piece).
  int64_t part_slots = 0;
};

// Builds the adjoint cone templates.  Returns "" on success, else why the
// schedule does not fit.
std::string plan_adjoint_fused(const Tables &t, int64_t nt, const AdjParams &p, AdjFusedPlan &out);

}  // namespace fdmt
