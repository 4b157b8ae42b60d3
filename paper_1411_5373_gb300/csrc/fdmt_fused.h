// Fused schedule of the FDMT: several merge levels per launch.
//
// A launch covers the levels (lb, lt] of the addition rule (section 4 of
// arXiv:1411.5373).  Its work items are "cones": one band B of level lt, a
// range of its delay rows, and one time tile [T0, T0 + W).  Following the
// addition rule down from those rows gives, for every sub-band of B at every
// level l in [lb, lt), a contiguous row range and a time window
// [T0 - o, T0 - o + W + s): the lower half keeps the parent's window, the
// upper half's window starts dl(last row) samples earlier and is
// dl(last) - dl(first) samples wider.  The level-lb rows of the cone are
// staged in shared memory by TMA (zero-filled outside [0, Nt), which is the
// paper's copy rule), the levels in between are computed in shared memory,
// and level lt is written to global memory.  A launch that starts at level 0
// stages input channels and computes the Option-1 partial sums itself.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "fdmt_tables.h"

namespace fdmt {

// Warps per block of the fused kernel (the planner balances work over them).
constexpr int32_t kFusedBlockWarps = 8;
// Row blocks are copied 2^p rows at a time, p <= kMaxBlockP.
constexpr int32_t kMaxBlockP = 5;

// TMA copy into shared memory of rows of the launch's base level (or of
// the input).  Row boxes: global row `row`, columns T0 + xoff + [0, nbox *
// box) in nbox copies of the launch's box width.  Row blocks: rows row ..
// row + 2^nbox - 1, columns T0 + xoff + [0, kchunks * chunk) in one copy,
// landing with row pitch kchunks * chunk.
struct FusedLoad {
  int32_t row;
  int32_t smem;  // byte offset in the block's shared memory
  int32_t xoff;  // first column relative to T0 (<= 0; 16-byte aligned, a chunk multiple for row blocks)
  int32_t nbox;  // row boxes: number of boxes; row blocks: log2 of the rows copied
};

// Option-1 initialisation of one channel inside a cone: rows a..e of
// level 0 over `width` columns, from the staged input row.
struct FusedInit {
  int32_t x_smem;    // byte offset of the staged input sample at the node's time T0 - o
  int32_t dst_smem;  // byte offset of row a of the level-0 node
  int32_t a, e;      // first and last sweep row needed
  int32_t width;     // columns (W + spread)
  int32_t chan;      // channel (for the weight)
  int32_t dst_stride;  // row stride of the node, elements
  int32_t pad;
};

// One output row of one level of a cone:
//   dst[tau] = lo[tau] + hi[tau],  tau in [0, width)
// lo / hi already include the column offsets of their windows; for the top
// level dst is the global row and column tau is time T0 + tau.
struct FusedOp {
  int32_t dst;
  int32_t lo;
  int32_t hi;
  int32_t width;
};

struct FusedTemplate {
  int32_t load_begin, load_count;
  int32_t init_begin, init_count;
  int32_t level_begin;  // index into level_ops: first op of each computed level
  int32_t n_levels;     // computed levels (lt - lb); the last writes global memory
  int32_t tx_bytes;     // bytes the TMA loads deliver
  int32_t smem_bytes;   // dynamic shared memory this template needs
};

struct FusedGroup {
  int32_t lb = 0, lt = 0;
  int32_t W = 0;              // time tile of this launch
  int32_t in_size = 4;        // bytes per staged sample (input, or the level-lb state)
  int32_t out_size = 4;       // bytes per sample of the level-lt state written
  int32_t box = 0;            // row boxes: TMA box width, elements (a multiple of 128 bytes)
  int32_t chunk = 0;          // row blocks (chunk > 0): chunk elements, chunks per copy,
  int32_t kchunks = 0;        //   and the largest copy (2^max_p rows)
  int32_t max_p = 0;
  bool from_input = false;
  int32_t tpl_begin = 0, tpl_count = 0;
  int32_t smem_bytes = 0;     // group-wide layout: barrier + S + Pa + Pb
  int32_t s_end = 0, pa_end = 0;  // byte offsets where S and Pa end
  int64_t ntiles = 0;
  double hbm_bytes = 0;       // model: loaded + written bytes per launch
  double smem_traffic = 0;    // model: shared-memory bytes moved per launch
};

struct FusedParams {
  int32_t W = 0;              // time tile of every group (multiple of 64); 0 = per group by the model
  int32_t smem_budget = 112 * 1024;
  std::vector<int32_t> bounds;  // level boundaries 0 = b0 < b1 < ... = L; empty = choose
  std::vector<int32_t> group_W;       // with bounds: tile per group (0 = W / choose)
  std::vector<int32_t> group_budget;  // with bounds: budget per group (0 = smem_budget)
  int32_t staging = 0;                // 0 = row blocks where nt allows, 1 = row boxes, 2 = row blocks
  bool narrow = false;                // store launch-boundary levels whose uint8 sums fit as uint16
};

struct FusedPlan {
  int32_t W = 0;  // tile of the first group (each group has its own)
  int32_t state_size = 4, input_size = 4, acc_size = 4;
  std::vector<int32_t> level_size;  // [l]: bytes per stored sample of level l (level L: the output)
  std::vector<FusedGroup> groups;
  std::vector<FusedTemplate> tpls;
  std::vector<FusedLoad> loads;
  std::vector<FusedInit> inits;
  std::vector<FusedOp> ops;
  std::vector<int32_t> level_ops;
  // Workspace: intermediate level states between launches (ping-pong).
  size_t ws_split = 0, ws_bytes = 0;
  double model_seconds = 0;
};

// Builds the cone templates for the given parameters.  Returns "" on
// success, else why the schedule does not fit.
std::string plan_fused(const Tables &t, int64_t nt, int32_t state_size, int32_t input_size,
                       const FusedParams &p, FusedPlan &out);

}  // namespace fdmt
