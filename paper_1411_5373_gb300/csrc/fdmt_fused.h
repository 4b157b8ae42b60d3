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

// Compute stages of a work item.  The levels (lb, lt] of a cone are not all
// stored: a stage computes one level from the stored level below it
// (kStageSingle), two levels at once with the level between them never
// stored (kStagePair), or, in a launch that starts at the input, level 1
// straight from the staged input samples (kStageWalk: the Option-1 partial
// sums of level 0 are running sums in registers and are never stored).  The
// last stage writes the group's top level to global memory.
enum : int32_t { kStageWalk = 0, kStageSingle = 1, kStagePair = 2, kStageSearch = 3 };
// Stage word flag: the stage writes the group's top level into shared memory
// in the search layout (pidx) for the search stage that follows it.
constexpr int32_t kStagePadded = 16;
constexpr int32_t kStageKindMask = 15;
// Stage word flag: some op of the stage has a passed-up or one-term half
// (kOpLoOne, kOpHiOne, kOpNoHi; walks: kWalkNoUpper), which only Nf not a
// power of two produces; stages without it run code without those tests.
constexpr int32_t kStageGeneral = 32;

// Boxcar search in the last launch (section 4.2, pulse profile): widths
// 2^k, k < K <= kSearchMaxWidths; the top level's time window carries
// search_hist(K) columns of history before the tile.
#if defined(__CUDACC__)
#define FDMT_HOST_DEVICE __host__ __device__
#else
#define FDMT_HOST_DEVICE
#endif
constexpr int32_t kSearchMaxWidths = 9;
inline int32_t search_hist(int32_t k) { return k <= 1 ? 0 : (((1 << (k - 1)) - 1) + 15) / 16 * 16; }
// Search-layout index of column c of a row of 4-byte values: 4 words of
// padding after every 16 columns (no bank conflicts between the 16-column
// runs of neighbouring lanes).
FDMT_HOST_DEVICE inline int32_t search_pidx(int32_t c) { return c + 4 * (c >> 4); }

// Columns of one op: 32 lanes x kLaneCols columns each (lane l holds columns
// l, l + 32, ...).
#ifndef FDMT_LANE_COLS
#define FDMT_LANE_COLS 8
#endif
constexpr int32_t kLaneCols = FDMT_LANE_COLS;
constexpr int32_t kPieceCols = 32 * kLaneCols;
// Ops read whole pieces whatever their width: the block's shared memory
// ends with this much slack so those reads stay inside it.
constexpr int32_t kOverRead = kPieceCols * 4;
// Op descriptors: each warp copies its ops kDescChunk at a time into its own
// slot of shared memory (one round trip to L2 per chunk) and reads them back
// as broadcasts.  The slots lie between the last region and the slack.
constexpr int32_t kDescChunk = 16;
constexpr int32_t kDescSlotBytes = kDescChunk * 32;  // 32-byte FusedOp
constexpr int32_t kDescBytes = kFusedBlockWarps * kDescSlotBytes;

// Reuse flags of an op, valid against the previous op of the same warp's
// list (same column piece):
//   kOpLoSame  the lower operand (single) or lower half sum (pair) is the
//              previous op's (same lower row: the addition rule's dl did not
//              change);
//   kOpHiShift the upper half sum (pair) is the previous op's one column
//              later (same upper row, dl one larger).
constexpr int32_t kOpLoSame = 1;
constexpr int32_t kOpHiShift = 2;
// Terms of an op where a band has no channel above its border (Nf not a
// power of two, section 4.2: its lower half's rows pass up unchanged):
//   kOpLoOne  the lower half sum is the single term s[p0]
//   kOpHiOne  the upper half sum is the single term s[p2]
//   kOpNoHi   no upper part: the output is the lower part (single: s[p0])
constexpr int32_t kOpLoOne = 4;
constexpr int32_t kOpHiOne = 8;
constexpr int32_t kOpNoHi = 16;
// Walk flag: the band has a single channel (no upper channel).
constexpr int32_t kWalkNoUpper = 1;

// One output row piece of a single or pair stage.  Columns tau in
// [0, width) of the piece:
//   single: out[tau] = s[p0 + tau] + s[p1 + tau]
//   pair:   out[tau] = (s[p0 + tau] + s[p1 + tau]) + (s[p2 + tau] + s[p3 + tau])
// (s = shared memory; p0..p3 are byte offsets that already include the
// sources' column offsets; the bracketing is the level-by-level order).  dst
// is the output's byte offset, or for the top stage its global row, written
// at columns T0 + col + tau.
struct FusedOp {
  int32_t dst;
  int32_t p0, p1, p2, p3;
  int32_t width;
  int32_t flags;
  int32_t col;
};

// Level 1 of one band of two input channels, rows a..e (e - a < 32), over
// one column piece, from the staged samples of the two channels (section 4:
// Option-1 sums, then the addition rule).  Row Dt = dl + j sums
//   x_lo[tau] + ... + x_lo[tau - dl]  and  x_hi[tau - dl] + ... + x_hi[tau - dl - j]
// (each in that order) and adds the two; dl starts at dl0 for row a and
// grows by one at row a + 1 + i when bit i of `bits` is set (else j grows).
struct FusedWalk {
  int32_t dst;      // byte offset of row a at the piece's first column; top stage: global row of row a
  int32_t dst_row;  // bytes from one output row to the next in shared memory
  int32_t x_lo, x_hi;  // byte offsets of the two channels' staged samples at the piece's first column
  int32_t width, col;  // columns of the piece, first column within the tile
  int32_t a, e, dl0;
  int32_t bits;
  int32_t chan;     // lower channel (channel weights; the upper one is chan + 1)
  int32_t flags;    // kWalkNoUpper: a single channel, whose Option-1 rows pass up
};

// Per stage of a template: kind, then the first op (or walk) of each warp
// and the end of the stage's ops.
constexpr int32_t kStageWords = 2 + kFusedBlockWarps;

struct FusedTemplate {
  int32_t load_begin, load_count;
  int32_t walk_begin, walk_count;
  int32_t stage_begin;  // index into FusedPlan::stages (kStageWords per stage)
  int32_t n_stages;     // the last writes global memory
  int32_t tx_bytes;     // bytes the TMA loads deliver
  int32_t smem_bytes;   // dynamic shared memory this template needs
};

// Arguments of a launch that ends with the boxcar search.
struct SearchArgs {
  void *part_v;    // per (row, width, tile): the largest value (A's accumulator type)
  int *part_r;     //   and the region where it first occurs
  int32_t nk;      // widths searched
  int32_t nseg;    // tiles of the launch (partial slots per row and width)
  uint32_t q_off;  // byte offset of the item's per (row, width) bests in shared memory
  uint32_t q_row;  //   and their bytes
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
  int32_t smem_bytes = 0;     // group-wide layout: barrier + S + Pa + Pb (+ Pt + Q with a search)
  int32_t s_end = 0, pa_end = 0;  // byte offsets where S and Pa end
  int32_t search_k = 0;       // boxcar widths searched in this launch (0 = none; last group only)
  int32_t hist = 0;           // history columns of the top level's window (search)
  int32_t q_off = 0;          // search: byte offset of an item's per (row, width) bests
  int32_t q_row = 0;          //   and their bytes
  int64_t ntiles = 0;
  double hbm_bytes = 0;       // model: loaded + written bytes per launch
  double smem_traffic = 0;    // model: shared-memory bytes moved per launch
  double ops = 0;             // model: ops and walks per launch
  double block_slots = 0;     // model: resident blocks on the GPU
  double seconds = 0;         // model: launch time
};

struct FusedParams {
  int32_t W = 0;              // time tile of every group (multiple of 64); 0 = per group by the model
  int32_t smem_budget = 112 * 1024;
  std::vector<int32_t> bounds;  // level boundaries 0 = b0 < b1 < ... = L; empty = choose
  std::vector<int32_t> group_W;       // with bounds: tile per group (0 = W / choose)
  std::vector<int32_t> group_budget;  // with bounds: budget per group (0 = smem_budget)
  int32_t staging = 0;                // 0 = row blocks where nt allows, 1 = row boxes, 2 = row blocks
  bool narrow = false;                // store launch-boundary levels whose uint8 sums fit as uint16
  int32_t search_k = 0;               // boxcar widths searched by the last launch (0 = none)
};

struct FusedPlan {
  int32_t W = 0;  // tile of the first group (each group has its own)
  int32_t state_size = 4, input_size = 4, acc_size = 4;
  std::vector<int32_t> level_size;  // [l]: bytes per stored sample of level l (level L: the output)
  std::vector<FusedGroup> groups;
  std::vector<FusedTemplate> tpls;
  std::vector<FusedLoad> loads;
  std::vector<FusedWalk> walks;
  std::vector<FusedOp> ops;
  std::vector<int32_t> stages;
  // Workspace: intermediate level states between launches (ping-pong).
  size_t ws_split = 0, ws_bytes = 0;
  double model_seconds = 0;
  bool general = false;  // some stage holds passed-up or one-term halves (kStageGeneral)
};

// Levels a group (lb, lt] keeps in shared memory (see fdmt_fused_plan.cpp).
std::vector<int32_t> stored_levels(int32_t lb, int32_t lt);

// Builds the cone templates for the given parameters.  Returns "" on
// success, else why the schedule does not fit.
std::string plan_fused(const Tables &t, int64_t nt, int32_t state_size, int32_t input_size,
                       const FusedParams &p, FusedPlan &out);

}  // namespace fdmt
