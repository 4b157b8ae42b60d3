// Host-side delay-table builder for the FDMT (section 4, Algorithm 1 of
// Zackay & Ofek, arXiv:1411.5373).  FP64 arithmetic, int32 results; the
// kernels only ever see the integer tables produced here.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace fdmt {

// One output row of a merge level: next[row] = prev[lo] + prev[hi] shifted
// later by `shift` samples (zero before t = shift: the copy rule).
struct RowOp {
  int32_t lo;     // absolute row of the lower sub-band in the previous level
  int32_t hi;     // absolute row of the upper sub-band in the previous level;
                  // < 0: no upper sub-band, the row is a copy of `lo`
  int32_t shift;  // samples the upper sub-band arrives earlier (= dl)
  int32_t band;   // band index within the level (for diagnostics / fused tiles)
};

// One row of the transposed merge: child[row][u] =
//   sum_{i < count} parent[first + i][u + shift0 + i * step]   (u + shift < Nt)
// Two transposed levels composed: child row c of level l - 2 gathers
// parent rows of level l, term k being parent[row][u + shift].
struct AdjTerm {
  int32_t row;    // absolute parent row (level l)
  int32_t shift;  // time offset of this contribution
};
struct AdjRun {
  int32_t first;  // first term
  int32_t count;  // terms
};

struct AdjOp {
  int32_t first;   // absolute parent row (level l) of the first contribution
  int32_t count;   // number of parent rows reading this child row
  int32_t shift0;  // time offset of the first contribution
  int32_t step;    // 0 for a lower child (no shift), 1 for an upper child
};

// Level-0 rows of one channel: rows [row0, row0 + sweep] hold the partial
// sums over 1 .. sweep+1 consecutive samples (Option-1 initialisation).
struct InitOp {
  int32_t row0;
  int32_t sweep;
};

struct Tables {
  double f_min = 0, f_max = 0;
  int32_t nf = 0, nd = 0, levels = 0;
  // band_rows[l][b], band_row0[l][b]: rows of band b at level l and the
  // absolute index of its first row in the level's state.
  std::vector<std::vector<int32_t>> band_rows, band_row0;
  std::vector<int32_t> level_rows;                       // total rows per level
  std::vector<std::vector<std::vector<int32_t>>> dl;     // [l][b][Dt], l >= 1
  std::vector<InitOp> init;                              // per channel
  std::vector<RowOp> ops;                                // levels 1..L concatenated
  std::vector<int64_t> ops_begin;                        // [l] first op of level l (l>=1)
  std::vector<AdjOp> adj;                                // child rows of levels 0..L-1
  std::vector<int64_t> adj_begin;                        // [l] first adj op for level-l children
  std::vector<AdjRun> adj2;                              // composed pairs: child rows of levels 0..L-2
  std::vector<AdjTerm> adj2_terms;
  std::vector<int64_t> adj2_begin;                       // [l] first run for level-l children (l <= L-2)
  int32_t max_sweep = 0;
};

// Edge k of the channel grid: f_min + ((f_max - f_min) * k) / nf.
double channel_edge(double f_min, double f_max, int32_t nf, int64_t k);

// Returns an empty string on success, else a description of the bad argument.
// gamma: the curves' power law Dt ~ f^gamma (-2: cold-plasma dispersion).
std::string build_tables(double f_min, double f_max, int32_t nf, int32_t nd, Tables &t, double gamma = -2.0);

// Bands of level l: ceil(nf / 2^l); band b spans channels
// [b 2^l, min((b+1) 2^l, nf)).  Nf not a power of two (section 4.2: the
// split is unequal, f1 the border): a band with no channel above its border
// has no upper sub-band and passes its lower one up unchanged (RowOp.hi < 0).
int32_t bands_at(int32_t nf, int32_t l);
bool has_upper(const Tables &t, int32_t l, int32_t b);

// Delay of channel k's lower edge e_k for total delay d_min (the d_min
// pre-shift of section 4.2): s_k = floor(d_min r(e_k) + 1/2), r(f) =
// (f_min^gamma - f^gamma) / (f_min^gamma - f_max^gamma), FP64 in this order.
std::vector<int32_t> input_shifts(double f_min, double f_max, int32_t nf, int32_t d_min, double gamma = -2.0);

}  // namespace fdmt
