// Delay tables of the FDMT, built once per plan on the host in FP64.
//
// Section 4 of Zackay & Ofek (arXiv:1411.5373): iteration l merges pairs of
// sub-bands of 2^(l-1) channels.  A band [f0, f2] with border f1 combines its
// halves by the addition rule
//     A_{f0}^{f2}(t0, Dt) = A_{f0}^{f1}(t0, dl) + A_{f1}^{f2}(t0 - dl, Dt - dl)
// where dl rounds C * Dt and C = (f0^-2 - f1^-2) / (f0^-2 - f2^-2) is
// Eq. (C_{f2,f0}); for another functional form Dt ~ f^gamma (section 4.2)
// the power -2 becomes gamma.  Rounding: dl = floor(C * Dt + 1/2).  Channels are
// intervals of width (f_max - f_min) / Nf; f1 is the border between the two
// halves (the paper's "f1 = (f2 - f0)/2" is read as that border).
//
// Nf need not be a power of two: band b of level l spans channels
// [b 2^l, min((b+1) 2^l, Nf)), so the last band of a level may be narrower
// and split unequally at its border (section 4.2); a band with no channel
// above the border is its lower sub-band passed up unchanged.
//
// Row extents are sized from the top: the whole band has Nd rows and each
// half holds exactly the rows its parent reads.  Because dl and Dt - dl are
// both non-decreasing in Dt with steps of 0 or 1, every child row from 0 to
// the largest one read is read at least once, by a contiguous run of parent
// rows -- which is what makes the gather-form transpose (AdjOp) possible.
//
// This file must be compiled without floating-point contraction
// (-ffp-contract=off) so that the FP64 expressions round exactly as written
// on every host architecture.
#include "fdmt_tables.h"

#include <algorithm>
#include <cmath>
#include <cstdio>

namespace fdmt {

double channel_edge(double f_min, double f_max, int32_t nf, int64_t k) {
  return f_min + (f_max - f_min) * (double)k / (double)nf;
}

static double inv_sq(double f) { return 1.0 / (f * f); }

// f^gamma; the dispersion law's f^-2 as 1 / (f f).
static double power_law(double f, double gamma) { return gamma == -2.0 ? inv_sq(f) : std::pow(f, gamma); }

int32_t bands_at(int32_t nf, int32_t l) { return (int32_t)(((int64_t)nf + ((int64_t)1 << l) - 1) >> l); }

bool has_upper(const Tables &t, int32_t l, int32_t b) {
  return 2 * (size_t)b + 1 < t.band_rows[l - 1].size();
}

std::vector<int32_t> input_shifts(double f_min, double f_max, int32_t nf, int32_t d_min, double gamma) {
  std::vector<int32_t> s((size_t)nf, 0);
  const double p0 = power_law(f_min, gamma), p1 = power_law(f_max, gamma);
  for (int32_t k = 0; k < nf; ++k) {
    const double r = (p0 - power_law(channel_edge(f_min, f_max, nf, k), gamma)) / (p0 - p1);
    s[(size_t)k] = (int32_t)std::floor((double)d_min * r + 0.5);
  }
  return s;
}

std::string build_tables(double f_min, double f_max, int32_t nf, int32_t nd, Tables &t, double gamma) {
  if (!std::isfinite(gamma) || gamma == 0.0) return "gamma must be finite and nonzero";
  if (!std::isfinite(f_min) || !std::isfinite(f_max) || !(f_min > 0.0) || !(f_max > f_min))
    return "need 0 < f_min < f_max (finite)";
  if (nf < 2) return "nf must be >= 2";
  if (nd < 1) return "nd must be >= 1";
  if ((int64_t)nf + (int64_t)nd > (int64_t)1 << 30) return "nf + nd too large";

  int32_t L = 0;  // ceil(log2 nf)
  while ((1 << L) < nf) ++L;
  t = Tables();
  t.f_min = f_min;
  t.f_max = f_max;
  t.nf = nf;
  t.nd = nd;
  t.levels = L;
  t.band_rows.assign(L + 1, {});
  t.band_row0.assign(L + 1, {});
  t.dl.assign(L + 1, {});
  t.level_rows.assign(L + 1, 0);

  // Top-down row extents and lower-row tables.
  t.band_rows[L] = {nd};
  for (int32_t l = L; l >= 1; --l) {
    const int32_t nb = bands_at(nf, l);
    t.band_rows[l - 1].assign(bands_at(nf, l - 1), 0);
    t.dl[l].assign(nb, {});
    for (int32_t b = 0; b < nb; ++b) {
      const int64_t k0 = (int64_t)b << l, k1 = k0 + ((int64_t)1 << (l - 1));
      const int32_t rows = t.band_rows[l][b];
      if (k1 >= nf) {
        // No channel above the border: the band passes up unchanged.
        std::vector<int32_t> &dl = t.dl[l][b];
        dl.resize(rows);
        for (int32_t dt = 0; dt < rows; ++dt) dl[dt] = dt;
        t.band_rows[l - 1][2 * b] = rows;
        continue;
      }
      const int64_t k2 = std::min<int64_t>(k0 + ((int64_t)1 << l), nf);
      const double f0 = channel_edge(f_min, f_max, nf, k0);
      const double f1 = channel_edge(f_min, f_max, nf, k1);
      const double f2 = channel_edge(f_min, f_max, nf, k2);
      const double q0 = power_law(f0, gamma), q1 = power_law(f1, gamma), q2 = power_law(f2, gamma);
      const double c = (q0 - q1) / (q0 - q2);
      std::vector<int32_t> &dl = t.dl[l][b];
      dl.resize(rows);
      for (int32_t dt = 0; dt < rows; ++dt) dl[dt] = (int32_t)std::floor(c * (double)dt + 0.5);
      // Sanity of the monotone-step property the kernels rely on.
      for (int32_t dt = 1; dt < rows; ++dt) {
        const int32_t a = dl[dt] - dl[dt - 1];
        if (a < 0 || a > 1) return "internal: dl table is not a 0/1-step sequence";
      }
      if (dl[0] != 0) return "internal: dl[0] != 0";
      t.band_rows[l - 1][2 * b] = dl[rows - 1] + 1;
      t.band_rows[l - 1][2 * b + 1] = (rows - 1) - dl[rows - 1] + 1;
    }
  }

  // Absolute first row of every band within its level.
  for (int32_t l = 0; l <= L; ++l) {
    const size_t nb = t.band_rows[l].size();
    t.band_row0[l].assign(nb, 0);
    int64_t acc = 0;
    for (size_t b = 0; b < nb; ++b) {
      t.band_row0[l][b] = (int32_t)acc;
      acc += t.band_rows[l][b];
    }
    t.level_rows[l] = (int32_t)acc;
  }

  // Level 0: one InitOp per channel.
  t.init.resize(nf);
  t.max_sweep = 0;
  for (int32_t k = 0; k < nf; ++k) {
    t.init[k].row0 = t.band_row0[0][k];
    t.init[k].sweep = t.band_rows[0][k] - 1;
    if (t.init[k].sweep > t.max_sweep) t.max_sweep = t.init[k].sweep;
  }

  // Forward row program of levels 1..L.
  t.ops.clear();
  t.ops_begin.assign(L + 2, 0);
  for (int32_t l = 1; l <= L; ++l) {
    t.ops_begin[l] = (int64_t)t.ops.size();
    const int32_t nb = bands_at(nf, l);
    for (int32_t b = 0; b < nb; ++b) {
      const int32_t lo0 = t.band_row0[l - 1][2 * b];
      if (!has_upper(t, l, b)) {  // copy: no upper term
        for (int32_t dt = 0; dt < t.band_rows[l][b]; ++dt) t.ops.push_back(RowOp{lo0 + dt, -1, 0, b});
        continue;
      }
      const int32_t hi0 = t.band_row0[l - 1][2 * b + 1];
      for (int32_t dt = 0; dt < t.band_rows[l][b]; ++dt) {
        const int32_t j = t.dl[l][b][dt];
        t.ops.push_back(RowOp{lo0 + j, hi0 + (dt - j), j, b});
      }
    }
  }
  t.ops_begin[L + 1] = (int64_t)t.ops.size();

  // Transposed program: for each child row of level l-1, the run of parent
  // rows of level l that read it.
  t.adj.clear();
  t.adj_begin.assign(L + 1, 0);
  for (int32_t l = 1; l <= L; ++l) {
    t.adj_begin[l - 1] = (int64_t)t.adj.size();
    const int32_t nb = bands_at(nf, l);
    for (int32_t b = 0; b < nb; ++b) {
      const int32_t p0 = t.band_row0[l][b];
      const int32_t rows = t.band_rows[l][b];
      const std::vector<int32_t> &dl = t.dl[l][b];
      if (!has_upper(t, l, b)) {  // child row dt is parent row dt
        for (int32_t dt = 0; dt < rows; ++dt) t.adj.push_back(AdjOp{p0 + dt, 1, 0, 0});
        continue;
      }
      const int32_t n_lo = t.band_rows[l - 1][2 * b];
      const int32_t n_hi = t.band_rows[l - 1][2 * b + 1];
      std::vector<AdjOp> lo(n_lo, AdjOp{0, 0, 0, 0}), hi(n_hi, AdjOp{0, 0, 0, 1});
      for (int32_t dt = 0; dt < rows; ++dt) {
        AdjOp &a = lo[dl[dt]];
        if (a.count == 0) a.first = p0 + dt;
        ++a.count;
        const int32_t m = dt - dl[dt];
        AdjOp &h = hi[m];
        if (h.count == 0) {
          h.first = p0 + dt;
          h.shift0 = dl[dt];
        }
        ++h.count;
      }
      for (const AdjOp &a : lo)
        if (a.count == 0) return "internal: lower child row never read";
      for (const AdjOp &a : hi)
        if (a.count == 0) return "internal: upper child row never read";
      t.adj.insert(t.adj.end(), lo.begin(), lo.end());
      t.adj.insert(t.adj.end(), hi.begin(), hi.end());
    }
  }
  t.adj_begin[L] = (int64_t)t.adj.size();

  // Two transposed levels composed (levels l and l - 1 into l - 2): the
  // terms of child c are, for each level-(l-1) row r it reads with shift s1,
  // the level-l rows r reads with shift s2, at shift s1 + s2.
  t.adj2.clear();
  t.adj2_terms.clear();
  t.adj2_begin.assign(L + 1, 0);
  for (int32_t c_level = 0; c_level + 2 <= L; ++c_level) {
    t.adj2_begin[c_level] = (int64_t)t.adj2.size();
    for (int32_t c = 0; c < t.level_rows[c_level]; ++c) {
      const AdjOp &a1 = t.adj[t.adj_begin[c_level] + c];
      AdjRun run{(int32_t)t.adj2_terms.size(), 0};
      for (int32_t i = 0; i < a1.count; ++i) {
        const int32_t r = a1.first + i, s1 = a1.shift0 + i * a1.step;
        const AdjOp &a2 = t.adj[t.adj_begin[c_level + 1] + r];
        for (int32_t j = 0; j < a2.count; ++j) {
          t.adj2_terms.push_back(AdjTerm{a2.first + j, s1 + a2.shift0 + j * a2.step});
          ++run.count;
        }
      }
      t.adj2.push_back(run);
    }
  }
  t.adj2_begin[L] = (int64_t)t.adj2.size();
  return "";
}

}  // namespace fdmt
