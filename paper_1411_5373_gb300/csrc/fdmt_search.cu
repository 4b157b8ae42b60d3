// Boxcar search of an FDMT output (contracts in include/fdmt.h).
//
// Section 4.2 ("Pulse profile") of Zackay & Ofek (arXiv:1411.5373): a
// uniform pulse profile convolved with the time axis commutes with the whole
// transform, so several widths are tested on one output.  For width
// w = 2^k and row d, B_w[d][t] = sum_{i<w} A[d][t - i] (zero before t = 0)
// is summed as a binary tree, B_1 = A and B_2w[t] = B_w[t] + B_w[t - w];
// the result per (row, width) is the maximum over t and the first t that
// reaches it.  Integer outputs are summed exactly (int32 when the caller's
// bound on |A| proves it cannot overflow, else int64), float outputs in
// float32 with that tree order, so every B value is bit-identical to a plain
// evaluation of the recursion.
//
// Two kernels.
//
// search_kernel streams the rows.  Work items are (row, segment of `seg`
// samples), row-major; each persistent block takes a contiguous range of
// items, so it walks along a few rows and the history below each segment
// (`halo` >= 2^(K-1) - 1 samples) was read by the same block just before.
// Each item's window (history + segment) is copied into shared memory with
// cp.async while the previous item is being searched.  The widths are built
// in phases of four doublings: a thread holds a run of 16 columns of B_S at
// stride S (S = 1, 16, 256) plus the 16 before them, doubles four times in
// registers (B_2S .. B_16S) and stores B_16S for the next phase, so shared
// memory sees two reads and one write per column per four widths.  For each
// width a thread keeps only the largest value seen and the REGION of 16*S
// consecutive samples (its run, or its group of runs) where it first saw
// it; the block merges them when its walk leaves a row and writes one
// (value, region) per (row, width, first segment of the walk).
//
// search_finalize_kernel (one block per row) takes per width the largest
// value and the earliest region holding it, recomputes that width over the
// region from A (the same additions in the same order), and returns the
// first time in it where the value occurs.  Any earlier occurrence would sit
// in an earlier region, so that time is the first one of the whole row.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>

#include "../../include/fdmt.h"
#include "fdmt_internal.h"

namespace fdmt {
namespace {

constexpr int kSearchThreads = 256;
constexpr int kPass = kSearchThreads * 16;  // columns one phase pass covers
constexpr int kMaxWidths = 13;
constexpr int kWarps = kSearchThreads / 32;
constexpr int kMaxSeg = 3 * kPass;
constexpr int kNoRegion = INT32_MIN;
constexpr int kFinalizeElems = kPass + (1 << (kMaxWidths - 1));  // widest region + history
constexpr int kFinalizeWarpElems = 512;                          // 256-sample region + history

// Shared-memory layout of window column c: 16 bytes of padding after each
// run of 16 columns, so the 16-column runs of consecutive threads fall on
// different banks.
template <class T>
__host__ __device__ constexpr int pidx(int c) {
  return c + (int)(16 / sizeof(T)) * (c >> 4);
}

__device__ __forceinline__ float add_tree(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ int32_t add_tree(int32_t a, int32_t b) { return a + b; }
__device__ __forceinline__ int64_t add_tree(int64_t a, int64_t b) { return a + b; }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ int32_t vmax(int32_t a, int32_t b) { return max(a, b); }
__device__ __forceinline__ int64_t vmax(int64_t a, int64_t b) { return a > b ? a : b; }
template <class T> __device__ __forceinline__ T lowest();
template <> __device__ __forceinline__ float lowest<float>() { return -__int_as_float(0x7f800000); }
template <> __device__ __forceinline__ int32_t lowest<int32_t>() { return INT32_MIN; }
template <> __device__ __forceinline__ int64_t lowest<int64_t>() { return LLONG_MIN; }

// log2 of the stride of the phase that builds width index k.
__host__ __device__ constexpr int stride_log2(int k) { return k <= 4 ? 0 : (k <= 8 ? 4 : 8); }

// Max of x[16..31] over the columns col0 + S*i inside [lo, hi) joins the
// running best (bv, br) with `region` when it is larger (a tie keeps the
// earlier region, so each thread keeps the first region of its maximum).
// `full`: all 16 columns are inside.  The running best starts at -inf with
// no region, so a run of finite values always takes it.
template <class TB, int S>
__device__ __forceinline__ void track(const TB (&x)[32], bool full, int col0, int lo, int hi, int region, TB &bv,
                                      int &br) {
  TB m;
  if (full) {
    TB t[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) t[i] = vmax(x[16 + i], x[24 + i]);
#pragma unroll
    for (int i = 0; i < 4; ++i) t[i] = vmax(t[i], t[i + 4]);
    m = vmax(vmax(t[0], t[2]), vmax(t[1], t[3]));
  } else {
    m = lowest<TB>();
#pragma unroll
    for (int i = 16; i < 32; ++i) {
      const int c = col0 + S * (i - 16);
      if (c >= lo && c < hi) m = vmax(m, x[i]);
    }
  }
  const bool up = m > bv;
  bv = up ? m : bv;
  br = up ? region : br;
}

// One phase: B_S (src, element type TS, written at the columns >= src_lo)
// -> B_2S .. B_16S at the columns [lo, n) (the widest also to dst, if any).
// Width indices K0 .. K0+3 are tracked while below nk, and index 0 (B_1
// itself) when S == 1.  t0 = time of window column 0.
template <class TS, class TB, int S>
__device__ __forceinline__ void phase(const TS *src, TB *dst, int src_lo, int n, int lo, int halo, int lim,
                                      int nk, int t0, TB (&bv)[kMaxWidths], int (&br)[kMaxWidths]) {
  constexpr int G = 16 * S;                           // columns of one thread group
  constexpr int K0 = S == 1 ? 1 : (S == 16 ? 5 : 9);  // width index of 2S
  constexpr int P = 16 / (int)sizeof(TS);             // padding elements per run of src
  const int r = threadIdx.x % S, gi = threadIdx.x / S;
  for (int pass = lo; pass < n; pass += kPass) {
    const int base = pass + gi * G;
    if (base >= n) break;
    TB x[32];
    bool full;
    if (S == 1) {
      // Two whole runs: columns base - 16 .. base + 15 (n is a multiple of 16).
      constexpr int E = 16 / sizeof(TS);
      const int4 *lo_run = reinterpret_cast<const int4 *>(src + pidx<TS>(base >= 16 ? base - 16 : 0));
      const int4 *hi_run = reinterpret_cast<const int4 *>(src + pidx<TS>(base));
#pragma unroll
      for (int v = 0; v < 16 / E; ++v) {
        const int4 a = base >= 16 ? lo_run[v] : make_int4(0, 0, 0, 0);
        const int4 b = hi_run[v];
        const TS *pa = reinterpret_cast<const TS *>(&a);
        const TS *pb = reinterpret_cast<const TS *>(&b);
#pragma unroll
        for (int e = 0; e < E; ++e) {
          x[v * E + e] = (TB)pa[e];
          x[16 + v * E + e] = (TB)pb[e];
        }
      }
      full = base >= halo && base + 15 < lim;
      if (full || (base + 15 >= halo && base < lim)) track<TB, 1>(x, full, base, halo, lim, t0 + base, bv[0], br[0]);
    } else {
      full = base + r >= halo && base + r + 15 * S < lim;
      const int c0 = base + r - 16 * S;
      if (c0 >= src_lo && c0 + 31 * S < n) {
        // Interior: column c0 + S*j sits at a fixed stride in the padded layout.
        const TS *p = src + pidx<TS>(c0);
#pragma unroll
        for (int j = 0; j < 32; ++j) x[j] = (TB)p[j * (S + P * (S / 16))];
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int c = c0 + S * j;
          x[j] = (c >= src_lo && c < n) ? (TB)src[pidx<TS>(c)] : TB(0);
        }
      }
    }
#pragma unroll
    for (int m = 1; m <= 4; ++m) {
      if (dst == nullptr && K0 + m - 1 >= nk) break;
      const int h = 1 << (m - 1);
#pragma unroll
      for (int i = 31; i >= (1 << m); --i) x[i] = add_tree(x[i], x[i - h]);
      const bool any = full || (base + r + 15 * S >= halo && base + r < lim);
      if (K0 + m - 1 < nk && any)
        track<TB, S>(x, full, base + r, halo, lim, t0 + base, bv[K0 + m - 1], br[K0 + m - 1]);
    }
    if (dst != nullptr) {
      if (S == 1) {
        constexpr int E = 16 / sizeof(TB);
        int4 *out = reinterpret_cast<int4 *>(dst + pidx<TB>(base));
#pragma unroll
        for (int v = 0; v < 16 / E; ++v) {
          int4 o;
          TB *po = reinterpret_cast<TB *>(&o);
#pragma unroll
          for (int e = 0; e < E; ++e) po[e] = x[16 + v * E + e];
          out[v] = o;
        }
      } else {
        constexpr int PB = 16 / (int)sizeof(TB);
        const int c0 = base + r;
        if (c0 + 15 * S < n) {
          TB *p = dst + pidx<TB>(c0);
#pragma unroll
          for (int j = 16; j < 32; ++j) p[(j - 16) * (S + PB * (S / 16))] = x[j];
        } else {
#pragma unroll
          for (int j = 16; j < 32; ++j) {
            const int c = c0 + S * (j - 16);
            if (c < n) dst[pidx<TB>(c)] = x[j];
          }
        }
      }
    }
  }
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Copy window columns [0, n) (times t0 ..) of a row into buf, zeros outside
// [0, nt): 16-byte asynchronous copies when rows are 16-byte aligned, else
// plain loads and stores.  Commits one cp.async group either way.
template <class TA>
__device__ __forceinline__ void stage_window(TA *buf, const TA *row, int t0, int nt, int n, int vec) {
  for (int c = 4 * threadIdx.x; c < n; c += 4 * kSearchThreads) {
    const int t = t0 + c;
    if (vec) {
      const bool in = t >= 0 && t < nt;  // nt % 4 == 0: a vector is all in or all out
      cp_async16(buf + pidx<TA>(c), in ? row + t : row, in ? 16 : 0);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) buf[pidx<TA>(c + e)] = (t + e >= 0 && t + e < nt) ? row[t + e] : TA(0);
    }
  }
  cp_async_commit();
}

struct SearchGeom {
  int seg, halo, n, lo1, lo16, lo256;
};

template <class TB>
struct RowBest {
  TB v[kMaxWidths][kWarps];
  int r[kMaxWidths][kWarps];
};

// Merge the block's running bests of row d (segments s_first .. s_last) and
// write them to partial slot s_first; the other slots of the walk are marked
// empty.  Resets the running bests.
template <class TB>
__device__ __forceinline__ void flush_row(TB (&bv)[kMaxWidths], int (&br)[kMaxWidths], int nk, RowBest<TB> &red,
                                          int64_t d, int s_first, int s_last, int nseg, TB *part_v, int *part_r) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < kMaxWidths; ++k) {
    if (k >= nk) break;
    TB m = br[k] == kNoRegion ? lowest<TB>() : bv[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = vmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    int reg = (br[k] != kNoRegion && bv[k] == m) ? br[k] : INT32_MAX;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) reg = min(reg, __shfl_xor_sync(0xffffffffu, reg, o));
    if (lane == 0) {
      red.v[k][warp] = m;
      red.r[k][warp] = reg == INT32_MAX ? kNoRegion : reg;
    }
    bv[k] = lowest<TB>();
    br[k] = kNoRegion;
  }
  __syncthreads();
  if (threadIdx.x < nk) {
    const int k = threadIdx.x;
    TB m = lowest<TB>();
    int reg = kNoRegion;
    for (int w = 0; w < kWarps; ++w) {
      const int rw = red.r[k][w];
      if (rw == kNoRegion) continue;
      if (reg == kNoRegion || red.v[k][w] > m || (red.v[k][w] == m && rw < reg)) {
        m = red.v[k][w];
        reg = rw;
      }
    }
    const int64_t row = (d * nk + k) * nseg;
    part_v[row + s_first] = m;
    part_r[row + s_first] = reg;
    for (int s = s_first + 1; s <= s_last; ++s) part_r[row + s] = kNoRegion;
  }
  // red is rewritten at the next flush, after the next item's barriers.
}

// MINB = resident blocks per SM the registers must allow: 3 for the
// narrow windows of K <= 9 with 4-byte sums (shared memory allows more), 1
// for K >= 10 (one block's windows fill the SM) and for int64 sums.
template <class TA, class TB, int MINB>
__global__ void __launch_bounds__(kSearchThreads, MINB)
search_kernel(const TA *__restrict__ A, int nt, int nk, SearchGeom g, int nseg, int items, int per_block, int vec,
              TB *__restrict__ part_v, int *__restrict__ part_r) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ RowBest<TB> red;
  const int n = g.n, halo = g.halo;
  const size_t a_bytes = (size_t)pidx<TA>(n) * sizeof(TA);
  const size_t b_bytes = (size_t)pidx<TB>(n) * sizeof(TB);
  TA *const abuf0 = reinterpret_cast<TA *>(smem);
  TA *const abuf1 = reinterpret_cast<TA *>(smem + a_bytes);
  TB *const b16 = reinterpret_cast<TB *>(smem + 2 * a_bytes);
  TB *const b256 = reinterpret_cast<TB *>(smem + 2 * a_bytes + b_bytes);
  const int begin = blockIdx.x * per_block;
  const int end = min(begin + per_block, items);
  if (begin >= end) return;
  TB bv[kMaxWidths];
  int br[kMaxWidths];
#pragma unroll
  for (int k = 0; k < kMaxWidths; ++k) {
    bv[k] = lowest<TB>();
    br[k] = kNoRegion;
  }
  int d = begin / nseg, s = begin - d * nseg;
  int s_first = s;
  stage_window(abuf0, A + (int64_t)d * nt, s * g.seg - halo, nt, n, vec);
  for (int item = begin; item < end; ++item) {
    const int it = item - begin;
    if (item + 1 < end) {
      const int dn = s + 1 == nseg ? d + 1 : d, sn = s + 1 == nseg ? 0 : s + 1;
      stage_window((it & 1) ? abuf0 : abuf1, A + (int64_t)dn * nt, sn * g.seg - halo, nt, n, vec);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int t0 = s * g.seg - halo;
    const int lim = halo + min(g.seg, nt - s * g.seg);
    phase<TA, TB, 1>((it & 1) ? abuf1 : abuf0, nk > 5 ? b16 : nullptr, 0, n, g.lo1, halo, lim, nk, t0, bv, br);
    if (nk > 5) {
      __syncthreads();
      phase<TB, TB, 16>(b16, nk > 9 ? b256 : nullptr, g.lo1, n, g.lo16, halo, lim, nk, t0, bv, br);
      if (nk > 9) {
        __syncthreads();
        phase<TB, TB, 256>(b256, nullptr, g.lo16, n, g.lo256, halo, lim, nk, t0, bv, br);
      }
    }
    if (s + 1 == nseg || item + 1 == end) flush_row(bv, br, nk, red, d, s_first, s, nseg, part_v, part_r);
    __syncthreads();  // this window buffer is refilled next
    if (++s == nseg) {
      s = 0;
      ++d;
    }
    if (s == 0) s_first = 0;
  }
}

// Per row d: for each width the largest partial value and the earliest
// region holding it; then that width recomputed over the region (in place,
// the additions of the tree in the same order) and the first time with the
// value.  Widths of regions up to 256 samples go one per warp, wider ones
// use the whole block.
template <class TA, class TB, class TP>
__global__ void __launch_bounds__(kSearchThreads)
search_finalize_kernel(const TA *__restrict__ A, int nt, int nk, int nseg, const TB *__restrict__ part_v,
                       const int *__restrict__ part_r, TP *__restrict__ peak, int32_t *__restrict__ time) {
  extern __shared__ __align__(16) unsigned char smem[];
  TB *buf = reinterpret_cast<TB *>(smem);
  __shared__ TB s_m[kMaxWidths];
  __shared__ int s_r[kMaxWidths];
  __shared__ int s_t;
  const int d = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;  // kWarps, or fewer when K <= 9
  const TA *row = A + (int64_t)d * nt;
  for (int k = warp; k < nk; k += nwarps) {
    const int64_t base = ((int64_t)d * nk + k) * nseg;
    TB m = lowest<TB>();
    int reg = kNoRegion;
    for (int s = lane; s < nseg; s += 32) {
      const int rs = part_r[base + s];
      if (rs == kNoRegion) continue;
      const TB v = part_v[base + s];
      if (reg == kNoRegion || v > m || (v == m && rs < reg)) {
        m = v;
        reg = rs;
      }
    }
    TB mm = reg == kNoRegion ? lowest<TB>() : m;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mm = vmax(mm, __shfl_xor_sync(0xffffffffu, mm, o));
    int rr = (reg != kNoRegion && m == mm) ? reg : INT32_MAX;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rr = min(rr, __shfl_xor_sync(0xffffffffu, rr, o));
    if (lane == 0) {
      s_m[k] = mm;
      s_r[k] = rr;
    }
  }
  __syncthreads();
  // Regions of 16 or 256 samples: one warp per width, in place in its slice.
  for (int k = warp; k < nk && k <= 8; k += nwarps) {
    if (s_r[k] == INT32_MAX) {  // no finite candidate (only possible for non-finite input)
      if (lane == 0) {
        peak[(int64_t)d * nk + k] = (TP)s_m[k];
        time[(int64_t)d * nk + k] = 0;
      }
      continue;
    }
    TB *wb = buf + warp * kFinalizeWarpElems;
    const int w = 1 << k, L = 16 << stride_log2(k);
    const int t_lo = s_r[k] - (w - 1), cnt = L + w - 1;
    for (int i = lane; i < cnt; i += 32) {
      const int t = t_lo + i;
      wb[i] = (t >= 0 && t < nt) ? (TB)row[t] : TB(0);
    }
    __syncwarp();
    for (int h = 1; h < w; h *= 2) {
      for (int top = cnt; top > 0; top -= 128) {  // in place, chunks from the top down
        const int lo_i = top - 128;
        TB nv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int i = lo_i + lane + 32 * j;
          if (i >= 0 && i < top) nv[j] = i >= h ? add_tree(wb[i], wb[i - h]) : wb[i];
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int i = lo_i + lane + 32 * j;
          if (i >= 0 && i < top) wb[i] = nv[j];
        }
        __syncwarp();
      }
    }
    int first = INT32_MAX;
    for (int i = w - 1 + lane; i < cnt; i += 32) {
      const int t = t_lo + i;
      if (t >= 0 && t < nt && wb[i] == s_m[k]) {
        first = t;
        break;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
    if (lane == 0) {
      peak[(int64_t)d * nk + k] = (TP)s_m[k];
      time[(int64_t)d * nk + k] = first == INT32_MAX ? 0 : first;
    }
  }
  // Regions of 4096 samples: the whole block, one width at a time.
  for (int k = 9; k < nk; ++k) {
    __syncthreads();
    if (s_r[k] == INT32_MAX) {
      if (threadIdx.x == 0) {
        peak[(int64_t)d * nk + k] = (TP)s_m[k];
        time[(int64_t)d * nk + k] = 0;
      }
      continue;
    }
    const int w = 1 << k, L = 16 << stride_log2(k);
    const int t_lo = s_r[k] - (w - 1), cnt = L + w - 1;
    for (int i = threadIdx.x; i < cnt; i += kSearchThreads) {
      const int t = t_lo + i;
      buf[i] = (t >= 0 && t < nt) ? (TB)row[t] : TB(0);
    }
    if (threadIdx.x == 0) s_t = INT32_MAX;
    __syncthreads();
    // In place, in chunks from the top down: a chunk reads itself and the
    // chunks below it (still old) before it is written.
    for (int h = 1; h < w; h *= 2) {
      for (int top = cnt; top > 0; top -= 4 * kSearchThreads) {
        const int lo_i = top - 4 * kSearchThreads;
        TB nv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int i = lo_i + threadIdx.x + kSearchThreads * j;
          if (i >= 0 && i < top) nv[j] = i >= h ? add_tree(buf[i], buf[i - h]) : buf[i];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int i = lo_i + threadIdx.x + kSearchThreads * j;
          if (i >= 0 && i < top) buf[i] = nv[j];
        }
        __syncthreads();
      }
    }
    for (int i = w - 1 + threadIdx.x; i < cnt; i += kSearchThreads) {
      const int t = t_lo + i;
      if (t >= 0 && t < nt && buf[i] == s_m[k]) {
        atomicMin(&s_t, t);
        break;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      peak[(int64_t)d * nk + k] = (TP)s_m[k];
      time[(int64_t)d * nk + k] = s_t == INT32_MAX ? 0 : s_t;
    }
  }
}

int halo_of(int nk) { return ((1 << (nk - 1)) - 1 + 15) / 16 * 16; }

// Columns each phase produces: what the later phases read (the rest of the
// widest window below the segment), or only the segment for the last phase.
SearchGeom geom_for(int nk, int seg) {
  SearchGeom g;
  g.seg = seg;
  g.halo = halo_of(nk);
  g.n = seg + g.halo;
  const int wmax = 1 << (nk - 1);
  auto lo_of = [&](int span, bool last) {
    const int lo = last ? g.halo : g.halo - wmax + span;
    return lo < 0 ? 0 : lo / 16 * 16;
  };
  g.lo1 = lo_of(16, nk <= 5);
  g.lo16 = lo_of(256, nk <= 9);
  g.lo256 = lo_of(4096, true);
  return g;
}

int passes(int n, int lo) { return (n - lo + kPass - 1) / kPass; }

size_t smem_of(const SearchGeom &g, int nk, size_t ta, size_t tb) {
  const size_t a = (size_t)(g.n + (int)(16 / ta) * (g.n >> 4)) * ta;
  const size_t b = (size_t)(g.n + (int)(16 / tb) * (g.n >> 4)) * tb;
  return 2 * a + (nk > 5 ? b : 0) + (nk > 9 ? b : 0);
}

constexpr size_t kSmemLimit = 200 * 1024;

// Segment length: the most output columns per phase pass that fit the
// shared-memory limit (ties: the shorter segment).  Depends only on
// (nk, nt, element sizes), so the workspace size can be computed up front.
SearchGeom choose_geom(int nk, int64_t nt, size_t ta, size_t tb) {
  SearchGeom best = geom_for(nk, 16);
  double best_rate = -1.0;
  const int64_t cap = nt < kMaxSeg ? (nt + 15) / 16 * 16 : kMaxSeg;
  for (int seg = 16; seg <= cap; seg += 16) {
    const SearchGeom g = geom_for(nk, seg);
    if (smem_of(g, nk, ta, tb) > kSmemLimit) break;
    int p = passes(g.n, g.lo1);
    if (nk > 5) p += passes(g.n, g.lo16);
    if (nk > 9) p += passes(g.n, g.lo256);
    const int64_t nseg = (nt + seg - 1) / seg;
    const double rate = (double)nt / (double)(nseg * p);
    if (rate > best_rate * (1.0 + 1e-9)) {
      best_rate = rate;
      best = g;
    }
  }
  return best;
}

template <class TA, class TB, class TP>
cudaError_t launch_search(const void *A, int32_t nd, int64_t nt, int32_t nk, void *peak, int32_t *time, void *ws,
                          cudaStream_t s) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const SearchGeom g = choose_geom(nk, nt, sizeof(TA), sizeof(TB));
  const size_t smem = smem_of(g, nk, sizeof(TA), sizeof(TB));
  void (*kern)(const TA *, int, int, SearchGeom, int, int, int, int, TB *, int *) = search_kernel<TA, TB, 1>;
  if constexpr (sizeof(TB) == 4) {
    if (nk <= 9) kern = search_kernel<TA, TB, 3>;
  }
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSearchThreads, smem)) != cudaSuccess)
    return e;
  const int nseg = (int)((nt + g.seg - 1) / g.seg);
  const int items = nd * nseg;
  const int grid0 = std::min(items, sms * std::max(per_sm, 1));
  const int per_block = (items + grid0 - 1) / grid0;
  const int grid = (items + per_block - 1) / per_block;
  TB *part_v = static_cast<TB *>(ws);
  int *part_r = reinterpret_cast<int *>(static_cast<char *>(ws) + (size_t)nd * nk * nseg * sizeof(int64_t));
  const int vec = (nt % 4 == 0) && (reinterpret_cast<uintptr_t>(A) % 16 == 0);
  kern<<<grid, kSearchThreads, smem, s>>>(static_cast<const TA *>(A), (int)nt, nk, g, nseg, items, per_block, vec,
                                          part_v, part_r);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // Widths up to 256 need one warp each (and its slice of shared memory);
  // wider ones the whole block and the widest region.
  const int fwarps = nk <= 9 ? std::min(nk, kWarps) : kWarps;
  const size_t fsmem = (nk <= 9 ? (size_t)fwarps * kFinalizeWarpElems : (size_t)kFinalizeElems) * sizeof(TB);
  auto fin = search_finalize_kernel<TA, TB, TP>;
  if ((e = cudaFuncSetAttribute(fin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem)) != cudaSuccess)
    return e;
  fin<<<nd, 32 * fwarps, fsmem, s>>>(static_cast<const TA *>(A), (int)nt, nk, nseg, part_v, part_r,
                                        static_cast<TP *>(peak), time);
  return cudaGetLastError();
}

template <class TA, class TB, class TP>
cudaError_t launch_finalize(const void *A, int32_t nd, int64_t nt, int32_t nk, int32_t nseg, const void *part_v,
                            const int *part_r, void *peak, int32_t *time, cudaStream_t s) {
  const int fwarps = nk <= 9 ? std::min(nk, kWarps) : kWarps;
  const size_t fsmem = (nk <= 9 ? (size_t)fwarps * kFinalizeWarpElems : (size_t)kFinalizeElems) * sizeof(TB);
  auto fin = search_finalize_kernel<TA, TB, TP>;
  cudaError_t e = cudaFuncSetAttribute(fin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem);
  if (e != cudaSuccess) return e;
  fin<<<nd, 32 * fwarps, fsmem, s>>>(static_cast<const TA *>(A), (int)nt, nk, nseg, static_cast<const TB *>(part_v),
                                        part_r, static_cast<TP *>(peak), time);
  return cudaGetLastError();
}

}  // namespace

cudaError_t search_finalize(int dtype, bool wide, const void *A, int32_t nd, int64_t nt, int32_t nk, int32_t nseg,
                            const void *part_v, const int *part_r, void *peak, int32_t *time, cudaStream_t s) {
  if (dtype != FDMT_U8_I32) return launch_finalize<float, float, float>(A, nd, nt, nk, nseg, part_v, part_r, peak, time, s);
  if (wide)
    return launch_finalize<int32_t, int64_t, int64_t>(A, nd, nt, nk, nseg, part_v, part_r, peak, time, s);
  return launch_finalize<int32_t, int32_t, int64_t>(A, nd, nt, nk, nseg, part_v, part_r, peak, time, s);
}

// Segments per row (the launch picks the same geometry from the same
// arguments).
int64_t search_segments(bool wide, int64_t nt, int32_t nk) {
  const SearchGeom g = choose_geom(nk, nt, 4, wide ? 8 : 4);
  return (nt + g.seg - 1) / g.seg;
}

}  // namespace fdmt

extern "C" {

int fdmt_search_workspace_bytes(int32_t nd, int64_t nt, int32_t n_widths, size_t *bytes) {
  if (bytes == nullptr || nd < 1 || nt < 1 || n_widths < 1 || n_widths > fdmt::kMaxWidths)
    return FDMT_ERR_INVALID_ARG;
  // Enough for either accumulator size.
  const int64_t nseg = std::max(fdmt::search_segments(false, nt, n_widths),
                                fdmt::search_segments(true, nt, n_widths));
  *bytes = (size_t)nd * (size_t)n_widths * (size_t)nseg * (sizeof(int64_t) + sizeof(int32_t));
  return FDMT_OK;
}

int fdmt_search(const void *A, int32_t dtype, int32_t nd, int64_t nt, int32_t n_widths, int64_t value_bound,
                void *peak, int32_t *time, void *workspace, size_t ws_bytes, void *stream) {
  size_t need = 0;
  if (fdmt_search_workspace_bytes(nd, nt, n_widths, &need) != FDMT_OK) return FDMT_ERR_INVALID_ARG;
  if (A == nullptr || peak == nullptr || time == nullptr || value_bound < 0) return FDMT_ERR_INVALID_ARG;
  if (dtype != FDMT_U8_I32 && dtype != FDMT_F32_F32 && dtype != FDMT_F32_F16STATE) return FDMT_ERR_INVALID_ARG;
  // Times (and region starts up to 2^14 outside [0, nt)) are int32.
  if (nt > INT32_MAX - (1 << 14)) return FDMT_ERR_UNSUPPORTED;
  if (workspace == nullptr || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 15u))
    return FDMT_ERR_WORKSPACE;
  if ((int64_t)nd * std::max(fdmt::search_segments(false, nt, n_widths), fdmt::search_segments(true, nt, n_widths)) >
      INT32_MAX)
    return FDMT_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (dtype != FDMT_U8_I32) {
    e = fdmt::launch_search<float, float, float>(A, nd, nt, n_widths, peak, time, workspace, s);
  } else if (value_bound > 0 && value_bound <= (int64_t)(INT32_MAX >> (n_widths - 1))) {
    // |window sum| <= 2^(K-1) * value_bound <= INT32_MAX: int32 is exact.
    e = fdmt::launch_search<int32_t, int32_t, int64_t>(A, nd, nt, n_widths, peak, time, workspace, s);
  } else {
    e = fdmt::launch_search<int32_t, int64_t, int64_t>(A, nd, nt, n_widths, peak, time, workspace, s);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FDMT_ERR_CUDA;
  }
  return FDMT_OK;
}

}  // extern "C"
