// Boxcar search of an FDMT output (contracts in include/fdmt.h).
//
// Section 4.2 ("Pulse profile") of Zackay & Ofek (arXiv:1411.5373): a
// uniform pulse profile convolved with the time axis commutes with the whole
// transform, so several widths are tested on one output.  For width
// w = 2^k and row d, B_w[d][t] = sum_{i<w} A[d][t - i] (zero before t = 0)
// is summed as a binary tree, B_1 = A and B_2w[t] = B_w[t] + B_w[t - w];
// the result per (row, width) is the maximum over t and the first t that
// reaches it.  Integer outputs are summed in int64 (exact at any width),
// float outputs in float32 with that tree order (bit-identical to a plain
// evaluation of the recursion).
//
// Schedule.  Work items are (row, segment of `seg` samples), row-major, so
// the blocks running at one time read neighbouring segments of a row and the
// history below each segment (`halo` >= 2^(K-1) - 1 samples) comes from L2.
// Persistent blocks take items in a fixed stride; each item's window (history
// + segment) is copied into shared memory with cp.async while the previous
// item is being searched (two window buffers).  The widths are built in
// phases of four doublings: a thread holds a run of 16 columns of B_S at
// stride S (S = 1, 16, 256) plus the 16 before them, doubles four times in
// registers (B_2S .. B_16S), keeps the running maximum of each width, and
// stores B_16S for the next phase, so shared memory sees two reads and one
// write per column per four widths.  The segment length is chosen so every
// phase needs few 4096-column passes.  A second kernel reduces the segments
// of each (row, width) in time order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/fdmt.h"

namespace fdmt {
namespace {

constexpr int kSearchThreads = 256;
constexpr int kPass = kSearchThreads * 16;  // columns one phase pass covers
constexpr int kMaxWidths = 13;
constexpr int kWarps = kSearchThreads / 32;
constexpr int kMaxSeg = 3 * kPass;

// Shared-memory layout of window column c: 16 bytes of padding after each
// run of 16 columns, so the 16-column runs of consecutive threads fall on
// different banks.
template <class T>
__host__ __device__ constexpr int pidx(int c) {
  return c + (int)(16 / sizeof(T)) * (c >> 4);
}

__device__ __forceinline__ float add_tree(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ int64_t add_tree(int64_t a, int64_t b) { return a + b; }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ int64_t vmax(int64_t a, int64_t b) { return a > b ? a : b; }

// (value, column) order: larger value first, then the earlier column; a
// negative column marks "no candidate".
template <class TB>
__device__ __forceinline__ bool better(TB v, int c, TB bv, int bc) {
  if (c < 0) return false;
  if (bc < 0) return true;
  return v > bv || (v == bv && c < bc);
}

template <class TB>
struct Best {
  TB v;
  int c;
};

// The first maximum of x[16..31] (columns col0 + S*i) joins the running best
// if it beats it; only columns in [lo, hi) count.  A thread meets its
// columns in increasing order, so a strict comparison keeps the first.
template <class TB, int S>
__device__ __forceinline__ void track(const TB (&x)[32], int col0, int lo, int hi, Best<TB> &b) {
  if (col0 >= lo && col0 + S * 15 < hi) {
    TB m = x[16];
#pragma unroll
    for (int i = 17; i < 32; ++i) m = vmax(m, x[i]);
    if (b.c < 0 || m > b.v) {
      int first = 15;
      TB fv = x[31];  // the stored value, so a zero keeps its own sign
#pragma unroll
      for (int i = 30; i >= 16; --i)
        if (x[i] == m) {
          first = i - 16;
          fv = x[i];
        }
      b.v = fv;
      b.c = col0 + S * first;
    }
  } else {
#pragma unroll
    for (int i = 16; i < 32; ++i) {
      const int c = col0 + S * (i - 16);
      if (c >= lo && c < hi && (b.c < 0 || x[i] > b.v)) {
        b.v = x[i];
        b.c = c;
      }
    }
  }
}

// Warp-reduce `nb` running bests and leave them in red[k][warp].
template <class TB, int NB>
__device__ __forceinline__ void warp_reduce(Best<TB> (&best)[NB], int k0, int nk, Best<TB> (*red)[kWarps]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    if (k0 + i >= nk) break;
    Best<TB> b = best[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const TB ov = __shfl_xor_sync(0xffffffffu, b.v, o);
      const int oc = __shfl_xor_sync(0xffffffffu, b.c, o);
      if (better(ov, oc, b.v, b.c)) {
        b.v = ov;
        b.c = oc;
      }
    }
    if (lane == 0) red[k0 + i][warp] = b;
  }
}

// One phase: B_S (src, element type TS, written at the columns >= src_lo)
// -> B_2S .. B_16S at the columns [lo, n) (the widest also to dst, if any).
// Width indices K0 .. K0+3 are tracked while below nk, and index 0 (B_1
// itself) when S == 1.
template <class TS, class TB, int S>
__device__ __forceinline__ void phase(const TS *src, TB *dst, int src_lo, int n, int lo, int halo, int lim,
                                      int nk, Best<TB> (*red)[kWarps]) {
  constexpr int G = 16 * S;                           // columns of one thread group
  constexpr int K0 = S == 1 ? 1 : (S == 16 ? 5 : 9);  // width index of 2S
  constexpr int NB = S == 1 ? 5 : 4;
  Best<TB> best[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) best[i] = {TB(0), -1};
  const int r = threadIdx.x % S, gi = threadIdx.x / S;
  for (int pass = lo; pass < n; pass += kPass) {
    const int base = pass + gi * G;
    if (base >= n) break;
    TB x[32];
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
      track<TB, 1>(x, base, halo, lim, best[0]);
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int c = base + r + S * (j - 16);
        x[j] = (c >= src_lo && c < n) ? (TB)src[pidx<TS>(c)] : TB(0);
      }
    }
#pragma unroll
    for (int m = 1; m <= 4; ++m) {
      if (dst == nullptr && K0 + m - 1 >= nk) break;
      const int h = 1 << (m - 1);
#pragma unroll
      for (int i = 31; i >= (1 << m); --i) x[i] = add_tree(x[i], x[i - h]);
      if (K0 + m - 1 < nk) track<TB, S>(x, base + r, halo, lim, best[NB - 4 + m - 1]);
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
#pragma unroll
        for (int j = 16; j < 32; ++j) {
          const int c = base + r + S * (j - 16);
          if (c < n) dst[pidx<TB>(c)] = x[j];
        }
      }
    }
  }
  warp_reduce<TB, NB>(best, S == 1 ? 0 : K0, nk, red);
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

// Copy window columns [0, n) of the item into buf (zeros outside [0, nt)):
// 16-byte asynchronous copies when rows are 16-byte aligned, else plain
// loads and stores.
template <class TA>
__device__ __forceinline__ void stage_window(TA *buf, const TA *row, int64_t t0, int64_t nt, int n, int vec) {
  for (int c = 4 * threadIdx.x; c < n; c += 4 * kSearchThreads) {
    const int64_t t = t0 + c;
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

template <class TA, class TB>
__global__ void __launch_bounds__(kSearchThreads)
search_kernel(const TA *__restrict__ A, int64_t nt, int nk, SearchGeom g, int nseg, int64_t items, int vec,
              TB *__restrict__ part_v, int32_t *__restrict__ part_t) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Best<TB> red[kMaxWidths][kWarps];
  const int n = g.n, halo = g.halo;
  const size_t a_bytes = (size_t)pidx<TA>(n) * sizeof(TA);
  const size_t b_bytes = (size_t)pidx<TB>(n) * sizeof(TB);
  TA *const abuf0 = reinterpret_cast<TA *>(smem);
  TA *const abuf1 = reinterpret_cast<TA *>(smem + a_bytes);
  TB *b16 = reinterpret_cast<TB *>(smem + 2 * a_bytes);
  TB *b256 = reinterpret_cast<TB *>(smem + 2 * a_bytes + b_bytes);
  int64_t item = blockIdx.x;
  if (item < items) {
    const int64_t d = item / nseg, s = item % nseg;
    stage_window(abuf0, A + d * nt, s * g.seg - halo, nt, n, vec);
  }
  for (int it = 0; item < items; ++it, item += gridDim.x) {
    const int64_t next = item + gridDim.x;
    if (next < items) {
      const int64_t d = next / nseg, s = next % nseg;
      stage_window((it & 1) ? abuf0 : abuf1, A + d * nt, s * g.seg - halo, nt, n, vec);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int64_t d = item / nseg, s = item % nseg;
    const int64_t t0 = s * g.seg - halo;
    const int lim = halo + (int)((nt - s * g.seg) < (int64_t)g.seg ? (nt - s * g.seg) : (int64_t)g.seg);
    phase<TA, TB, 1>((it & 1) ? abuf1 : abuf0, nk > 5 ? b16 : nullptr, 0, n, g.lo1, halo, lim, nk, red);
    if (nk > 5) {
      __syncthreads();
      phase<TB, TB, 16>(b16, nk > 9 ? b256 : nullptr, g.lo1, n, g.lo16, halo, lim, nk, red);
      if (nk > 9) {
        __syncthreads();
        phase<TB, TB, 256>(b256, nullptr, g.lo16, n, g.lo256, halo, lim, nk, red);
      }
    }
    __syncthreads();
    if (threadIdx.x < nk) {
      const int k = threadIdx.x;
      Best<TB> b = red[k][0];
      for (int w = 1; w < kWarps; ++w)
        if (better(red[k][w].v, red[k][w].c, b.v, b.c)) b = red[k][w];
      const int64_t slot = (d * nk + k) * nseg + s;
      part_v[slot] = b.v;
      part_t[slot] = (int32_t)(t0 + b.c);  // every segment holds >= 1 column
    }
    __syncthreads();  // the window buffer and red[] are refilled next
  }
}

// One thread per (row, width): the segments' maxima in time order.
template <class TB>
__global__ void search_reduce_kernel(const TB *__restrict__ part_v, const int32_t *__restrict__ part_t,
                                     int64_t pairs, int nseg, TB *__restrict__ peak, int32_t *__restrict__ time) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pairs) return;
  TB bv = part_v[i * nseg];
  int32_t bt = part_t[i * nseg];
  for (int s = 1; s < nseg; ++s) {
    const TB v = part_v[i * nseg + s];
    if (v > bv) {  // segments in time order: a tie keeps the earlier one
      bv = v;
      bt = part_t[i * nseg + s];
    }
  }
  peak[i] = bv;
  time[i] = bt;
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

// Segment length: the most output columns per phase pass that fit the
// shared-memory limit (ties: the shorter segment).
SearchGeom choose_geom(int nk, int64_t nt, size_t ta, size_t tb, size_t smem_limit) {
  SearchGeom best = geom_for(nk, 16);
  double best_rate = -1.0;
  const int64_t cap = nt < kMaxSeg ? (nt + 15) / 16 * 16 : kMaxSeg;
  for (int seg = 16; seg <= cap; seg += 16) {
    const SearchGeom g = geom_for(nk, seg);
    if (smem_of(g, nk, ta, tb) > smem_limit) break;
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

template <class TA, class TB>
cudaError_t launch_search(const void *A, int32_t nd, int64_t nt, int32_t nk, void *peak, int32_t *time, void *ws,
                          cudaStream_t s) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const SearchGeom g = choose_geom(nk, nt, sizeof(TA), sizeof(TB), 200 * 1024);
  const size_t smem = smem_of(g, nk, sizeof(TA), sizeof(TB));
  auto kern = search_kernel<TA, TB>;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSearchThreads, smem)) != cudaSuccess)
    return e;
  const int64_t nseg = (nt + g.seg - 1) / g.seg;
  const int64_t items = (int64_t)nd * nseg;
  const int64_t grid = std::min<int64_t>(items, (int64_t)sms * (per_sm > 0 ? per_sm : 1));
  const int64_t pairs = (int64_t)nd * nk;
  TB *part_v = static_cast<TB *>(ws);
  int32_t *part_t = reinterpret_cast<int32_t *>(static_cast<char *>(ws) + pairs * nseg * sizeof(int64_t));
  const int vec = (nt % 4 == 0) && (reinterpret_cast<uintptr_t>(A) % 16 == 0);
  kern<<<(unsigned)grid, kSearchThreads, smem, s>>>(static_cast<const TA *>(A), nt, nk, g, (int)nseg, items, vec,
                                                     part_v, part_t);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  search_reduce_kernel<TB><<<(unsigned)((pairs + 255) / 256), 256, 0, s>>>(part_v, part_t, pairs, (int)nseg,
                                                                           static_cast<TB *>(peak), time);
  return cudaGetLastError();
}

}  // namespace

// Segments per row for the workspace size (the launch picks the same
// geometry from the same arguments).
int64_t search_segments(int32_t dtype, int64_t nt, int32_t nk) {
  const size_t tb = dtype == FDMT_U8_I32 ? sizeof(int64_t) : sizeof(float);
  const SearchGeom g = choose_geom(nk, nt, 4, tb, 200 * 1024);
  return (nt + g.seg - 1) / g.seg;
}

}  // namespace fdmt

extern "C" {

int fdmt_search_workspace_bytes(int32_t nd, int64_t nt, int32_t n_widths, size_t *bytes) {
  if (bytes == nullptr || nd < 1 || nt < 1 || n_widths < 1 || n_widths > fdmt::kMaxWidths)
    return FDMT_ERR_INVALID_ARG;
  // Enough for either dtype: the float geometry never has fewer segments.
  const int64_t nseg = std::max(fdmt::search_segments(FDMT_F32_F32, nt, n_widths),
                                fdmt::search_segments(FDMT_U8_I32, nt, n_widths));
  *bytes = (size_t)nd * (size_t)n_widths * (size_t)nseg * (sizeof(int64_t) + sizeof(int32_t));
  return FDMT_OK;
}

int fdmt_search(const void *A, int32_t dtype, int32_t nd, int64_t nt, int32_t n_widths, void *peak,
                int32_t *time, void *workspace, size_t ws_bytes, void *stream) {
  size_t need = 0;
  if (fdmt_search_workspace_bytes(nd, nt, n_widths, &need) != FDMT_OK) return FDMT_ERR_INVALID_ARG;
  if (A == nullptr || peak == nullptr || time == nullptr) return FDMT_ERR_INVALID_ARG;
  if (dtype != FDMT_U8_I32 && dtype != FDMT_F32_F32 && dtype != FDMT_F32_F16STATE) return FDMT_ERR_INVALID_ARG;
  if (nt > INT32_MAX) return FDMT_ERR_UNSUPPORTED;  // peak times are int32
  if (workspace == nullptr || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 15u))
    return FDMT_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cudaError_t e =
      dtype == FDMT_U8_I32
          ? fdmt::launch_search<int32_t, int64_t>(A, nd, nt, n_widths, peak, time, workspace, s)
          : fdmt::launch_search<float, float>(A, nd, nt, n_widths, peak, time, workspace, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FDMT_ERR_CUDA;
  }
  return FDMT_OK;
}

}  // extern "C"
