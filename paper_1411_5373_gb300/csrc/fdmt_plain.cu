// Plain schedule of the FDMT: one launch for the initialisation, then one
// launch per merge level (section 4, Algorithm 1 of arXiv:1411.5373), plus
// the transposed (adjoint) levels.  Every kernel streams whole time rows:
// 4 consecutive samples per thread, 16-byte vector loads and stores, the
// shifted operand assembled from two aligned vector loads.
#include <cuda_runtime.h>

#include <type_traits>

#include "fdmt_common.cuh"
#include "fdmt_internal.h"

namespace fdmt {

constexpr int kThreads = 256;
constexpr int kTile = kThreads * 4;  // samples per block per pass

static inline dim3 row_grid(int64_t rows, int64_t nt) {
  int64_t tiles = (nt + kTile - 1) / kTile;
  if (tiles > 65535) tiles = 65535;
  return dim3((unsigned)rows, (unsigned)tiles, 1);
}

// ---------------------------------------------------------------------------
// Initialisation, Option 1 of section 4: for channel k and j = 0 .. sweep_k,
//   state[row0_k + j][t] = sum_{i=0..j} x[k][t - i]   (x = w[k] * I, zero for t < 0)
// accumulated as row j = row j-1 + x[t - j].  One block per (channel, tile);
// the tile plus a halo of `sweep` samples is staged in shared memory.
template <class TIn, class TS, class A>
__global__ void __launch_bounds__(kThreads)
init_kernel(const TIn *__restrict__ in, const float *__restrict__ w, TS *__restrict__ state,
            const InitOp *__restrict__ init, int64_t nt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  A *xs = reinterpret_cast<A *>(smem_raw);
  const int k = blockIdx.x;
  const InitOp op = init[k];
  const int sweep = op.sweep;
  const TIn *src = in + (int64_t)k * nt;
  for (int64_t tile = (int64_t)blockIdx.y * kTile; tile < nt; tile += (int64_t)gridDim.y * kTile) {
    const int n = sweep + kTile;
    for (int i = threadIdx.x; i < n; i += kThreads) {
      const int64_t t = tile - sweep + i;
      A v = A(0);
      if (t >= 0 && t < nt) {
        v = acc_of(src[t]);
        if constexpr (std::is_floating_point<A>::value) {
          if (w != nullptr) v = __fmul_rn(v, w[k]);
        }
      }
      xs[i] = v;
    }
    __syncthreads();
    const int64_t t0 = tile + 4 * threadIdx.x;
    if (t0 < nt) {
      const int c0 = sweep + 4 * threadIdx.x;
      A run[4] = {xs[c0], xs[c0 + 1], xs[c0 + 2], xs[c0 + 3]};
      TS *dst = state + (int64_t)op.row0 * nt + t0;
      store4(dst, run);
      for (int j = 1; j <= sweep; ++j) {
#pragma unroll
        for (int c = 0; c < 4; ++c) run[c] = acc_add(run[c], xs[c0 + c - j]);
        store4(dst + (int64_t)j * nt, run);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// One merge level: next[r][t] = prev[lo][t] + prev[hi][t - shift], the second
// term zero for t < shift (the copy rule).  Block (r, tile).
template <class TS, class TO, class A>
__global__ void __launch_bounds__(kThreads)
merge_kernel(const TS *__restrict__ prev, TO *__restrict__ next, const RowOp *__restrict__ ops,
             int64_t nt) {
  const int r = blockIdx.x;
  const RowOp op = ops[r];
  const TS *lo = prev + (int64_t)op.lo * nt;
  TO *dst = next + (int64_t)r * nt;
  if (op.hi < 0) {  // a band with no upper sub-band: the row passes up unchanged
    for (int64_t t0 = ((int64_t)blockIdx.y * kThreads + threadIdx.x) * 4; t0 < nt;
         t0 += (int64_t)gridDim.y * kTile) {
      A a[4];
      load4(lo + t0, a);
      store4(dst + t0, a);
    }
    return;
  }
  const TS *hi = prev + (int64_t)op.hi * nt;
  for (int64_t t0 = ((int64_t)blockIdx.y * kThreads + threadIdx.x) * 4; t0 < nt;
       t0 += (int64_t)gridDim.y * kTile) {
    A a[4], b[4], o[4];
    load4(lo + t0, a);
    load4_shifted(hi, t0 - op.shift, nt, b);
#pragma unroll
    for (int c = 0; c < 4; ++c) o[c] = acc_add(a[c], b[c]);
    store4(dst + t0, o);
  }
}

// ---------------------------------------------------------------------------
// Transposed merge level (gather form, no atomics):
//   child[c][u] = sum_{i < count} parent[first + i][u + shift0 + i*step], zero past nt.
// I is the column index type: 32-bit columns keep the kernel at 32
// registers (8 blocks of 256 threads per SM), used whenever nt allows.
template <class I>
__device__ __forceinline__ void adj_load4(const float *row, I u, I nt, float (&v)[4]) {
  const I base = u & ~(I)3;  // floor to a multiple of 4 (two's complement)
  const int rem = (int)(u & (I)3);
  float a[4], b[4];
  if (base >= 0 && base < nt) load4(row + base, a); else zero4(a);
  if (rem == 0) {
    v[0] = a[0]; v[1] = a[1]; v[2] = a[2]; v[3] = a[3];
    return;
  }
  if (base + 4 >= 0 && base + 4 < nt) load4(row + base + 4, b); else zero4(b);
  switch (rem) {
    case 1: v[0] = a[1]; v[1] = a[2]; v[2] = a[3]; v[3] = b[0]; break;
    case 2: v[0] = a[2]; v[1] = a[3]; v[2] = b[0]; v[3] = b[1]; break;
    default: v[0] = a[3]; v[1] = b[0]; v[2] = b[1]; v[3] = b[2]; break;
  }
}

template <class I>
__global__ void __launch_bounds__(kThreads, 8)
adj_merge_kernel(const float *__restrict__ parent, float *__restrict__ child,
                 const AdjOp *__restrict__ ops, I nt) {
  const int c = blockIdx.x;
  const AdjOp op = ops[c];
  float *dst = child + (int64_t)c * nt;
  for (I u0 = ((I)blockIdx.y * kThreads + threadIdx.x) * 4; u0 < nt; u0 += (I)gridDim.y * kTile) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int i = 0; i < op.count; ++i) {
      float v[4];
      adj_load4<I>(parent + (int64_t)(op.first + i) * nt, u0 + (I)op.shift0 + (I)i * op.step, nt, v);
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = __fadd_rn(acc[q], v[q]);
    }
    store4(dst + u0, acc);
  }
}

// Two transposed levels at once (levels l and l - 1 into l - 2):
//   child[c][u] = sum_{k < count} parent[row_k][u + shift_k]
// over the composed terms of child c; the intermediate level never reaches
// memory.
template <class I>
__global__ void __launch_bounds__(kThreads, 8)
adj_merge2_kernel(const float *__restrict__ parent, float *__restrict__ child, const AdjRun *__restrict__ runs,
                  const AdjTerm *__restrict__ terms, I nt) {
  const int c = blockIdx.x;
  const AdjRun run = runs[c];
  float *dst = child + (int64_t)c * nt;
  for (I u0 = ((I)blockIdx.y * kThreads + threadIdx.x) * 4; u0 < nt; u0 += (I)gridDim.y * kTile) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < run.count; ++k) {
      const AdjTerm tm = terms[run.first + k];
      float v[4];
      adj_load4<I>(parent + (int64_t)tm.row * nt, u0 + (I)tm.shift, nt, v);
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = __fadd_rn(acc[q], v[q]);
    }
    store4(dst + u0, acc);
  }
}

// Transposed initialisation: g[k][s] = sum_{j=0..sweep} sum_{i=0..j} g0[row0+j][s+i],
// written to gi; scaled by w[k] here only when no weight gradient is wanted
// (otherwise weights_epilogue_kernel needs the unscaled g and scales it).
template <class I>
__global__ void __launch_bounds__(kThreads, 8)
adj_init_kernel(const float *__restrict__ g0, const float *__restrict__ w, float *__restrict__ gi,
                const InitOp *__restrict__ init, I nt) {
  const int k = blockIdx.x;
  const InitOp op = init[k];
  for (I s0 = ((I)blockIdx.y * kThreads + threadIdx.x) * 4; s0 < nt; s0 += (I)gridDim.y * kTile) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int j = 0; j <= op.sweep; ++j) {
      const float *row = g0 + (int64_t)(op.row0 + j) * nt;
      for (int i = 0; i <= j; ++i) {
        float v[4];
        adj_load4<I>(row, s0 + (I)i, nt, v);
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = __fadd_rn(acc[q], v[q]);
      }
    }
    if (w != nullptr) {
      const float wk = w[k];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = __fmul_rn(acc[q], wk);
    }
    store4(gi + (int64_t)k * nt + s0, acc);
  }
}

// Weight gradient and scaling, one block per channel:
//   gw[k] = sum_s x[k][s] * g[k][s]  (fixed-order block reduction), then g[k] *= w[k].
constexpr int kReduceThreads = 512;
__global__ void __launch_bounds__(kReduceThreads)
weights_epilogue_kernel(const float *__restrict__ x, const float *__restrict__ w,
                        float *__restrict__ g, float *__restrict__ gw, int64_t nt) {
  __shared__ float part[kReduceThreads / 32];
  const int k = blockIdx.x;
  const float *xr = x + (int64_t)k * nt;
  float *gr = g + (int64_t)k * nt;
  const float wk = w ? w[k] : 1.0f;
  float acc = 0.f;
  for (int64_t s0 = (int64_t)threadIdx.x * 4; s0 < nt; s0 += kReduceThreads * 4) {
    float a[4], b[4];
    load4(xr + s0, a);
    load4(gr + s0, b);
#pragma unroll
    for (int q = 0; q < 4; ++q) acc = __fadd_rn(acc, __fmul_rn(a[q], b[q]));
    if (w != nullptr) {
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = __fmul_rn(b[q], wk);
      store4(gr + s0, b);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < kReduceThreads / 32 ? part[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) gw[k] = v;
  }
}

// ---------------------------------------------------------------------------
// Launchers.

template <class TIn, class TS, class A>
static cudaError_t launch_init(const DeviceTables &dt, const void *in, const float *w, void *state,
                               int64_t nt, cudaStream_t s) {
  const size_t smem = sizeof(A) * (size_t)(dt.max_sweep + kTile);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(init_kernel<TIn, TS, A>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dt.prof->begin(s, K_INIT, 0);
  init_kernel<TIn, TS, A><<<row_grid(dt.nf, nt), kThreads, smem, s>>>(
      static_cast<const TIn *>(in), w, static_cast<TS *>(state), dt.init, nt);
  dt.prof->end(s);
  return cudaGetLastError();
}

template <class TS, class TO, class A>
static cudaError_t launch_merge(const DeviceTables &dt, int level, const void *prev, void *next,
                                int64_t nt, cudaStream_t s) {
  const int64_t rows = dt.level_rows[level];
  dt.prof->begin(s, K_MERGE, level);
  merge_kernel<TS, TO, A><<<row_grid(rows, nt), kThreads, 0, s>>>(
      static_cast<const TS *>(prev), static_cast<TO *>(next), dt.ops + dt.ops_begin[level], nt);
  dt.prof->end(s);
  return cudaGetLastError();
}

template <class TIn, class TS, class TO, class A>
static cudaError_t run_plain_typed(const DeviceTables &dt, const void *in, const float *w,
                                   void *out, void *const bufs[2], int64_t nt, cudaStream_t s) {
  cudaError_t e = launch_init<TIn, TS, A>(dt, in, w, bufs[0], nt, s);
  if (e != cudaSuccess) return e;
  for (int l = 1; l <= dt.levels; ++l) {
    const void *prev = bufs[(l - 1) & 1];
    if (l == dt.levels)
      e = launch_merge<TS, TO, A>(dt, l, prev, out, nt, s);
    else
      e = launch_merge<TS, TS, A>(dt, l, prev, bufs[l & 1], nt, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t run_plain(const DeviceTables &dt, int dtype, const void *in, const float *w, void *out,
                      void *const bufs[2], int64_t nt, cudaStream_t s) {
  switch (dtype) {
    case 0: return run_plain_typed<uint8_t, int32_t, int32_t, int32_t>(dt, in, nullptr, out, bufs, nt, s);
    case 1: return run_plain_typed<float, float, float, float>(dt, in, w, out, bufs, nt, s);
    case 2: return run_plain_typed<float, __half, float, float>(dt, in, w, out, bufs, nt, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t run_adjoint_plain(const DeviceTables &dt, const float *grad_out, const float *in,
                              const float *w, float *grad_in, float *grad_w, void *const bufs[2],
                              int64_t nt, cudaStream_t s) {
  // Level L's gradient is grad_out; two levels per step are gathered from
  // it downwards (one for a last odd level); step k writes buffer k % 2.
  const float *parent = grad_out;
  const bool narrow = nt < ((int64_t)1 << 31) - kTile;
  int k = 0;
  for (int l = dt.levels; l >= 1; ++k) {
    float *child = static_cast<float *>(bufs[k & 1]);
    cudaError_t e;
    if (l >= 2) {
      const int64_t rows = dt.level_rows[l - 2];
      const AdjRun *runs = dt.adj2 + dt.adj2_begin[l - 2];
      dt.prof->begin(s, K_ADJ_MERGE2, l);
      if (narrow)
        adj_merge2_kernel<int32_t><<<row_grid(rows, nt), kThreads, 0, s>>>(parent, child, runs, dt.adj2_terms,
                                                                            (int32_t)nt);
      else
        adj_merge2_kernel<int64_t><<<row_grid(rows, nt), kThreads, 0, s>>>(parent, child, runs, dt.adj2_terms, nt);
      l -= 2;
    } else {
      const int64_t rows = dt.level_rows[l - 1];
      dt.prof->begin(s, K_ADJ_MERGE, l);
      if (narrow)
        adj_merge_kernel<int32_t><<<row_grid(rows, nt), kThreads, 0, s>>>(parent, child,
                                                                           dt.adj + dt.adj_begin[l - 1], (int32_t)nt);
      else
        adj_merge_kernel<int64_t><<<row_grid(rows, nt), kThreads, 0, s>>>(parent, child,
                                                                           dt.adj + dt.adj_begin[l - 1], nt);
      l -= 1;
    }
    dt.prof->end(s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    parent = child;
  }
  dt.prof->begin(s, K_ADJ_INIT, 0);
  if (nt < ((int64_t)1 << 31) - kTile)
    adj_init_kernel<int32_t><<<row_grid(dt.nf, nt), kThreads, 0, s>>>(parent, grad_w ? nullptr : w, grad_in,
                                                                      dt.init, (int32_t)nt);
  else
    adj_init_kernel<int64_t><<<row_grid(dt.nf, nt), kThreads, 0, s>>>(parent, grad_w ? nullptr : w, grad_in,
                                                                      dt.init, nt);
  dt.prof->end(s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || grad_w == nullptr) return e;
  return run_weights_epilogue(dt, in, w, grad_in, grad_w, nt, s);
}

cudaError_t run_weights_epilogue(const DeviceTables &dt, const float *in, const float *w, float *grad_in,
                                 float *grad_w, int64_t nt, cudaStream_t s) {
  dt.prof->begin(s, K_WEIGHTS, 0);
  weights_epilogue_kernel<<<dt.nf, kReduceThreads, 0, s>>>(in, w, grad_in, grad_w, nt);
  dt.prof->end(s);
  return cudaGetLastError();
}

}  // namespace fdmt
