// FFT-FDMT (contracts in include/fdmt.h).
//
// Section 5, Algorithm 2 of Zackay & Ofek (arXiv:1411.5373): Fourier
// transform the time axis, so that every shifted row addition of Algorithm 1
// becomes a product with a shift vector exp(-2 pi i k s / N) and all
// additions stay within one Fourier bin k; then transform back.
//
// Three launches per transform:
//
//  1. forward: every input row is cut into overlapping blocks of N = 2^LN
//     samples, block j covering samples [j S - G, j S - G + N) with
//     G = Nd - 1 and hop S = N - G (zeros outside [0, Nt)).  Two consecutive
//     blocks ride in one complex sequence, block 2p in the real part and
//     block 2p+1 in the imaginary part (the machine-word paragraph's
//     packing: the transform is real-linear, so the two come back apart),
//     and each sequence gets an in-block Stockham FFT.  Output
//     X[c][p N + k], one row per channel.
//  2. merge: one CTA owns B consecutive bins (of one block pair) and runs all
//     levels of Algorithm 1 on them in shared memory.  The level-0 rows
//     (Option-1 partial sums) never exist: row j of channel c is
//     X_c(k) sum_{i <= j} w^{ik}, w = exp(-2 pi i k / N), formed where level
//     1 reads it; each later row is lo + hi w^{dl} with the integer tables of
//     the direct transform.  The top level is written over X in place
//     (Y[d][p N + k]): a CTA reads its own bins' X rows at level 1 only and
//     no other CTA touches them.
//  3. inverse: each output row's sequences are inverse transformed
//     (conj(FFT(conj Y)) / N); the cyclic wrap reaches only the first G
//     samples of a block, so samples [G, N) of block j are output columns
//     [j S, j S + S).
//
// Shifts are cyclic within a block (the zero-padding paragraph); the
// overlap of G samples plays the padding's part, block by block, so the
// Fourier length stays in shared memory instead of spanning the whole time
// axis.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <new>
#include <string>
#include <vector>

#include "../../include/fdmt.h"
#include "fdmt_internal.h"
#include "fdmt_stockham.cuh"
#include "fdmt_tables.h"

namespace fdmt {
namespace {

constexpr int kFftThreads = 256;
constexpr int kFftSamples = 4096;  // complex samples per FFT block
// Merge blocks: 512 threads (two blocks per SM) for 4 or 8 bins, 256
// threads (four per SM) for 1 or 2 bins.
template <int B>
__host__ __device__ constexpr int merge_threads() { return B >= 4 ? 512 : 256; }
constexpr int kMinLn = 8, kMaxLn = 12;
constexpr size_t kSmemLimit = 200 * 1024;
constexpr size_t kSmemTwoPerSm = 112 * 1024;  // two merge blocks per SM (228 KB, 1 KB reserved each)
constexpr size_t kSmemFourPerSm = 56 * 1024;  // four merge blocks per SM
constexpr int kMaxLevels = 31;

struct MergeArgs {
  const float2 *X;   // [Nf][ld] forward transforms (aliases Y)
  float2 *Y;         // [Nd][ld] top level, written over X
  int64_t ld;
  const float2 *tw;  // exp(-2 pi i m / N), m < N
  uint32_t mask;     // N - 1
  const int4 *ops1;  // level 1: (channel lo, partial sum lo, channel hi or -1, partial sum hi)
  const uint2 *ops;  // levels >= 2: (lo | hi << 16 (hi 0xffff: none), shift)
  int32_t nf, levels, max_w, max_shift, cap_odd, cap_even;
  int64_t ob[kMaxLevels + 2];  // first entry of level l in ops (l >= 2)
  int32_t rows[kMaxLevels + 2];
};

constexpr uint32_t kNoUpper = 0xffffu;
constexpr int kPrefetch = 6;  // row ops per thread fetched a level ahead
__device__ __forceinline__ float2 cmad(float2 a, float2 b, float2 c) {  // a b + c
  return make_float2(__fmaf_rn(a.x, b.x, __fmaf_rn(-a.y, b.y, c.x)), __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, c.y)));
}

// The B bins of one row (B consecutive float2), moved 16 bytes at a time.
template <int B>
struct Bins {
  float2 v[B];
  // A row of four bins takes two 16-byte accesses; odd groups of four lanes
  // take the second half first, so that one warp instruction over
  // consecutive rows covers all 32 banks (4 wavefronts, not 8).
  __device__ __forceinline__ static bool swap() { return B == 4 && ((threadIdx.x >> 2) & 1); }
  __device__ __forceinline__ void load(const float2 *p) {
    if constexpr (B == 1) {
      v[0] = *p;
    } else if constexpr (B == 4) {
      const bool sw = swap();
      const float4 *q = reinterpret_cast<const float4 *>(p);
      const float4 t0 = q[sw ? 1 : 0], t1 = q[sw ? 0 : 1];
      const float4 a = sw ? t1 : t0, b = sw ? t0 : t1;
      v[0] = make_float2(a.x, a.y);
      v[1] = make_float2(a.z, a.w);
      v[2] = make_float2(b.x, b.y);
      v[3] = make_float2(b.z, b.w);
    } else {
#pragma unroll
      for (int h = 0; h < B / 2; ++h) {
        const float4 t = reinterpret_cast<const float4 *>(p)[h];
        v[2 * h] = make_float2(t.x, t.y);
        v[2 * h + 1] = make_float2(t.z, t.w);
      }
    }
  }
  __device__ __forceinline__ void store(float2 *p) const {
    if constexpr (B == 1) {
      *p = v[0];
    } else if constexpr (B == 4) {
      const bool sw = swap();
      float4 *q = reinterpret_cast<float4 *>(p);
      const float4 a = make_float4(v[0].x, v[0].y, v[1].x, v[1].y), b = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
      q[sw ? 1 : 0] = sw ? b : a;
      q[sw ? 0 : 1] = sw ? a : b;
    } else {
#pragma unroll
      for (int h = 0; h < B / 2; ++h)
        reinterpret_cast<float4 *>(p)[h] = make_float4(v[2 * h].x, v[2 * h].y, v[2 * h + 1].x, v[2 * h + 1].y);
    }
  }
};

// Asynchronous global -> shared copies of one row of B bins (8 B per bin).
template <int B>
__device__ __forceinline__ void cp_async_row(float2 *dst, const float2 *src, int h) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst + 2 * h);
  if constexpr (B == 1)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src + 2 * h) : "memory");
}

// Shared memory of a merge block, in rows of B bins: geometric sums
// [max_w], shift vectors [max_shift + 1], odd levels [cap_odd], even levels
// [cap_even] (during level 1 the even buffer holds the block's input tile,
// Nf rows, so cap_even >= Nf).  One thread computes one row op for all B
// bins.
template <int B>
__global__ void __launch_bounds__(merge_threads<B>(), B >= 4 ? 2 : 4) fft_merge_kernel(const MergeArgs a) {
  constexpr int LB = fft::ilog2(B);
  constexpr int kMergeThreads = merge_threads<B>();
  extern __shared__ __align__(16) float2 sm[];
  float2 *G = sm;                             // [max_w][B]: sum_{i <= j} w^{ik}
  float2 *W = G + a.max_w * B;                // [max_shift + 1][B]: w^{sk}
  float2 *b_odd = W + (a.max_shift + 1) * B;  // [cap_odd][B]
  float2 *b_even = b_odd + a.cap_odd * B;     // [cap_even][B]
  const int64_t g0 = (int64_t)blockIdx.x * B;
  // The block's input tile X[c][g0 .. g0 + B) of every channel, copied
  // asynchronously (all rows in flight at once) while the shift vectors
  // are filled.
  {
    constexpr int CPR = B == 1 ? 1 : B / 2;  // copies per row
    for (int i = threadIdx.x; i < a.nf * CPR; i += kMergeThreads) {
      const int c = i / CPR, h = i - c * CPR;
      cp_async_row<B>(b_even + c * B, a.X + c * a.ld + g0, h);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  for (int i = threadIdx.x; i < (a.max_shift + 1) << LB; i += kMergeThreads) {
    const uint32_t k = (uint32_t)(g0 + (i & (B - 1))) & a.mask;
    W[i] = a.tw[((uint32_t)(i >> LB) * k) & a.mask];
  }
  if (threadIdx.x < B) {
    // Option-1 row j of channel c is X_c(k) G[j] (Algorithm 2, steps 1 and 3 in one).
    const uint32_t k = (uint32_t)(g0 + threadIdx.x) & a.mask;
    float2 s = make_float2(0.0f, 0.0f);
    for (int j = 0; j < a.max_w; ++j) {
      s = fft::cadd(s, a.tw[((uint32_t)j * k) & a.mask]);
      G[j * B + threadIdx.x] = s;
    }
  }
  // Row ops of the next level, fetched one level ahead (their latency
  // overlaps the current level's work and barrier).
  uint2 pf[kPrefetch];
  auto fetch = [&](int l) {
    const uint2 *ops = a.ops + a.ob[l];
#pragma unroll
    for (int u = 0; u < kPrefetch; ++u) {
      const int q = threadIdx.x + u * kMergeThreads;
      pf[u] = q < a.rows[l] ? ops[q] : make_uint2(0u, 0u);
    }
  };
  if (a.levels >= 2) fetch(2);
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  // Level 1 from the transformed input: lo + hi w^{dl}, dl = the lower row.
  for (int q = threadIdx.x; q < a.rows[1]; q += kMergeThreads) {
    const int4 op1 = a.ops1[q];
    Bins<B> x1, xh1;
    x1.load(b_even + (op1.x << LB));
    if (op1.z >= 0) xh1.load(b_even + (op1.z << LB));
    Bins<B> g, v;
    g.load(G + (op1.y << LB));
#pragma unroll
    for (int j = 0; j < B; ++j) v.v[j] = fft::cmul(x1.v[j], g.v[j]);
    if (op1.z >= 0) {
      Bins<B> gh, w;
      gh.load(G + (op1.w << LB));
      w.load(W + (op1.y << LB));
#pragma unroll
      for (int j = 0; j < B; ++j) v.v[j] = cmad(fft::cmul(xh1.v[j], gh.v[j]), w.v[j], v.v[j]);
    }
    v.store(b_odd + (q << LB));
  }
  __syncthreads();
  for (int l = 2; l <= a.levels; ++l) {
    const float2 *src = (l & 1) ? b_even : b_odd;
    float2 *dst = (l & 1) ? b_odd : b_even;
    const bool to_global = l == a.levels;
    uint2 cur[kPrefetch];
#pragma unroll
    for (int u = 0; u < kPrefetch; ++u) cur[u] = pf[u];
    if (l < a.levels) fetch(l + 1);
    const uint2 *ops = a.ops + a.ob[l];
#pragma unroll
    for (int u = 0; u < kPrefetch + 1; ++u) {
      for (int q = threadIdx.x + u * kMergeThreads; q < a.rows[l]; q += (u < kPrefetch ? a.rows[l] : kMergeThreads)) {
        const uint2 op = u < kPrefetch ? cur[u < kPrefetch ? u : 0] : ops[q];
        const uint32_t lo = op.x & 0xffffu, hi = op.x >> 16;
        Bins<B> v;
        v.load(src + (lo << LB));
        if (hi != kNoUpper) {
          Bins<B> h, w;
          h.load(src + (hi << LB));
          w.load(W + (op.y << LB));
#pragma unroll
          for (int j = 0; j < B; ++j) v.v[j] = cmad(h.v[j], w.v[j], v.v[j]);
        }
        if (to_global)
          v.store(a.Y + (int64_t)q * a.ld + g0);
        else
          v.store(dst + (q << LB));
      }
    }
    __syncthreads();
  }
  if (a.levels == 1) {  // Nf = 2: level 1 went to shared memory (X is read there)
    for (int i = threadIdx.x; i < (a.rows[1] << LB); i += kMergeThreads)
      a.Y[(int64_t)(i >> LB) * a.ld + g0 + (i & (B - 1))] = b_odd[i];
  }
}

// Last-pass destination of the forward transforms: the transforms of a
// block, back to back in global memory.
struct GlobalDst {
  float2 *__restrict__ x;
  __device__ __forceinline__ void operator()(int i, float2 v) const { x[i] = v; }
};

// First-pass source of the forward transforms: transform f of the block
// holds block pairs p0 + f of one input row; element n is
// in[t] + i in[t + S], t = 2 (p0 + f) S - G + n, zero outside [0, Nt).
template <typename TIn, int LN>
struct PairSrc {
  const TIn *__restrict__ row;
  int64_t nt, hop, first;  // first = 2 p0 S - G
  __device__ __forceinline__ float2 operator()(int i) const {
    const int f = i >> LN, n = i & ((1 << LN) - 1);
    const int64_t ta = first + 2 * hop * f + n, tb = ta + hop;
    const float re = (ta >= 0 && ta < nt) ? (float)row[ta] : 0.0f;
    const float im = (tb >= 0 && tb < nt) ? (float)row[tb] : 0.0f;
    return make_float2(re, im);
  }
};

template <int LN, typename TIn>
__global__ void __launch_bounds__(kFftThreads)
fft_forward_kernel(const TIn *__restrict__ in, int64_t nt, int64_t hop, int32_t guard, int64_t npair, int F,
                   float2 *__restrict__ X, int64_t ld) {
  constexpr int NF = 1 << LN;
  extern __shared__ __align__(16) float2 sm[];
  const int padded = fft::pad16(F * NF);
  float2 *buf0 = sm, *buf1 = sm + padded, *tw = buf1 + padded;
  const int64_t c = blockIdx.y;
  const int64_t p0 = (int64_t)blockIdx.x * F;
  const int Fh = (int)((npair - p0) < (int64_t)F ? (npair - p0) : (int64_t)F);
  fft::twiddles<kFftThreads, LN>(tw);
  __syncthreads();
  const PairSrc<TIn, LN> src{in + c * nt, nt, hop, 2 * p0 * hop - guard};
  fft::transform_to<kFftThreads, LN>(src, GlobalDst{X + c * ld + p0 * NF}, buf0, buf1, tw, Fh);
}

// Last-pass destination of the inverse transforms: element n of transform
// f is y = conj(v) / N of block pair p0 + f; samples n >= G are output
// columns 2 (p0 + f) S + n - G (real part) and that + S (imaginary part).
template <int LN>
struct PairSink {
  float *__restrict__ row;
  int64_t nt, hop, first;  // first = 2 p0 S - G
  int32_t guard;
  __device__ __forceinline__ void operator()(int i, float2 v) const {
    const int f = i >> LN, n = i & ((1 << LN) - 1);
    if (n < guard) return;
    constexpr float scale = 1.0f / (float)(1 << LN);
    const int64_t ta = first + 2 * hop * f + n, tb = ta + hop;
    if (ta < nt) row[ta] = v.x * scale;
    if (tb < nt) row[tb] = -v.y * scale;
  }
};

struct ConjSrc {
  const float2 *x;
  __device__ __forceinline__ float2 operator()(int i) const {
    const float2 v = x[i];
    return make_float2(v.x, -v.y);
  }
};

template <int LN>
__global__ void __launch_bounds__(kFftThreads)
fft_inverse_kernel(const float2 *__restrict__ Y, int64_t ld, int64_t nt, int64_t hop, int32_t guard, int64_t npair,
                   int F, float *__restrict__ out) {
  constexpr int NF = 1 << LN;
  extern __shared__ __align__(16) float2 sm[];
  const int padded = fft::pad16(F * NF);
  float2 *buf0 = sm, *buf1 = sm + padded, *tw = buf1 + padded;
  const int64_t d = blockIdx.y;
  const int64_t p0 = (int64_t)blockIdx.x * F;
  const int Fh = (int)((npair - p0) < (int64_t)F ? (npair - p0) : (int64_t)F);
  fft::twiddles<kFftThreads, LN>(tw);
  __syncthreads();
  // y = conj(FFT(conj Y)) / N: real part -> block 2p, -imag -> block 2p+1.
  const PairSink<LN> sink{out + d * nt, nt, hop, 2 * p0 * hop - guard, guard};
  fft::transform_to<kFftThreads, LN>(ConjSrc{Y + d * ld + p0 * NF}, sink, buf0, buf1, tw, Fh);
}

size_t fft_smem(int ln, int F) { return fft::smem_bytes(ln, F); }

template <int LN, typename TIn>
cudaError_t launch_forward(const TIn *in, int32_t nf, int64_t nt, int64_t hop, int32_t guard, int64_t npair, int F,
                           float2 *X, int64_t ld, cudaStream_t s) {
  const size_t smem = fft_smem(LN, F);
  cudaError_t e = cudaFuncSetAttribute(fft_forward_kernel<LN, TIn>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((npair + F - 1) / F), (unsigned)nf);
  fft_forward_kernel<LN, TIn><<<grid, kFftThreads, smem, s>>>(in, nt, hop, guard, npair, F, X, ld);
  return cudaGetLastError();
}

template <int LN>
cudaError_t launch_inverse(const float2 *Y, int32_t nd, int64_t ld, int64_t nt, int64_t hop, int32_t guard,
                           int64_t npair, int F, float *out, cudaStream_t s) {
  const size_t smem = fft_smem(LN, F);
  cudaError_t e = cudaFuncSetAttribute(fft_inverse_kernel<LN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((npair + F - 1) / F), (unsigned)nd);
  fft_inverse_kernel<LN><<<grid, kFftThreads, smem, s>>>(Y, ld, nt, hop, guard, npair, F, out);
  return cudaGetLastError();
}

template <int B>
cudaError_t launch_merge(const MergeArgs &a, int64_t nk, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(fft_merge_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fft_merge_kernel<B><<<(unsigned)(nk / B), merge_threads<B>(), smem, s>>>(a);
  return cudaGetLastError();
}

size_t merge_smem(int B, int max_w, int max_shift, int cap_odd, int cap_even) {
  return ((size_t)max_w + (size_t)max_shift + 1 + (size_t)cap_odd + (size_t)cap_even) * (size_t)B * sizeof(float2);
}

}  // namespace
}  // namespace fdmt

struct fdmt_fft_s {
  int32_t nf = 0, nd = 0, dtype = 0, levels = 0, ln = 0, bins = 0, max_w = 0, max_shift = 0, cap_odd = 0,
          cap_even = 0, F = 1;
  int64_t nt = 0, hop = 0, npair = 0, nk = 0;
  int device = -1;
  bool host_only = false;
  size_t ws_bytes = 0, merge_smem = 0;
  std::vector<int64_t> ob;
  std::vector<int32_t> rows;
  int4 *ops1 = nullptr;  // level 1
  uint2 *ops = nullptr;  // levels >= 2, packed
  float2 *tw = nullptr;
  fdmt::Profiler prof;
};

namespace {

void profile_release(fdmt::Profiler &pr) {
  for (cudaEvent_t e : pr.start) cudaEventDestroy(e);
  for (cudaEvent_t e : pr.stop) cudaEventDestroy(e);
  pr = fdmt::Profiler();
}

void release(fdmt_fft_s *p) {
  if (p == nullptr) return;
  profile_release(p->prof);
  cudaFree(p->ops);
  cudaFree(p->ops1);
  cudaFree(p->tw);
  delete p;
}

}  // namespace

extern "C" {

int fdmt_fft_plan(double f_min, double f_max, int32_t nf, int64_t nt, int32_t nd, int32_t dtype, int32_t block,
                  int32_t bins, uint32_t flags, fdmt_fft_t *out) {
  using namespace fdmt;
  if (out == nullptr) return FDMT_ERR_INVALID_ARG;
  *out = nullptr;
  if (dtype != FDMT_F32_F32 && dtype != FDMT_U8_I32) return FDMT_ERR_INVALID_ARG;
  if (nt < 1 || nd < 1 || nf < 2 || nf > 65535 || nd > 65535) return FDMT_ERR_INVALID_ARG;
  if (flags & ~(uint32_t)FDMT_PLAN_HOST_ONLY) return FDMT_ERR_INVALID_ARG;
  if (bins != 0 && bins != 1 && bins != 2 && bins != 4 && bins != 8) return FDMT_ERR_INVALID_ARG;
  const int64_t guard = (int64_t)nd - 1;
  int ln = 0;
  if (block == 0) {  // hop >= 3/4 of the block where the sizes allow
    ln = kMinLn;
    while (ln < kMaxLn && ((int64_t)1 << ln) < 4 * guard) ++ln;
  } else {
    if (block < (1 << kMinLn) || block > (1 << kMaxLn) || (block & (block - 1)) != 0) return FDMT_ERR_INVALID_ARG;
    while ((1 << ln) < block) ++ln;
  }
  const int64_t N = (int64_t)1 << ln;
  if (N <= guard) return FDMT_ERR_UNSUPPORTED;  // Nd - 1 >= block: no output per block
  Tables t;
  const std::string err = build_tables(f_min, f_max, nf, nd, t);
  if (!err.empty()) return FDMT_ERR_INVALID_ARG;
  if (t.levels > kMaxLevels) return FDMT_ERR_UNSUPPORTED;
  fdmt_fft_s *p = new (std::nothrow) fdmt_fft_s;
  if (p == nullptr) return FDMT_ERR_NO_MEMORY;
  p->nf = nf;
  p->nd = nd;
  p->dtype = dtype;
  p->nt = nt;
  p->levels = t.levels;
  p->ln = ln;
  p->hop = N - guard;
  const int64_t nblk = (nt + p->hop - 1) / p->hop;
  p->npair = (nblk + 1) / 2;
  p->nk = p->npair * N;
  p->F = (int)std::max<int64_t>(1, kFftSamples / N);
  p->max_w = t.max_sweep + 1;
  for (const RowOp &op : t.ops)
    if (op.hi >= 0) p->max_shift = std::max(p->max_shift, op.shift);
  for (int l = 1; l <= t.levels; ++l) {
    const bool stored = l < t.levels || t.levels == 1;
    if (!stored) continue;
    if (l & 1)
      p->cap_odd = std::max(p->cap_odd, t.level_rows[l]);
    else
      p->cap_even = std::max(p->cap_even, t.level_rows[l]);
  }
  p->cap_even = std::max(p->cap_even, nf);  // the input tile during level 1
  if (bins == 0) {
    // Measured at Nf = Nd = 1024: 2 bins x 256 threads, four blocks per SM,
    // beat 4 bins x 512 threads, two per SM (0.89 against 0.94 ms); then
    // whatever fits.
    const struct {
      int b;
      size_t limit;
    } pref[] = {{2, kSmemFourPerSm}, {4, kSmemTwoPerSm}, {1, kSmemFourPerSm}, {8, kSmemLimit},
                {4, kSmemLimit},     {2, kSmemLimit},   {1, kSmemLimit}};
    for (const auto &c : pref)
      if (merge_smem(c.b, p->max_w, p->max_shift, p->cap_odd, p->cap_even) <= c.limit) {
        bins = c.b;
        break;
      }
  }
  p->bins = bins;
  p->merge_smem = bins ? merge_smem(bins, p->max_w, p->max_shift, p->cap_odd, p->cap_even) : kSmemLimit + 1;
  if (p->merge_smem > kSmemLimit || p->nk / bins > INT32_MAX || p->npair > INT32_MAX ||
      p->hop > INT32_MAX / 2) {
    delete p;
    return FDMT_ERR_UNSUPPORTED;
  }
  const int64_t rows_ws = std::max(nf, nd);
  if (p->nk > INT64_MAX / 8 / rows_ws) {
    delete p;
    return FDMT_ERR_UNSUPPORTED;
  }
  p->ws_bytes = (size_t)rows_ws * (size_t)p->nk * sizeof(float2);
  p->ob.assign(t.levels + 2, 0);
  p->rows.assign(t.levels + 2, 0);
  for (int l = 1; l <= t.levels; ++l) p->rows[l] = t.level_rows[l];
  p->host_only = (flags & FDMT_PLAN_HOST_ONLY) != 0;
  if (!p->host_only) {
    if (cudaGetDevice(&p->device) != cudaSuccess) {
      cudaGetLastError();
      delete p;
      return FDMT_ERR_CUDA;
    }
    // level-0 row -> (channel, partial sum)
    std::vector<int2> r0(t.level_rows[0]);
    for (int32_t c = 0; c < nf; ++c)
      for (int32_t j = 0; j <= t.init[c].sweep; ++j) r0[t.init[c].row0 + j] = make_int2(c, j);
    std::vector<int4> ops1;
    for (int64_t i = t.ops_begin[1]; i < t.ops_begin[2]; ++i) {
      const RowOp &op = t.ops[i];
      const int2 lo = r0[op.lo];
      const int2 hi = op.hi >= 0 ? r0[op.hi] : make_int2(-1, 0);
      if (op.hi >= 0 && op.shift != lo.y) {  // level 1 shifts the upper channel by the lower row
        release(p);
        return FDMT_ERR_INVALID_ARG;
      }
      ops1.push_back(make_int4(lo.x, lo.y, hi.x, hi.y));
    }
    std::vector<uint2> packed;
    for (int l = 2; l <= t.levels; ++l) {
      p->ob[l] = (int64_t)packed.size();
      for (int64_t i = t.ops_begin[l]; i < t.ops_begin[l + 1]; ++i) {
        const RowOp &op = t.ops[i];
        // rows of stored levels fit 16 bits (the shared-memory cap bounds them)
        const uint32_t hi = op.hi >= 0 ? (uint32_t)op.hi : kNoUpper;
        packed.push_back(make_uint2((uint32_t)op.lo | (hi << 16), op.hi >= 0 ? (uint32_t)op.shift : 0u));
      }
    }
    std::vector<float2> tw(N);
    for (int64_t m = 0; m < N; ++m) {
      const double ang = -2.0 * 3.14159265358979323846 * (double)m / (double)N;
      tw[m] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    const size_t n1 = std::max<size_t>(ops1.size(), 1), np = std::max<size_t>(packed.size(), 1);
    bool ok = cudaMalloc(&p->ops1, n1 * sizeof(int4)) == cudaSuccess &&
              cudaMalloc(&p->ops, np * sizeof(uint2)) == cudaSuccess &&
              cudaMalloc(&p->tw, tw.size() * sizeof(float2)) == cudaSuccess;
    ok = ok && cudaMemcpy(p->ops1, ops1.data(), ops1.size() * sizeof(int4), cudaMemcpyHostToDevice) == cudaSuccess &&
         (packed.empty() ||
          cudaMemcpy(p->ops, packed.data(), packed.size() * sizeof(uint2), cudaMemcpyHostToDevice) == cudaSuccess) &&
         cudaMemcpy(p->tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      release(p);
      return FDMT_ERR_NO_MEMORY;
    }
  }
  *out = p;
  return FDMT_OK;
}

void fdmt_fft_destroy(fdmt_fft_t p) { release(p); }

int fdmt_fft_workspace_bytes(fdmt_fft_t p, size_t *bytes) {
  if (p == nullptr || bytes == nullptr) return FDMT_ERR_INVALID_ARG;
  *bytes = p->ws_bytes;
  return FDMT_OK;
}

int fdmt_fft_info(fdmt_fft_t p, int32_t *block, int64_t *hop, int64_t *pairs, int32_t *bins) {
  if (p == nullptr) return FDMT_ERR_INVALID_ARG;
  if (block) *block = 1 << p->ln;
  if (hop) *hop = p->hop;
  if (pairs) *pairs = p->npair;
  if (bins) *bins = p->bins;
  return FDMT_OK;
}

int fdmt_fft_execute(fdmt_fft_t p, const void *in, float *out, void *workspace, size_t ws_bytes, void *stream) {
  using namespace fdmt;
  if (p == nullptr || in == nullptr || out == nullptr || workspace == nullptr) return FDMT_ERR_INVALID_ARG;
  if (p->host_only) return FDMT_ERR_INVALID_ARG;
  if (ws_bytes < p->ws_bytes || (reinterpret_cast<uintptr_t>(workspace) & 15u) ||
      (reinterpret_cast<uintptr_t>(out) & 3u) || (p->dtype == FDMT_F32_F32 && (reinterpret_cast<uintptr_t>(in) & 3u)))
    return FDMT_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) {
    cudaGetLastError();
    return FDMT_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float2 *X = static_cast<float2 *>(workspace);
  const int32_t guard = p->nd - 1;
  cudaError_t e = cudaSuccess;
  p->prof.begin(s, K_FFT_FORWARD, 0);
#define FDMT_FWD(LN)                                                                                          \
  case LN:                                                                                                    \
    e = p->dtype == FDMT_U8_I32                                                                               \
            ? launch_forward<LN>(static_cast<const uint8_t *>(in), p->nf, p->nt, p->hop, guard, p->npair, p->F, X, \
                                 p->nk, s)                                                                    \
            : launch_forward<LN>(static_cast<const float *>(in), p->nf, p->nt, p->hop, guard, p->npair, p->F, X,   \
                                 p->nk, s);                                                                   \
    break;
  switch (p->ln) {
    FDMT_FWD(8)
    FDMT_FWD(9)
    FDMT_FWD(10)
    FDMT_FWD(11)
    FDMT_FWD(12)
    default: return FDMT_ERR_UNSUPPORTED;
  }
#undef FDMT_FWD
  p->prof.end(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FDMT_ERR_CUDA;
  }
  MergeArgs a{};
  a.X = X;
  a.Y = X;
  a.ld = p->nk;
  a.tw = p->tw;
  a.mask = (uint32_t)((1u << p->ln) - 1u);
  a.ops1 = p->ops1;
  a.ops = p->ops;
  a.nf = p->nf;
  a.levels = p->levels;
  a.max_w = p->max_w;
  a.max_shift = p->max_shift;
  a.cap_odd = p->cap_odd;
  a.cap_even = p->cap_even;
  for (int l = 0; l <= p->levels; ++l) {
    a.ob[l] = p->ob[l];
    a.rows[l] = p->rows[l];
  }
  p->prof.begin(s, K_FFT_MERGE, p->levels);
  switch (p->bins) {
    case 8: e = launch_merge<8>(a, p->nk, p->merge_smem, s); break;
    case 4: e = launch_merge<4>(a, p->nk, p->merge_smem, s); break;
    case 2: e = launch_merge<2>(a, p->nk, p->merge_smem, s); break;
    default: e = launch_merge<1>(a, p->nk, p->merge_smem, s); break;
  }
  p->prof.end(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FDMT_ERR_CUDA;
  }
#define FDMT_INV(LN) \
  case LN: e = launch_inverse<LN>(X, p->nd, p->nk, p->nt, p->hop, guard, p->npair, p->F, out, s); break;
  p->prof.begin(s, K_FFT_INVERSE, 0);
  switch (p->ln) {
    FDMT_INV(8)
    FDMT_INV(9)
    FDMT_INV(10)
    FDMT_INV(11)
    FDMT_INV(12)
    default: return FDMT_ERR_UNSUPPORTED;
  }
#undef FDMT_INV
  p->prof.end(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FDMT_ERR_CUDA;
  }
  return FDMT_OK;
}

int fdmt_fft_profile_enable(fdmt_fft_t p, int32_t capacity) {
  if (p == nullptr || capacity < 0 || p->host_only) return FDMT_ERR_INVALID_ARG;
  profile_release(p->prof);
  fdmt::Profiler &pr = p->prof;
  for (int32_t i = 0; i < capacity; ++i) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
      if (a) cudaEventDestroy(a);
      profile_release(pr);
      cudaGetLastError();
      return FDMT_ERR_CUDA;
    }
    pr.start.push_back(a);
    pr.stop.push_back(b);
  }
  pr.kernel.assign(capacity, -1);
  pr.level.assign(capacity, -1);
  pr.next = 0;
  return FDMT_OK;
}

int fdmt_fft_profile_read(fdmt_fft_t p, int32_t *kernel_ids, float *ms, int32_t n, int64_t *launches) {
  if (p == nullptr || launches == nullptr) return FDMT_ERR_INVALID_ARG;
  fdmt::Profiler &pr = p->prof;
  *launches = pr.next;
  if (!pr.on()) return FDMT_OK;
  const int64_t cap = (int64_t)pr.start.size();
  const int64_t have = pr.next < cap ? pr.next : cap;
  if (have > 0 && (kernel_ids == nullptr || ms == nullptr)) return FDMT_ERR_INVALID_ARG;
  const int64_t first = pr.next - have;
  int64_t written = 0;
  for (int64_t j = 0; j < have && written < n; ++j) {
    const size_t i = (size_t)((first + j) % cap);
    float t = 0.f;
    if (cudaEventSynchronize(pr.stop[i]) != cudaSuccess ||
        cudaEventElapsedTime(&t, pr.start[i], pr.stop[i]) != cudaSuccess) {
      cudaGetLastError();
      return FDMT_ERR_CUDA;
    }
    kernel_ids[written] = pr.kernel[i];
    ms[written] = t;
    ++written;
  }
  pr.next = 0;
  return FDMT_OK;
}

}  // extern "C"
