// In-block Stockham FFT over shared memory, shared by the STFT filterbank
// and FFT-FDMT kernels.
//
// A block of THREADS threads transforms F sequences of 2^LN complex64
// samples at once.  Each pass takes radix R = min(16, 2^LN / NS) (NS = the
// size of the transforms already done): a work item loads R values at
// stride 2^LN / R, multiplies them by the pass twiddles
// exp(-2 pi i r k / (NS R)), does an R-point DFT in registers (radix-2
// stages with constant twiddles) and stores the results at stride NS,
// ping-ponging between two buffers; a 1024-point transform takes three
// passes.  The first pass reads through a source functor (global memory,
// two real rows packed as one complex row, ...); later passes read shared
// memory.  Buffers hold element i at pad16(i) and the twiddle table
// exp(-2 pi i m / 2^LN) holds entry m at pad4(m): the padding keeps the
// strided stores and twiddle reads off shared bank conflicts.  The result is
// in natural order.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace fdmt {
namespace fft {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y)); }
// Complex product with fused multiply-adds (the transforms are compared
// within an error bound, not bit for bit).
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}

// exp(-2 pi i j / len) for the in-register DFTs (len <= 16): the values of
// cos and sin at multiples of pi/8.
__device__ __forceinline__ float2 unit_root(int j, int len) {
  const int e = j * (16 / len);  // exponent in units of 2 pi / 16
  constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508977f, h = 0.70710678118654752f;
  switch (e & 15) {
    case 0: return make_float2(1.0f, 0.0f);
    case 1: return make_float2(c1, -s1);
    case 2: return make_float2(h, -h);
    case 3: return make_float2(s1, -c1);
    case 4: return make_float2(0.0f, -1.0f);
    case 5: return make_float2(-s1, -c1);
    case 6: return make_float2(-h, -h);
    case 7: return make_float2(-c1, -s1);
    default: return make_float2(-1.0f, 0.0f);  // e = 8 (j < len / 2 never reaches above)
  }
}

// Shared-memory index of transform element i: one padding slot after every
// 16 elements, so the stride-R stores of a pass spread over the banks.
__host__ __device__ constexpr int pad16(int i) { return i + (i >> 4); }

// Twiddle table index: one padding slot after every 4 entries, so the
// stride-4 twiddle reads of a radix-16 pass after 16-point transforms hit
// distinct banks.
__host__ __device__ constexpr int pad4(int m) { return m + (m >> 2); }

__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v >> 1); }

__host__ __device__ constexpr int bitrev_small(int r, int bits) {
  int o = 0;
  for (int i = 0; i < bits; ++i) o |= ((r >> i) & 1) << (bits - 1 - i);
  return o;
}

// Elements (padded) of F transforms of 2^LN samples plus the pad4 twiddle
// table of one block: the shared memory a block needs for two buffers.
__host__ __device__ constexpr size_t smem_bytes(int ln, int F) {
  return (2 * (size_t)pad16(F << ln) + (size_t)pad4(1 << ln)) * sizeof(float2);
}

// In-place R-point DFT, decimation in frequency: on return v[bitrev(k)] = X[k].
template <int R>
__device__ __forceinline__ void dft_regs(float2 (&v)[R]) {
#pragma unroll
  for (int len = R; len >= 2; len >>= 1) {
    const int h = len / 2;
#pragma unroll
    for (int base = 0; base < R; base += len) {
#pragma unroll
      for (int j = 0; j < h; ++j) {
        const float2 a = v[base + j], b = v[base + j + h];
        v[base + j] = cadd(a, b);
        const float2 d = csub(a, b);
        // exponent of the twiddle in units of 2 pi / 16 (compile-time)
        const int e = j * (16 / len);
        constexpr float hr = 0.70710678118654752f;
        if (j == 0)
          v[base + j + h] = d;
        else if (e == 4)  // times -i
          v[base + j + h] = make_float2(d.y, -d.x);
        else if (e == 2)  // times (1 - i) / sqrt(2)
          v[base + j + h] = make_float2(__fmul_rn(hr, __fadd_rn(d.x, d.y)), __fmul_rn(hr, __fsub_rn(d.y, d.x)));
        else if (e == 6)  // times -(1 + i) / sqrt(2)
          v[base + j + h] = make_float2(__fmul_rn(hr, __fsub_rn(d.y, d.x)), -__fmul_rn(hr, __fadd_rn(d.x, d.y)));
        else
          v[base + j + h] = cmul(d, unit_root(j, len));
      }
    }
  }
}

// Shared-memory source of a pass: element i at pad16(i).
struct SmemSrc {
  const float2 *x;
  __device__ __forceinline__ float2 operator()(int i) const { return x[pad16(i)]; }
};

// Global source: F transforms stored back to back.
struct GlobalSrc {
  const float2 *__restrict__ x;
  __device__ __forceinline__ float2 operator()(int i) const { return __ldg(x + i); }
};

// Shared-memory destination of a pass: element i at pad16(i).
struct SmemDst {
  float2 *y;
  __device__ __forceinline__ void operator()(int i, float2 v) const { y[pad16(i)] = v; }
};

// Fills the pad4 twiddle table exp(-2 pi i m / 2^LN) (sincospif).
template <int THREADS, int LN>
__device__ __forceinline__ void twiddles(float2 *tw) {
  for (int m = threadIdx.x; m < (1 << LN); m += THREADS) {
    float s, c;
    sincospif(-2.0f * (float)m / (float)(1 << LN), &s, &c);
    tw[pad4(m)] = make_float2(c, s);
  }
}

// One Stockham pass of radix R over the F transforms read through `src`
// (flattened element index f 2^LN + i) into `dst` (same indexing), after
// transforms of size NS: every index is a compile-time constant offset from
// the work item's base.  In the last pass (NS R = 2^LN) work item j of a
// transform writes elements j + r NS, so a warp's stores are consecutive.
template <int THREADS, int LN, int NS, int R, class Src, class Dst>
__device__ __forceinline__ void pass(const Src &src, const Dst &dst, const float2 *__restrict__ tw, int F) {
  constexpr int NF = 1 << LN;
  constexpr int LR = R == 2 ? 1 : (R == 4 ? 2 : (R == 8 ? 3 : 4));
  constexpr int LPER = LN - LR;
  constexpr int PER = 1 << LPER;  // work items per transform
  constexpr int LNS = ilog2(NS);
  for (int w = threadIdx.x; w < F * PER; w += THREADS) {
    const int f = w >> LPER, j = w & (PER - 1);
    const int k = j & (NS - 1);
    const int base = f * NF + j;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src(base + r * PER);
    if (NS > 1) {
      // exp(-2 pi i r k / (NS R)) = tw[r k NF / (NS R)]
      const int step = k << (LN - LNS - LR);
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[pad4(r * step)]);
    }
    dft_regs<R>(v);
    const int out0 = f * NF + (j >> LNS) * NS * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst(out0 + r * NS, v[bitrev_small(r, LR)]);
  }
}

// Remaining passes after transforms of size NS, buffers x -> y -> x ...;
// returns the buffer holding the result.
template <int THREADS, int LN, int NS>
__device__ __forceinline__ float2 *rest(float2 *x, float2 *y, const float2 *tw, int F) {
  if constexpr ((1 << LN) / NS <= 1) {
    return x;
  } else {
    constexpr int REM = (1 << LN) / NS;
    constexpr int R = REM >= 16 ? 16 : REM;
    pass<THREADS, LN, NS, R>(SmemSrc{x}, SmemDst{y}, tw, F);
    __syncthreads();
    return rest<THREADS, LN, NS * R>(y, x, tw, F);
  }
}

// Whole transform: the first pass reads through `src` into y, the rest
// alternate between the two shared buffers; returns the result buffer.
// Ends with a barrier (the result is visible to the whole block).
template <int THREADS, int LN, class Src>
__device__ __forceinline__ float2 *transform(const Src &src, float2 *x, float2 *y, const float2 *tw, int F) {
  constexpr int NF = 1 << LN;
  constexpr int R = NF >= 16 ? 16 : NF;
  pass<THREADS, LN, 1, R>(src, SmemDst{y}, tw, F);
  __syncthreads();
  return rest<THREADS, LN, R>(y, x, tw, F);
}

// Remaining passes after transforms of size NS, the last one writing
// through `sink` instead of shared memory.
template <int THREADS, int LN, int NS, class Sink>
__device__ __forceinline__ void rest_to(float2 *x, float2 *y, const Sink &sink, const float2 *tw, int F) {
  constexpr int REM = (1 << LN) / NS;
  constexpr int R = REM >= 16 ? 16 : REM;
  if constexpr (R == REM) {
    pass<THREADS, LN, NS, R>(SmemSrc{x}, sink, tw, F);
  } else {
    pass<THREADS, LN, NS, R>(SmemSrc{x}, SmemDst{y}, tw, F);
    __syncthreads();
    rest_to<THREADS, LN, NS * R>(y, x, sink, tw, F);
  }
}

// Whole transform from `src` to `sink` (element index f 2^LN + k, natural
// order): the first pass reads `src`, the last writes `sink`, the passes in
// between use the two shared buffers.  No barrier at the end.
template <int THREADS, int LN, class Src, class Sink>
__device__ __forceinline__ void transform_to(const Src &src, const Sink &sink, float2 *x, float2 *y, const float2 *tw,
                                             int F) {
  constexpr int NF = 1 << LN;
  constexpr int R = NF >= 16 ? 16 : NF;
  if constexpr (R == NF) {
    pass<THREADS, LN, 1, R>(src, sink, tw, F);
  } else {
    pass<THREADS, LN, 1, R>(src, SmemDst{y}, tw, F);
    __syncthreads();
    rest_to<THREADS, LN, R>(y, x, sink, tw, F);
  }
}

}  // namespace fft
}  // namespace fdmt
