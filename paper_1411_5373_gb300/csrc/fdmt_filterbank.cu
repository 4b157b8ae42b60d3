// STFT filterbank in front of the transform (contracts in include/fdmt.h).
//
// Section 2 of Zackay & Ofek (arXiv:1411.5373): the voltage series is cut
// into blocks of Nf samples, each block is Fourier transformed (STFT) and
// the squared magnitude at each frequency is kept, optionally binned in
// time (the footnote): I[c][t] = sum_{b < nbin} |X_{t nbin + b}[k(c)]|^2,
// with channel c in ascending frequency holding DFT bin k = (c + Nf/2) mod Nf
// of the complex (baseband) voltages.
//
// One block of threads transforms the Nf-sample blocks of T output times
// (T nbin transforms, up to 4096 complex samples) in shared memory with a
// Stockham FFT: each pass takes radix R = min(16, Nf / Ns) (Ns = the size of
// the transforms already done); a thread loads R values at stride Nf / R,
// multiplies them by the pass twiddles exp(-2 pi i r k / (Ns R)), does an
// R-point DFT in registers (radix-2 stages with constant twiddles) and
// stores the results at stride Ns, ping-ponging between two buffers, so an
// Nf = 1024 transform takes three passes and three barriers.  Twiddles come
// from a per-block table exp(-2 pi i m / Nf) (sincospif); one padding slot
// per 16 elements keeps the strided stores off shared bank conflicts.  The squared
// magnitudes are summed over the bin and written as an [Nf][T] tile.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/fdmt.h"

namespace fdmt {
namespace {

constexpr int kFbThreads = 256;
constexpr int kFbSamples = 4096;  // complex samples transformed per block at once

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y)); }
// Complex product with fused multiply-adds (the transform is compared
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

__host__ __device__ constexpr int bitrev_small(int r, int bits) {
  int o = 0;
  for (int i = 0; i < bits; ++i) o |= ((r >> i) & 1) << (bits - 1 - i);
  return o;
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
        v[base + j + h] = j == 0 ? d : cmul(d, unit_root(j, len));
      }
    }
  }
}

// One Stockham pass of radix R over the F transforms in x (Nf each) into y.
template <int R>
__device__ __forceinline__ void stockham_pass(const float2 *__restrict__ x, float2 *__restrict__ y,
                                              const float2 *__restrict__ tw, int nf, int log2nf, int ns, int F) {
  constexpr int LR = R == 2 ? 1 : (R == 4 ? 2 : (R == 8 ? 3 : 4));
  const int lper = log2nf - LR;
  const int per = 1 << lper;  // work items per transform
  for (int w = threadIdx.x; w < F * per; w += kFbThreads) {
    const int f = w >> lper, j = w & (per - 1);
    const int k = j & (ns - 1);
    const int base = f * nf + j;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = x[pad16(base + r * per)];
    if (ns > 1) {
      // exp(-2 pi i r k / (ns R)) = tw[r k nf / (ns R)]
      const int step = k << (log2nf - (31 - __clz(ns)) - LR);
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[(r * step) & (nf - 1)]);
    }
    dft_regs<R>(v);
    const int out0 = f * nf + (j / ns) * ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) y[pad16(out0 + r * ns)] = v[bitrev_small(r, LR)];
  }
}

__global__ void __launch_bounds__(kFbThreads)
filterbank_kernel(const float2 *__restrict__ v, int nf, int log2nf, int nbin, int64_t nt, int T,
                  float *__restrict__ out) {
  extern __shared__ __align__(16) float2 sm[];
  const int F = T * nbin;      // transforms per block
  const int padded = pad16(F * nf);
  float2 *buf0 = sm;             // [F][nf], padded
  float2 *buf1 = sm + padded;    // [F][nf], padded
  float2 *tw = buf1 + padded;    // [nf]
  const int64_t t_first = (int64_t)blockIdx.x * T;
  const int T_here = (int)((nt - t_first) < (int64_t)T ? (nt - t_first) : (int64_t)T);
  const int F_here = T_here * nbin;
  for (int m = threadIdx.x; m < nf; m += kFbThreads) {
    float s, c;
    sincospif(-2.0f * (float)m / (float)nf, &s, &c);
    tw[m] = make_float2(c, s);
  }
  const float4 *src = reinterpret_cast<const float4 *>(v + t_first * nbin * (int64_t)nf);
  for (int i = threadIdx.x; i < F_here * nf / 2; i += kFbThreads) {
    const float4 q = __ldg(src + i);
    buf0[pad16(2 * i)] = make_float2(q.x, q.y);
    buf0[pad16(2 * i + 1)] = make_float2(q.z, q.w);
  }
  __syncthreads();
  float2 *x = buf0, *y = buf1;
  for (int ns = 1; ns < nf;) {
    const int rem = nf / ns;
    if (rem >= 16) {
      stockham_pass<16>(x, y, tw, nf, log2nf, ns, F_here);
      ns *= 16;
    } else if (rem == 8) {
      stockham_pass<8>(x, y, tw, nf, log2nf, ns, F_here);
      ns *= 8;
    } else if (rem == 4) {
      stockham_pass<4>(x, y, tw, nf, log2nf, ns, F_here);
      ns *= 4;
    } else {
      stockham_pass<2>(x, y, tw, nf, log2nf, ns, F_here);
      ns *= 2;
    }
    __syncthreads();
    float2 *t = x;
    x = y;
    y = t;
  }
  // Consecutive threads take consecutive times of one channel row (T is a
  // power of two; the last block may hold fewer times).
  const int hnf = nf >> 1;
  const int lT = 31 - __clz(T);
  for (int i = threadIdx.x; i < nf * T; i += kFbThreads) {
    const int c = i >> lT, tt = i & (T - 1);
    if (tt >= T_here) continue;
    const int k = (c + hnf) & (nf - 1);
    float acc = 0.0f;
    for (int b = 0; b < nbin; ++b) {
      const float2 z = x[pad16((tt * nbin + b) * nf + k)];
      acc = __fadd_rn(acc, __fadd_rn(__fmul_rn(z.x, z.x), __fmul_rn(z.y, z.y)));
    }
    out[(int64_t)c * nt + t_first + tt] = acc;
  }
}

}  // namespace
}  // namespace fdmt

extern "C" int fdmt_filterbank(const void *volts, int64_t n, int32_t nf, int32_t nbin, float *out, int64_t nt,
                               void *stream) {
  if (volts == nullptr || out == nullptr || (reinterpret_cast<uintptr_t>(volts) & 15u) ||
      (reinterpret_cast<uintptr_t>(out) & 3u))
    return FDMT_ERR_INVALID_ARG;
  if (nf < 2 || nf > 4096 || (nf & (nf - 1)) != 0 || nbin < 1 || nbin > 1024) return FDMT_ERR_INVALID_ARG;
  if (nt < 1 || n < 0 || nt > n / ((int64_t)nf * nbin)) return FDMT_ERR_INVALID_ARG;
  int log2nf = 0;
  while ((1 << log2nf) < nf) ++log2nf;
  // Output times per block: a power of two, as many transforms as fit
  // kFbSamples (at least one time's bin).
  int T = fdmt::kFbSamples / (nf * nbin);
  if (T < 1) T = 1;
  while (T & (T - 1)) T &= T - 1;  // a power of two
  const size_t padded = (size_t)T * nbin * nf + ((size_t)T * nbin * nf >> 4);
  const size_t smem = (2 * padded + (size_t)nf) * sizeof(float2);
  if (smem > 200 * 1024) return FDMT_ERR_UNSUPPORTED;
  cudaError_t e = cudaFuncSetAttribute(fdmt::filterbank_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e == cudaSuccess) {
    const int64_t blocks = (nt + T - 1) / T;
    if (blocks > INT32_MAX) return FDMT_ERR_UNSUPPORTED;
    fdmt::filterbank_kernel<<<(unsigned)blocks, fdmt::kFbThreads, smem, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const float2 *>(volts), nf, log2nf, nbin, nt, T, out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FDMT_ERR_CUDA;
  }
  return FDMT_OK;
}
