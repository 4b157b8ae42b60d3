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
// the transforms already done; the first pass reads the voltages straight
// from global memory); a thread loads R values at stride Nf / R,
// multiplies them by the pass twiddles exp(-2 pi i r k / (Ns R)), does an
// R-point DFT in registers (radix-2 stages with constant twiddles) and
// stores the results at stride Ns, ping-ponging between two buffers, so an
// Nf = 1024 transform takes three passes and three barriers.  Twiddles come
// from a per-block table exp(-2 pi i m / Nf) (sincospif); padding slots keep
// the strided stores and twiddle reads off shared bank conflicts.  The squared
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

// One Stockham pass of radix R over the F transforms in x (Nf = 2^LN each)
// into y, after transforms of size NS: every index is a compile-time
// constant offset from the work item's base.
template <int LN, int NS, int R, bool GLOBAL_SRC = false>
__device__ __forceinline__ void stockham_pass(const float2 *__restrict__ x, float2 *__restrict__ y,
                                              const float2 *__restrict__ tw, int F) {
  constexpr int NF = 1 << LN;
  constexpr int LR = R == 2 ? 1 : (R == 4 ? 2 : (R == 8 ? 3 : 4));
  constexpr int LPER = LN - LR;
  constexpr int PER = 1 << LPER;  // work items per transform
  constexpr int LNS = ilog2(NS);
  for (int w = threadIdx.x; w < F * PER; w += kFbThreads) {
    const int f = w >> LPER, j = w & (PER - 1);
    const int k = j & (NS - 1);
    const int base = f * NF + j;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = GLOBAL_SRC ? __ldg(x + base + r * PER) : x[pad16(base + r * PER)];
    if (NS > 1) {
      // exp(-2 pi i r k / (NS R)) = tw[r k NF / (NS R)]
      const int step = k << (LN - LNS - LR);
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[pad4(r * step)]);
    }
    dft_regs<R>(v);
    const int out0 = f * NF + (j >> LNS) * NS * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) y[pad16(out0 + r * NS)] = v[bitrev_small(r, LR)];
  }
}

// All passes of an Nf = 2^LN transform: radix 16 while 16 remains, then the
// rest; returns the buffer holding the result.
template <int LN, int NS>
__device__ __forceinline__ float2 *stockham(float2 *x, float2 *y, const float2 *tw, int F) {
  if constexpr ((1 << LN) / NS <= 1) {
    return x;
  } else {
    constexpr int REM = (1 << LN) / NS;
    constexpr int R = REM >= 16 ? 16 : REM;
    stockham_pass<LN, NS, R>(x, y, tw, F);
    __syncthreads();
    return stockham<LN, NS * R>(y, x, tw, F);
  }
}

// The first pass reads the voltages straight from global memory (each
// thread's R loads are coalesced across the warp) into buffer y.
template <int LN>
__device__ __forceinline__ float2 *stockham_from_global(const float2 *src, float2 *x, float2 *y, const float2 *tw,
                                                        int F) {
  constexpr int NF = 1 << LN;
  constexpr int R = NF >= 16 ? 16 : NF;
  stockham_pass<LN, 1, R, true>(src, y, tw, F);
  __syncthreads();
  return stockham<LN, R>(y, x, tw, F);
}

template <int LN>
__global__ void __launch_bounds__(kFbThreads)
filterbank_kernel(const float2 *__restrict__ v, int nbin, int64_t nt, int T, float *__restrict__ out) {
  constexpr int NF = 1 << LN;
  extern __shared__ __align__(16) float2 sm[];
  const int F = T * nbin;      // transforms per block
  const int padded = pad16(F * NF);
  float2 *buf0 = sm;             // [F][nf], padded
  float2 *buf1 = sm + padded;    // [F][nf], padded
  float2 *tw = buf1 + padded;    // [nf], padded by pad4
  const int64_t t_first = (int64_t)blockIdx.x * T;
  const int T_here = (int)((nt - t_first) < (int64_t)T ? (nt - t_first) : (int64_t)T);
  const int F_here = T_here * nbin;
  for (int m = threadIdx.x; m < NF; m += kFbThreads) {
    float s, c;
    sincospif(-2.0f * (float)m / (float)NF, &s, &c);
    tw[pad4(m)] = make_float2(c, s);
  }
  __syncthreads();  // twiddles
  const float2 *x = stockham_from_global<LN>(v + t_first * nbin * (int64_t)NF, buf0, buf1, tw, F_here);
  // Consecutive threads take consecutive times of one channel row (T is a
  // power of two; the last block may hold fewer times).
  const int lT = 31 - __clz(T);
  for (int i = threadIdx.x; i < NF * T; i += kFbThreads) {
    const int c = i >> lT, tt = i & (T - 1);
    if (tt >= T_here) continue;
    const int k = (c + NF / 2) & (NF - 1);
    float acc = 0.0f;
    for (int b = 0; b < nbin; ++b) {
      const float2 z = x[pad16((tt * nbin + b) * NF + k)];
      acc = __fadd_rn(acc, __fadd_rn(__fmul_rn(z.x, z.x), __fmul_rn(z.y, z.y)));
    }
    out[(int64_t)c * nt + t_first + tt] = acc;
  }
}

template <int LN>
cudaError_t launch_filterbank(const float2 *v, int nbin, int64_t nt, int T, float *out, size_t smem,
                              cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(filterbank_kernel<LN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (nt + T - 1) / T;
  filterbank_kernel<LN><<<(unsigned)blocks, kFbThreads, smem, s>>>(v, nbin, nt, T, out);
  return cudaGetLastError();
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
  const size_t smem = (2 * padded + (size_t)nf + (size_t)nf / 4) * sizeof(float2);
  if (smem > 200 * 1024) return FDMT_ERR_UNSUPPORTED;
  if ((nt + T - 1) / T > INT32_MAX) return FDMT_ERR_UNSUPPORTED;
  const float2 *vv = static_cast<const float2 *>(volts);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  switch (log2nf) {
    case 1: e = fdmt::launch_filterbank<1>(vv, nbin, nt, T, out, smem, cs); break;
    case 2: e = fdmt::launch_filterbank<2>(vv, nbin, nt, T, out, smem, cs); break;
    case 3: e = fdmt::launch_filterbank<3>(vv, nbin, nt, T, out, smem, cs); break;
    case 4: e = fdmt::launch_filterbank<4>(vv, nbin, nt, T, out, smem, cs); break;
    case 5: e = fdmt::launch_filterbank<5>(vv, nbin, nt, T, out, smem, cs); break;
    case 6: e = fdmt::launch_filterbank<6>(vv, nbin, nt, T, out, smem, cs); break;
    case 7: e = fdmt::launch_filterbank<7>(vv, nbin, nt, T, out, smem, cs); break;
    case 8: e = fdmt::launch_filterbank<8>(vv, nbin, nt, T, out, smem, cs); break;
    case 9: e = fdmt::launch_filterbank<9>(vv, nbin, nt, T, out, smem, cs); break;
    case 10: e = fdmt::launch_filterbank<10>(vv, nbin, nt, T, out, smem, cs); break;
    case 11: e = fdmt::launch_filterbank<11>(vv, nbin, nt, T, out, smem, cs); break;
    default: e = fdmt::launch_filterbank<12>(vv, nbin, nt, T, out, smem, cs); break;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FDMT_ERR_CUDA;
  }
  return FDMT_OK;
}
