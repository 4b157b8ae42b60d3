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
// (T nbin transforms, ~8192 complex samples) in shared memory: a radix-2
// decimation-in-time FFT, loaded in bit-reversed order, log2 Nf butterfly
// stages in place, twiddles exp(-2 pi i m / Nf) from sincospif; then the
// squared magnitudes are summed over the bin and written as an [Nf][T] tile
// (T consecutive samples of every channel row).
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/fdmt.h"

namespace fdmt {
namespace {

constexpr int kFbThreads = 256;
constexpr int kFbSamples = 8192;  // complex samples transformed per block at once

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(__fsub_rn(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)),
                     __fadd_rn(__fmul_rn(a.x, b.y), __fmul_rn(a.y, b.x)));
}

__global__ void __launch_bounds__(kFbThreads)
filterbank_kernel(const float2 *__restrict__ v, int nf, int log2nf, int nbin, int64_t nt, int T,
                  float *__restrict__ out) {
  extern __shared__ __align__(16) float2 sm[];
  const int F = T * nbin;     // transforms per block
  float2 *x = sm;             // [F][nf]
  float2 *tw = sm + F * nf;   // [nf / 2]
  const int64_t t_first = (int64_t)blockIdx.x * T;
  const int T_here = (int)((nt - t_first) < (int64_t)T ? (nt - t_first) : (int64_t)T);
  const int F_here = T_here * nbin;
  const int hnf = nf >> 1;
  for (int m = threadIdx.x; m < hnf; m += kFbThreads) {
    float s, c;
    sincospif(-2.0f * (float)m / (float)nf, &s, &c);
    tw[m] = make_float2(c, s);
  }
  const float2 *src = v + t_first * nbin * (int64_t)nf;
  for (int i = threadIdx.x; i < F_here * nf; i += kFbThreads) {
    const int f = i >> log2nf, m = i & (nf - 1);
    x[f * nf + (int)(__brev((unsigned)m) >> (32 - log2nf))] = __ldg(src + i);
  }
  __syncthreads();
  for (int s = 1; s <= log2nf; ++s) {
    const int half = 1 << (s - 1);
    const int step = nf >> s;  // twiddle index stride of this stage
    for (int p = threadIdx.x; p < F_here * hnf; p += kFbThreads) {
      const int f = p >> (log2nf - 1), q = p & (hnf - 1);
      const int j = q & (half - 1), g = q >> (s - 1);
      const int i0 = f * nf + (g << s) + j, i1 = i0 + half;
      const float2 a = x[i0];
      const float2 b = cmul(x[i1], tw[j * step]);
      x[i0] = make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y));
      x[i1] = make_float2(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y));
    }
    __syncthreads();
  }
  // Consecutive threads take consecutive times of one channel row.
  for (int i = threadIdx.x; i < nf * T_here; i += kFbThreads) {
    const int c = i / T_here, tt = i - c * T_here;
    const int k = (c + hnf) & (nf - 1);
    float acc = 0.0f;
    for (int b = 0; b < nbin; ++b) {
      const float2 z = x[(tt * nbin + b) * nf + k];
      acc = __fadd_rn(acc, __fadd_rn(__fmul_rn(z.x, z.x), __fmul_rn(z.y, z.y)));
    }
    out[(int64_t)c * nt + t_first + tt] = acc;
  }
}

}  // namespace
}  // namespace fdmt

extern "C" int fdmt_filterbank(const void *volts, int64_t n, int32_t nf, int32_t nbin, float *out, int64_t nt,
                               void *stream) {
  if (volts == nullptr || out == nullptr || (reinterpret_cast<uintptr_t>(volts) & 7u) ||
      (reinterpret_cast<uintptr_t>(out) & 3u))
    return FDMT_ERR_INVALID_ARG;
  if (nf < 2 || nf > 4096 || (nf & (nf - 1)) != 0 || nbin < 1 || nbin > 1024) return FDMT_ERR_INVALID_ARG;
  if (nt < 1 || n < 0 || nt > n / ((int64_t)nf * nbin)) return FDMT_ERR_INVALID_ARG;
  int log2nf = 0;
  while ((1 << log2nf) < nf) ++log2nf;
  // Output times per block: as many transforms as fit kFbSamples (at least
  // one time's bin).
  int T = fdmt::kFbSamples / (nf * nbin);
  if (T < 1) T = 1;
  const size_t smem = ((size_t)T * nbin * nf + (size_t)(nf / 2)) * sizeof(float2);
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
