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
// (T nbin transforms, up to 4096 complex samples) in shared memory with the
// Stockham FFT of fdmt_stockham.cuh (radix 16 in registers, the first pass
// reading the voltages straight from global memory), so an Nf = 1024
// transform takes three passes and three barriers.  The squared magnitudes
// are summed over the bin and written as an [Nf][T] tile.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/fdmt.h"
#include "fdmt_stockham.cuh"

namespace fdmt {
namespace {

constexpr int kFbThreads = 256;
constexpr int kFbSamples = 4096;  // complex samples transformed per block at once

template <int LN>
__global__ void __launch_bounds__(kFbThreads)
filterbank_kernel(const float2 *__restrict__ v, int nbin, int64_t nt, int T, float *__restrict__ out) {
  constexpr int NF = 1 << LN;
  extern __shared__ __align__(16) float2 sm[];
  const int F = T * nbin;      // transforms per block
  const int padded = fft::pad16(F * NF);
  float2 *buf0 = sm;             // [F][nf], padded
  float2 *buf1 = sm + padded;    // [F][nf], padded
  float2 *tw = buf1 + padded;    // [nf], padded by pad4
  const int64_t t_first = (int64_t)blockIdx.x * T;
  const int T_here = (int)((nt - t_first) < (int64_t)T ? (nt - t_first) : (int64_t)T);
  const int F_here = T_here * nbin;
  fft::twiddles<kFbThreads, LN>(tw);
  __syncthreads();  // twiddles
  const float2 *x =
      fft::transform<kFbThreads, LN>(fft::GlobalSrc{v + t_first * nbin * (int64_t)NF}, buf0, buf1, tw, F_here);
  // Consecutive threads take consecutive times of one channel row (T is a
  // power of two; the last block may hold fewer times).
  const int lT = 31 - __clz(T);
  for (int i = threadIdx.x; i < NF * T; i += kFbThreads) {
    const int c = i >> lT, tt = i & (T - 1);
    if (tt >= T_here) continue;
    const int k = (c + NF / 2) & (NF - 1);
    float acc = 0.0f;
    for (int b = 0; b < nbin; ++b) {
      const float2 z = x[fft::pad16((tt * nbin + b) * NF + k)];
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
