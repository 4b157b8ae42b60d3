// Input mapping in front of the transform: channel order and the d_min
// pre-shift (contracts in include/fdmt.h, fdmt_curve_params).
//
// Section 4.2 of Zackay & Ofek (arXiv:1411.5373): to scan delays from d_min
// instead of 0, the input is first shifted by the delay of d_min, so that
// row d of the transform follows delay d_min + d.  Channel k (ascending
// frequency, lower edge e_k) is delayed by s_k = floor(d_min r(e_k) + 1/2)
// samples, r the delay fraction of the curve family:
//     I'[k][t] = I[src(k)][t - s_k]   (0 for t < s_k),
// with src(k) = k for ascending input rows and Nf - 1 - k for descending
// (channel 0 = f_max first).  The transposed map takes the gradient back:
//     grad_raw[src(k)][u] = g[k][u + s_k]   (0 for u + s_k >= Nt).
// One pass over the input each way, 16 bytes written per thread.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/fdmt.h"
#include "fdmt_internal.h"

namespace fdmt {
namespace {

constexpr int kMapThreads = 256;

template <class T>
__global__ void __launch_bounds__(kMapThreads)
map_input_kernel(const T *__restrict__ raw, T *__restrict__ out, const int32_t *__restrict__ shift, int nf,
                 int64_t nt, int descending) {
  constexpr int E = 16 / sizeof(T);
  const int k = blockIdx.y;
  const int64_t t0 = ((int64_t)blockIdx.x * kMapThreads + threadIdx.x) * E;
  if (t0 >= nt) return;
  const int src = descending ? nf - 1 - k : k;
  const int64_t s = shift[k];
  const T *row = raw + (int64_t)src * nt;
  const int64_t u = t0 - s;  // source of the first output sample
  if (sizeof(T) == 1 && u >= 0) {
    // Bytes: five aligned words around [u, u + 16), funnel-shifted into
    // place (rows start 16-byte aligned: nt is a multiple of 16).
    const int64_t a = u & ~(int64_t)3;
    const int r = (int)(u & 3);
    const uint32_t *wp = reinterpret_cast<const uint32_t *>(row + a);
    uint32_t q[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) q[i] = a + 4 * i < nt ? __ldg(wp + i) : 0u;
    uint4 o;
    o.x = __funnelshift_r(q[0], q[1], 8 * r);
    o.y = __funnelshift_r(q[1], q[2], 8 * r);
    o.z = __funnelshift_r(q[2], q[3], 8 * r);
    o.w = __funnelshift_r(q[3], q[4], 8 * r);
    *reinterpret_cast<uint4 *>(out + (int64_t)k * nt + t0) = o;
    return;
  }
  alignas(16) T v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int64_t ue = u + e;
    v[e] = ue >= 0 ? __ldg(row + ue) : T(0);
  }
  *reinterpret_cast<int4 *>(out + (int64_t)k * nt + t0) = *reinterpret_cast<const int4 *>(v);
}

__global__ void __launch_bounds__(kMapThreads)
unmap_grad_kernel(const float *__restrict__ g, float *__restrict__ grad, const int32_t *__restrict__ shift, int nf,
                  int64_t nt, int descending) {
  const int k = blockIdx.y;
  const int64_t u0 = ((int64_t)blockIdx.x * kMapThreads + threadIdx.x) * 4;
  if (u0 >= nt) return;
  const int dst = descending ? nf - 1 - k : k;
  const int64_t s = shift[k];
  const float *row = g + (int64_t)k * nt;
  float4 v;
  float *pv = reinterpret_cast<float *>(&v);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int64_t t = u0 + e + s;
    pv[e] = t < nt ? __ldg(row + t) : 0.0f;
  }
  *reinterpret_cast<float4 *>(grad + (int64_t)dst * nt + u0) = v;
}

}  // namespace

cudaError_t map_input(const DeviceTables &dt, int dtype, const void *raw, void *out, int64_t nt, cudaStream_t s) {
  const int per = kMapThreads * (dtype == FDMT_U8_I32 ? 16 : 4);
  const dim3 grid((unsigned)((nt + per - 1) / per), (unsigned)dt.nf);
  dt.prof->begin(s, K_MAP_INPUT, 0);
  if (dtype == FDMT_U8_I32)
    map_input_kernel<uint8_t><<<grid, kMapThreads, 0, s>>>(static_cast<const uint8_t *>(raw),
                                                           static_cast<uint8_t *>(out), dt.in_shift, dt.nf, nt,
                                                           dt.descending);
  else
    map_input_kernel<float><<<grid, kMapThreads, 0, s>>>(static_cast<const float *>(raw), static_cast<float *>(out),
                                                         dt.in_shift, dt.nf, nt, dt.descending);
  dt.prof->end(s);
  return cudaGetLastError();
}

cudaError_t unmap_grad(const DeviceTables &dt, const float *g, float *grad, int64_t nt, cudaStream_t s) {
  const int per = kMapThreads * 4;
  const dim3 grid((unsigned)((nt + per - 1) / per), (unsigned)dt.nf);
  dt.prof->begin(s, K_UNMAP_GRAD, 0);
  unmap_grad_kernel<<<grid, kMapThreads, 0, s>>>(g, grad, dt.in_shift, dt.nf, nt, dt.descending);
  dt.prof->end(s);
  return cudaGetLastError();
}

}  // namespace fdmt
