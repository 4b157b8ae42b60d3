// Element types and 4-wide vector helpers shared by the FDMT kernels.
//
// Every floating-point add and multiply goes through an explicitly rounded
// intrinsic (__fadd_rn / __fmul_rn), which the compiler never contracts into
// an FMA, so the association of each sum is exactly the one written.
#pragma once

#include <cuda_fp16.h>
#include <cstdint>

#include "fdmt_tables.h"

namespace fdmt {

// Scalar conversions into the accumulator type and back.
__device__ __forceinline__ float acc_of(float x) { return x; }
__device__ __forceinline__ float acc_of(__half x) { return __half2float(x); }
__device__ __forceinline__ int32_t acc_of(int32_t x) { return x; }
__device__ __forceinline__ int32_t acc_of(uint8_t x) { return (int32_t)x; }

template <class T> __device__ __forceinline__ T store_of(float x);
template <> __device__ __forceinline__ float store_of<float>(float x) { return x; }
template <> __device__ __forceinline__ __half store_of<__half>(float x) { return __float2half_rn(x); }

__device__ __forceinline__ float acc_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ int32_t acc_add(int32_t a, int32_t b) { return a + b; }

// Four consecutive elements <-> four accumulators.  p must be aligned to
// 4 elements (16 bytes for 4-byte types, 8 for half, 4 for uint8).
__device__ __forceinline__ void load4(const float *p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4 *>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load4(const int32_t *p, int32_t (&v)[4]) {
  const int4 q = *reinterpret_cast<const int4 *>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load4(const __half *p, float (&v)[4]) {
  const uint2 q = *reinterpret_cast<const uint2 *>(p);
  const __half2 a = *reinterpret_cast<const __half2 *>(&q.x);
  const __half2 b = *reinterpret_cast<const __half2 *>(&q.y);
  const float2 fa = __half22float2(a), fb = __half22float2(b);
  v[0] = fa.x; v[1] = fa.y; v[2] = fb.x; v[3] = fb.y;
}
__device__ __forceinline__ void load4(const uint8_t *p, int32_t (&v)[4]) {
  const uchar4 q = *reinterpret_cast<const uchar4 *>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}

__device__ __forceinline__ void store4(float *p, const float (&v)[4]) {
  *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store4(int32_t *p, const int32_t (&v)[4]) {
  *reinterpret_cast<int4 *>(p) = make_int4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store4(__half *p, const float (&v)[4]) {
  const __half2 a = __floats2half2_rn(v[0], v[1]);
  const __half2 b = __floats2half2_rn(v[2], v[3]);
  uint2 q;
  q.x = *reinterpret_cast<const unsigned *>(&a);
  q.y = *reinterpret_cast<const unsigned *>(&b);
  *reinterpret_cast<uint2 *>(p) = q;
}

template <class A> __device__ __forceinline__ void zero4(A (&v)[4]) {
  v[0] = v[1] = v[2] = v[3] = A(0);
}

// Elements u .. u+3 of a row of length nt (a multiple of 4), zero outside
// [0, nt), from at most two aligned vector loads.  `rem` = u mod 4 must be
// uniform across the warp for the select to stay divergence-free; the
// callers guarantee it (u = t0 - shift with t0 a multiple of 4 and one shift
// per row).
template <class T, class A>
__device__ __forceinline__ void load4_shifted(const T *row, int64_t u, int64_t nt, A (&v)[4]) {
  const int64_t base = (u >> 2) << 2;  // floor to a multiple of 4
  const int rem = (int)(u - base);
  A a[4], b[4];
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

}  // namespace fdmt
