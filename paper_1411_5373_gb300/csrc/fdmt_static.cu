// fdmt_execute_static: the plain forward transform with its scratch memory in
// a fixed device array that is part of this library, so the call itself
// allocates nothing.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the time
// they run the transform: a real-time pipeline that must not allocate once an
// observation has started (an allocation can stall, fragment the pool or fail
// mid-stream), or a host framework that owns all device memory through its
// own pool and forbids other allocations.  Such callers create the plan once
// at start-up (fdmt_plan allocates only its delay tables) and then call this
// entry point, which uses the array below instead of a caller workspace.
//
// The array costs FDMT_STATIC_SCRATCH_BYTES of device memory on every GPU
// that loads the library, held until the process exits.  Every call shares
// it and it keeps the previous call's contents; nothing in it has to start at
// zero, because the plain schedule writes every scratch row before reading
// it within the same call.  Calls that overlap on the GPU (different streams,
// or different host threads) race on the array.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/fdmt.h"
#include "fdmt_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[FDMT_STATIC_SCRATCH_BYTES];

// Device address of g_static_scratch in the current device's context.  In
// host code the symbol names a host-side stand-in, never the device memory,
// so the address must come from cudaGetSymbolAddress with that device
// current.  It is looked up on every call rather than cached: a cached
// address would outlive the context it belongs to if the host application
// resets the device (cudaDeviceReset) and the library's module is loaded
// again into the new context.  The lookup is a table read in the runtime
// once the module is loaded; the first call on a device may load it.
int scratch_address(void **out) {
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return FDMT_ERR_CUDA;
  }
  *out = p;
  return FDMT_OK;
}

}  // namespace

extern "C" int fdmt_execute_static(fdmt_plan_t plan, const void *in, const float *weights,
                                   void *out, void *stream) {
  fdmt::PlanView v;
  if (!fdmt::plan_view(plan, &v) || v.host_only) return FDMT_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return FDMT_ERR_CUDA;
  }
  if (dev != v.device) return FDMT_ERR_INVALID_ARG;
  if (in == nullptr || out == nullptr || (reinterpret_cast<uintptr_t>(in) & 15u) != 0 ||
      (reinterpret_cast<uintptr_t>(out) & 15u) != 0)
    return FDMT_ERR_INVALID_ARG;
  if (weights != nullptr && v.dtype == FDMT_U8_I32) return FDMT_ERR_INVALID_ARG;
  // The input mapping needs a copy of the input: not on this path.
  if (v.mapped) return FDMT_ERR_UNSUPPORTED;
  // This entry point always runs the plain schedule (one launch per level),
  // also for plans made with the fused schedule; plans whose plain-schedule
  // scratch does not fit the fixed array are refused.
  if (v.ws_bytes > (size_t)FDMT_STATIC_SCRATCH_BYTES) return FDMT_ERR_WORKSPACE;
  void *base = nullptr;
  int st = scratch_address(&base);
  if (st != FDMT_OK) return st;
  void *bufs[2] = {base, static_cast<char *>(base) + v.ws_split};
  cudaError_t e = fdmt::run_plain(*v.dev, v.dtype, in, weights, out, bufs, v.nt,
                                  static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FDMT_ERR_CUDA;
  }
  return FDMT_OK;
}
