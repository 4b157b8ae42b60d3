// Pipelined host execution (contracts in include/fdmt.h).
//
// A stream of independent transforms whose inputs and outputs live in host
// memory: step k copies its input to the device, transforms it and copies
// the output back, and consecutive steps overlap -- the input copy of step
// k + 1 and the output copy of step k - 1 run on their own CUDA streams
// while step k computes.  Two device slots (input and output buffers) take
// turns; events order each slot's reuse (a slot's input is overwritten only
// after the transform that read it, its output only after the copy that
// read it).  The copy engines then run both directions at once, so a step
// costs about the larger of its two copies instead of their sum.
//
// Built on the public entry points (fdmt_execute); the pipeline owns its
// streams, events and device buffers, allocated once at creation.
#include <cuda_runtime.h>

#include <cstdint>
#include <new>

#include "../../include/fdmt.h"

struct fdmt_pipeline_s {
  fdmt_plan_t plan = nullptr;  // borrowed
  size_t in_bytes = 0, out_bytes = 0, ws_bytes = 0;
  void *dev_in[2] = {nullptr, nullptr};
  void *dev_out[2] = {nullptr, nullptr};
  void *ws = nullptr;
  cudaStream_t s_in = nullptr, s_run = nullptr, s_out = nullptr;
  cudaEvent_t copied_in[2] = {nullptr, nullptr};  // input slot filled
  cudaEvent_t ran[2] = {nullptr, nullptr};        // transform of the slot done
  cudaEvent_t copied_out[2] = {nullptr, nullptr}; // output slot read back
  int64_t steps = 0;
};

namespace {

void release(fdmt_pipeline_s *p) {
  if (p == nullptr) return;
  for (int i = 0; i < 2; ++i) {
    cudaFree(p->dev_in[i]);
    cudaFree(p->dev_out[i]);
    if (p->copied_in[i]) cudaEventDestroy(p->copied_in[i]);
    if (p->ran[i]) cudaEventDestroy(p->ran[i]);
    if (p->copied_out[i]) cudaEventDestroy(p->copied_out[i]);
  }
  cudaFree(p->ws);
  if (p->s_in) cudaStreamDestroy(p->s_in);
  if (p->s_run) cudaStreamDestroy(p->s_run);
  if (p->s_out) cudaStreamDestroy(p->s_out);
  delete p;
}

}  // namespace

extern "C" {

int fdmt_pipeline_create(fdmt_plan_t plan, fdmt_pipeline_t *out) {
  if (out == nullptr) return FDMT_ERR_INVALID_ARG;
  *out = nullptr;
  int32_t levels = 0;
  if (plan == nullptr || fdmt_num_levels(plan, &levels) != FDMT_OK) return FDMT_ERR_INVALID_ARG;
  size_t ws = 0;
  int st = fdmt_workspace_bytes(plan, &ws);
  if (st != FDMT_OK) return st;
  int32_t nf = 0, nd = 0, dtype = 0;
  int64_t nt = 0;
  if ((st = fdmt_plan_shape(plan, &nf, &nt, &nd, &dtype)) != FDMT_OK) return st;
  fdmt_pipeline_s *p = new (std::nothrow) fdmt_pipeline_s;
  if (p == nullptr) return FDMT_ERR_NO_MEMORY;
  p->plan = plan;
  p->in_bytes = (size_t)nf * (size_t)nt * (dtype == FDMT_U8_I32 ? 1 : 4);
  p->out_bytes = (size_t)nd * (size_t)nt * 4;
  p->ws_bytes = ws;
  bool ok = true;
  for (int i = 0; i < 2 && ok; ++i)
    ok = cudaMalloc(&p->dev_in[i], p->in_bytes) == cudaSuccess &&
         cudaMalloc(&p->dev_out[i], p->out_bytes) == cudaSuccess;
  ok = ok && cudaMalloc(&p->ws, ws > 0 ? ws : 256) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    release(p);
    return FDMT_ERR_NO_MEMORY;
  }
  ok = cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking) == cudaSuccess &&
       cudaStreamCreateWithFlags(&p->s_run, cudaStreamNonBlocking) == cudaSuccess &&
       cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking) == cudaSuccess;
  for (int i = 0; i < 2 && ok; ++i)
    ok = cudaEventCreateWithFlags(&p->copied_in[i], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&p->ran[i], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&p->copied_out[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    release(p);
    return FDMT_ERR_CUDA;
  }
  *out = p;
  return FDMT_OK;
}

int fdmt_pipeline_push(fdmt_pipeline_t p, const void *host_in, void *host_out) {
  if (p == nullptr || host_in == nullptr || host_out == nullptr) return FDMT_ERR_INVALID_ARG;
  const int slot = (int)(p->steps & 1);
  const bool reuse = p->steps >= 2;
  cudaError_t e = cudaSuccess;
  // Input copy: the slot's previous transform must have read its input.
  if (reuse) e = cudaStreamWaitEvent(p->s_in, p->ran[slot], 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->dev_in[slot], host_in, p->in_bytes, cudaMemcpyHostToDevice, p->s_in);
  if (e == cudaSuccess) e = cudaEventRecord(p->copied_in[slot], p->s_in);
  // Transform: after the input copy, and after the slot's previous output
  // was copied back.
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->s_run, p->copied_in[slot], 0);
  if (e == cudaSuccess && reuse) e = cudaStreamWaitEvent(p->s_run, p->copied_out[slot], 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FDMT_ERR_CUDA;
  }
  const int st = fdmt_execute(p->plan, p->dev_in[slot], nullptr, p->dev_out[slot], p->ws, p->ws_bytes, p->s_run);
  if (st != FDMT_OK) return st;
  e = cudaEventRecord(p->ran[slot], p->s_run);
  // Output copy.
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->s_out, p->ran[slot], 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host_out, p->dev_out[slot], p->out_bytes, cudaMemcpyDeviceToHost, p->s_out);
  if (e == cudaSuccess) e = cudaEventRecord(p->copied_out[slot], p->s_out);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FDMT_ERR_CUDA;
  }
  ++p->steps;
  return FDMT_OK;
}

int fdmt_pipeline_wait(fdmt_pipeline_t p) {
  if (p == nullptr) return FDMT_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(p->s_in) != cudaSuccess || cudaStreamSynchronize(p->s_run) != cudaSuccess ||
      cudaStreamSynchronize(p->s_out) != cudaSuccess) {
    cudaGetLastError();
    return FDMT_ERR_CUDA;
  }
  return FDMT_OK;
}

void fdmt_pipeline_destroy(fdmt_pipeline_t p) {
  if (p == nullptr) return;
  fdmt_pipeline_wait(p);
  release(p);
}

}  // extern "C"
