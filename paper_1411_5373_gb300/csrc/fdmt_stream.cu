// Overlap-save streaming of the transform (contracts in include/fdmt.h).
//
// Output column t depends only on input columns [t - Nd + 1, t] (the
// recursion only ever looks back in time, Algorithm 1, and treats samples
// before the first as zero, the copy rule of section 4).  A continuous
// stream is therefore transformed chunk by chunk: each chunk is appended to
// the last `carry` >= Nd - 1 input columns of the previous one, the window
// (carry + chunk columns) is transformed with an ordinary plan, and the
// window's last `chunk` output columns are exactly the stream's output for
// that chunk.  The first chunk sees a carry of zeros, which is the copy rule.
//
// Built on the public entry points (fdmt_plan, fdmt_execute); the stream
// owns its window buffers, allocated once at creation.
#include <cuda_runtime.h>

#include <cstdint>
#include <new>

#include "../../include/fdmt.h"

struct fdmt_stream_s {
  fdmt_plan_t plan = nullptr;
  int32_t nf = 0, nd = 0, dtype = 0;
  int64_t chunk = 0, carry = 0, window = 0;
  size_t in_es = 0;
  void *win[2] = {nullptr, nullptr};  // input windows [nf][window], ping-pong
  void *wout = nullptr;               // window output [nd][window]
  void *ws = nullptr;
  size_t ws_bytes = 0;
  int cur = 0;                        // window holding the latest chunk
};

namespace {

size_t in_size(int32_t dtype) { return dtype == FDMT_U8_I32 ? 1 : 4; }

void release(fdmt_stream_s *s) {
  if (s == nullptr) return;
  if (s->plan != nullptr) fdmt_destroy(s->plan);
  cudaFree(s->win[0]);
  cudaFree(s->win[1]);
  cudaFree(s->wout);
  cudaFree(s->ws);
  delete s;
}

}  // namespace

extern "C" {

int fdmt_stream_create(double f_min, double f_max, int32_t nf, int64_t chunk, int32_t nd, int32_t dtype,
                       uint32_t flags, fdmt_stream_t *out) {
  if (out == nullptr) return FDMT_ERR_INVALID_ARG;
  *out = nullptr;
  if (chunk < 16 || chunk % 16 != 0 || nd < 1 || (flags & FDMT_PLAN_HOST_ONLY)) return FDMT_ERR_INVALID_ARG;
  if (dtype != FDMT_U8_I32 && dtype != FDMT_F32_F32 && dtype != FDMT_F32_F16STATE) return FDMT_ERR_INVALID_ARG;
  const int64_t carry = ((int64_t)nd - 1 + 15) / 16 * 16;
  const int64_t window = carry + chunk;
  // Validate the shape on the host before any device allocation.
  fdmt_plan_t probe = nullptr;
  int st = fdmt_plan(f_min, f_max, nf, window, nd, dtype, flags | FDMT_PLAN_HOST_ONLY, &probe);
  if (st != FDMT_OK) return st;
  fdmt_destroy(probe);

  fdmt_stream_s *s = new (std::nothrow) fdmt_stream_s;
  if (s == nullptr) return FDMT_ERR_NO_MEMORY;
  s->nf = nf;
  s->nd = nd;
  s->dtype = dtype;
  s->chunk = chunk;
  s->carry = carry;
  s->window = window;
  s->in_es = in_size(dtype);
  if ((st = fdmt_plan(f_min, f_max, nf, window, nd, dtype, flags, &s->plan)) != FDMT_OK) {
    release(s);
    return st;
  }
  if ((st = fdmt_workspace_bytes(s->plan, &s->ws_bytes)) != FDMT_OK) {
    release(s);
    return st;
  }
  const size_t in_bytes = (size_t)nf * window * s->in_es;
  const size_t out_bytes = (size_t)nd * window * 4;
  if (cudaMalloc(&s->win[0], in_bytes) != cudaSuccess || cudaMalloc(&s->win[1], in_bytes) != cudaSuccess ||
      cudaMalloc(&s->wout, out_bytes) != cudaSuccess ||
      cudaMalloc(&s->ws, s->ws_bytes > 0 ? s->ws_bytes : 256) != cudaSuccess) {
    cudaGetLastError();
    release(s);
    return FDMT_ERR_NO_MEMORY;
  }
  // The carry before the first chunk is zero (the copy rule).
  if (cudaMemset(s->win[0], 0, in_bytes) != cudaSuccess || cudaMemset(s->win[1], 0, in_bytes) != cudaSuccess) {
    cudaGetLastError();
    release(s);
    return FDMT_ERR_CUDA;
  }
  *out = s;
  return FDMT_OK;
}

int fdmt_stream_info(fdmt_stream_t s, int64_t *carry, int64_t *window) {
  if (s == nullptr) return FDMT_ERR_INVALID_ARG;
  if (carry != nullptr) *carry = s->carry;
  if (window != nullptr) *window = s->window;
  return FDMT_OK;
}

int fdmt_stream_push(fdmt_stream_t s, const void *in, void *out, void *stream) {
  if (s == nullptr || in == nullptr || out == nullptr) return FDMT_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15u) return FDMT_ERR_INVALID_ARG;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  const int nxt = s->cur ^ 1;
  char *dst = static_cast<char *>(s->win[nxt]);
  const char *prev = static_cast<const char *>(s->win[s->cur]);
  const size_t pitch = (size_t)s->window * s->in_es;
  cudaError_t e = cudaSuccess;
  // New window = [last `carry` columns of the previous window | chunk].
  if (s->carry > 0)
    e = cudaMemcpy2DAsync(dst, pitch, prev + (size_t)s->chunk * s->in_es, pitch, (size_t)s->carry * s->in_es, s->nf,
                          cudaMemcpyDeviceToDevice, cs);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(dst + (size_t)s->carry * s->in_es, pitch, in, (size_t)s->chunk * s->in_es,
                          (size_t)s->chunk * s->in_es, s->nf, cudaMemcpyDeviceToDevice, cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FDMT_ERR_CUDA;
  }
  const int st = fdmt_execute(s->plan, dst, nullptr, s->wout, s->ws, s->ws_bytes, stream);
  if (st != FDMT_OK) return st;
  // The window's last `chunk` output columns are the stream's output.
  e = cudaMemcpy2DAsync(out, (size_t)s->chunk * 4, static_cast<char *>(s->wout) + (size_t)s->carry * 4,
                        (size_t)s->window * 4, (size_t)s->chunk * 4, s->nd, cudaMemcpyDeviceToDevice, cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FDMT_ERR_CUDA;
  }
  s->cur = nxt;
  return FDMT_OK;
}

int fdmt_stream_reset(fdmt_stream_t s, void *stream) {
  if (s == nullptr) return FDMT_ERR_INVALID_ARG;
  const size_t in_bytes = (size_t)s->nf * s->window * s->in_es;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(s->win[0], 0, in_bytes, cs) != cudaSuccess ||
      cudaMemsetAsync(s->win[1], 0, in_bytes, cs) != cudaSuccess) {
    cudaGetLastError();
    return FDMT_ERR_CUDA;
  }
  s->cur = 0;
  return FDMT_OK;
}

void fdmt_stream_destroy(fdmt_stream_t s) { release(s); }

}  // extern "C"
