// Batched FDMT of independent beams with uneven shapes in one persistent
// launch (declarations and contracts in include/fdmt.h).
//
// Work items, in level-major order over all beams: level 0 = (beam,
// block of channels, time tile) computes the Option-1 partial sums of
// section 4; level l >= 1 = (beam, block of delay rows, time tile) applies
// the addition rule.  A block takes the next item from a global counter;
// an item of level l waits until all items of level l - 1 of its beam are
// done (a per-(beam, level) counter).  Items are handed out in an order in
// which every producer precedes its consumers and all blocks are resident,
// so a wait can only run out if a producer is missing; each wait is bounded
// by the global timer and a wait that runs out stops the whole launch
// through a status word instead of hanging.
//
// State written by other blocks is read with L1-bypassing loads (the
// ping-pong buffers are rewritten level after level, so an L1 line from an
// earlier level would be stale).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/fdmt.h"
#include "fdmt_batch_fused.h"
#include "fdmt_common.cuh"
#include "fdmt_internal.h"
#include "fdmt_tables.h"

namespace fdmt {
namespace {

constexpr int kBatchThreads = 256;
constexpr int kMaxLevels = 16;
constexpr int kChannelsPerItem = 4;

struct BeamDev {
  const void *in;
  void *out;
  void *buf[2];
  int64_t nt;
  int32_t nf, nd, levels, init_off;
  int64_t ops_off[kMaxLevels];  // [l] offset of level l's RowOps (l >= 1)
  int32_t rows[kMaxLevels];     // rows of level l
};

struct Seg {
  int64_t first;  // first global item index
  int32_t beam, level, rblocks, tiles;
  int32_t need;   // items of (beam, level - 1) that must be done first
  int32_t pad;
};

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// L1-bypassing vector loads.
__device__ __forceinline__ void load4_cg(const float *p, float (&v)[4]) {
  const float4 q = __ldcg(reinterpret_cast<const float4 *>(p));
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load4_cg(const int32_t *p, int32_t (&v)[4]) {
  const int4 q = __ldcg(reinterpret_cast<const int4 *>(p));
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load4_cg(const __half *p, float (&v)[4]) {
  const uint2 q = __ldcg(reinterpret_cast<const uint2 *>(p));
  const __half2 a = *reinterpret_cast<const __half2 *>(&q.x);
  const __half2 b = *reinterpret_cast<const __half2 *>(&q.y);
  const float2 fa = __half22float2(a), fb = __half22float2(b);
  v[0] = fa.x; v[1] = fa.y; v[2] = fb.x; v[3] = fb.y;
}

template <class T, class A>
__device__ __forceinline__ void load4_shifted_cg(const T *row, int64_t u, int64_t nt, A (&v)[4]) {
  const int64_t base = (u >> 2) << 2;
  const int rem = (int)(u - base);
  A a[4], b[4];
  if (base >= 0 && base < nt) load4_cg(row + base, a); else zero4(a);
  if (rem == 0) {
    v[0] = a[0]; v[1] = a[1]; v[2] = a[2]; v[3] = a[3];
    return;
  }
  if (base + 4 >= 0 && base + 4 < nt) load4_cg(row + base + 4, b); else zero4(b);
  switch (rem) {
    case 1: v[0] = a[1]; v[1] = a[2]; v[2] = a[3]; v[3] = b[0]; break;
    case 2: v[0] = a[2]; v[1] = a[3]; v[2] = b[0]; v[3] = b[1]; break;
    default: v[0] = a[3]; v[1] = b[0]; v[2] = b[1]; v[3] = b[2]; break;
  }
}

template <class TIn, class TS, class TO, class A>
__global__ void __launch_bounds__(kBatchThreads)
batch_kernel(const BeamDev *__restrict__ beams, const Seg *__restrict__ segs, int nsegs, int64_t total,
             const InitOp *__restrict__ inits, const RowOp *__restrict__ ops,
             unsigned long long *counter, int *done, int *status, int rows_per_item, int tile,
             uint64_t wait_ns) {
  __shared__ long long s_item;
  __shared__ int s_abort;
  for (;;) {
    if (threadIdx.x == 0) {
      s_item = (long long)atomicAdd(counter, 1ull);
      s_abort = 0;
    }
    __syncthreads();
    const long long g = s_item;
    if (g >= total) return;
    int lo = 0, hi = nsegs - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (segs[mid].first <= g) lo = mid; else hi = mid - 1;
    }
    const Seg sg = segs[lo];
    const BeamDev &bm = beams[sg.beam];
    const int64_t local = g - sg.first;
    const int rb = (int)(local / sg.tiles);
    const int64_t t_begin = (local % sg.tiles) * (int64_t)tile;
    const int64_t nt = bm.nt;
    if (sg.level > 0) {
      if (threadIdx.x == 0) {
        volatile int *d = done + sg.beam * kMaxLevels + (sg.level - 1);
        const uint64_t t0 = global_ns();
        while (*d < sg.need) {
          if (*(volatile int *)status != 0 || global_ns() - t0 > wait_ns) {
            atomicExch(status, 1);
            s_abort = 1;
            break;
          }
          __nanosleep(500);
        }
        __threadfence();
      }
      __syncthreads();
      if (s_abort) return;
    }
    const int64_t t_end = min(nt, t_begin + (int64_t)tile);
    if (sg.level == 0) {
      const int k0 = rb * kChannelsPerItem;
      const int k1 = min(bm.nf, k0 + kChannelsPerItem);
      const TIn *src = static_cast<const TIn *>(bm.in);
      TS *st = static_cast<TS *>(bm.buf[0]);
      for (int k = k0; k < k1; ++k) {
        const InitOp op = inits[bm.init_off + k];
        const TIn *x = src + (int64_t)k * nt;
        for (int64_t t0 = t_begin + 4 * threadIdx.x; t0 < t_end; t0 += 4 * kBatchThreads) {
          A run[4], v[4];
          load4(x + t0, run);
          TS *dst = st + (int64_t)op.row0 * nt + t0;
          store4(dst, run);
          for (int j = 1; j <= op.sweep; ++j) {
            load4_shifted(x, t0 - j, nt, v);
#pragma unroll
            for (int c = 0; c < 4; ++c) run[c] = acc_add(run[c], v[c]);
            store4(dst + (int64_t)j * nt, run);
          }
        }
      }
    } else {
      const int l = sg.level;
      const TS *prev = static_cast<const TS *>(bm.buf[(l - 1) & 1]);
      const int r0 = rb * rows_per_item;
      const int r1 = min(bm.rows[l], r0 + rows_per_item);
      const RowOp *lop = ops + bm.ops_off[l];
      for (int r = r0; r < r1; ++r) {
        const RowOp op = lop[r];
        const TS *lrow = prev + (int64_t)op.lo * nt;
        const TS *hrow = prev + (int64_t)(op.hi < 0 ? op.lo : op.hi) * nt;
        for (int64_t t0 = t_begin + 4 * threadIdx.x; t0 < t_end; t0 += 4 * kBatchThreads) {
          A a[4], b[4], o[4];
          load4_cg(lrow + t0, a);
          if (op.hi < 0) {  // no upper sub-band: the row passes up unchanged
#pragma unroll
            for (int c = 0; c < 4; ++c) o[c] = a[c];
          } else {
            load4_shifted_cg(hrow, t0 - op.shift, nt, b);
#pragma unroll
            for (int c = 0; c < 4; ++c) o[c] = acc_add(a[c], b[c]);
          }
          if (l == bm.levels)
            store4(static_cast<TO *>(bm.out) + (int64_t)r * nt + t0, o);
          else
            store4(static_cast<TS *>(bm.buf[l & 1]) + (int64_t)r * nt + t0, o);
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(done + sg.beam * kMaxLevels + sg.level, 1);
    }
  }
}

size_t in_elem(int dtype) { return dtype == FDMT_U8_I32 ? 1 : 4; }
size_t st_elem(int dtype) { return dtype == FDMT_F32_F16STATE ? 2 : 4; }
int64_t rup(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

}  // namespace
}  // namespace fdmt

using fdmt::BeamDev;
using fdmt::Seg;

struct fdmt_batch_s {
  int32_t n = 0, dtype = 0;
  int device = -1;
  fdmt_batch_params prm{};
  std::vector<fdmt_beam_desc> desc;
  std::vector<fdmt::Tables> tabs;
  std::vector<BeamDev> beams;        // host template (pointers filled per call)
  std::vector<size_t> ws_off, ws_split;
  size_t ws_bytes = 0;
  std::vector<Seg> segs_all;         // full work list
  std::vector<Seg> segs;             // work list in use (after drop_level)
  int64_t total = 0;
  // device
  BeamDev *d_beams = nullptr;
  Seg *d_segs = nullptr;
  fdmt::InitOp *d_inits = nullptr;
  fdmt::RowOp *d_ops = nullptr;
  unsigned long long *d_counter = nullptr;
  int *d_done = nullptr;
  int *d_status = nullptr;
  int grid = 0;
  // recorded launch for one set of pointers
  std::vector<const void *> key;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  fdmt::FusedBatch *fused = nullptr;  // fused schedule (params->schedule == 1)
  // Launch schedule (params->schedule == 2): one plan per beam, its launches
  // spread over a few streams forked from the caller's stream.
  std::vector<fdmt_plan_t> plans;
  std::vector<size_t> plan_ws_off, plan_ws;
  std::vector<int> order;  // largest beam first
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> joined;
  cudaEvent_t forked = nullptr;
};

namespace {

constexpr int kLaunchStreams = 4;

void batch_release(fdmt_batch_s *b) {
  fdmt::fused_batch_destroy(b->fused);
  b->fused = nullptr;
  for (fdmt_plan_t p : b->plans) fdmt_destroy(p);
  b->plans.clear();
  for (cudaStream_t st : b->streams) cudaStreamDestroy(st);
  b->streams.clear();
  for (cudaEvent_t ev : b->joined) cudaEventDestroy(ev);
  b->joined.clear();
  if (b->forked) cudaEventDestroy(b->forked);
  b->forked = nullptr;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  void *ptrs[] = {b->d_beams, b->d_segs, b->d_inits, b->d_ops, b->d_counter, b->d_done, b->d_status};
  for (void *p : ptrs)
    if (p) cudaFree(p);
}

template <class T>
cudaError_t upload_vec(const std::vector<T> &v, T **dst) {
  *dst = nullptr;
  if (v.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(dst), v.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// Level-major work list over the beams, skipping (drop_beam, drop_level).
void build_segments(fdmt_batch_s *b, int drop_beam, int drop_level) {
  const int rpi = b->prm.rows_per_item, tile = b->prm.tile;
  int max_l = 0;
  for (const fdmt::Tables &t : b->tabs) max_l = std::max(max_l, t.levels);
  std::vector<std::vector<int32_t>> items(b->n, std::vector<int32_t>(fdmt::kMaxLevels, 0));
  for (int i = 0; i < b->n; ++i) {
    const fdmt::Tables &t = b->tabs[i];
    const int32_t tiles = (int32_t)((b->desc[i].nt + tile - 1) / tile);
    for (int l = 0; l <= t.levels; ++l) {
      const int32_t rows = l == 0 ? t.nf : t.level_rows[l];
      const int32_t per = l == 0 ? fdmt::kChannelsPerItem : rpi;
      items[i][l] = ((rows + per - 1) / per) * tiles;
    }
  }
  b->segs.clear();
  int64_t first = 0;
  for (int l = 0; l <= max_l; ++l)
    for (int i = 0; i < b->n; ++i) {
      const fdmt::Tables &t = b->tabs[i];
      if (l > t.levels || (i == drop_beam && l == drop_level)) continue;
      const int32_t tiles = (int32_t)((b->desc[i].nt + tile - 1) / tile);
      Seg s{};
      s.first = first;
      s.beam = i;
      s.level = l;
      s.tiles = tiles;
      s.rblocks = items[i][l] / tiles;
      s.need = l > 0 ? items[i][l - 1] : 0;
      b->segs.push_back(s);
      first += items[i][l];
    }
  b->total = first;
}

template <class TIn, class TS, class TO, class A>
void *kernel_ptr() {
  return reinterpret_cast<void *>(fdmt::batch_kernel<TIn, TS, TO, A>);
}

void *batch_kernel_for(int dtype) {
  switch (dtype) {
    case FDMT_U8_I32: return kernel_ptr<uint8_t, int32_t, int32_t, int32_t>();
    case FDMT_F32_F32: return kernel_ptr<float, float, float, float>();
    default: return kernel_ptr<float, __half, float, float>();
  }
}

cudaError_t launch_batch(fdmt_batch_s *b, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(b->d_done, 0, sizeof(int) * (size_t)b->n * fdmt::kMaxLevels, s);
  if (e != cudaSuccess) return e;
  const int nsegs = (int)b->segs.size();
  const uint64_t wait_ns = (uint64_t)b->prm.wait_ms * 1000000ull;
  void *args[] = {&b->d_beams, &b->d_segs, (void *)&nsegs, &b->total, &b->d_inits, &b->d_ops,
                  &b->d_counter, &b->d_done, &b->d_status, &b->prm.rows_per_item, &b->prm.tile,
                  (void *)&wait_ns};
  return cudaLaunchKernel(batch_kernel_for(b->dtype), dim3(b->grid), dim3(fdmt::kBatchThreads), args, 0, s);
}

}  // namespace

extern "C" {

int fdmt_plan_batch(int32_t n, const fdmt_beam_desc *beams, int32_t dtype, uint32_t flags,
                    const fdmt_batch_params *params, fdmt_batch_t *out) {
  if (out == nullptr) return FDMT_ERR_INVALID_ARG;
  *out = nullptr;
  if (n < 1 || beams == nullptr || flags != 0) return FDMT_ERR_INVALID_ARG;
  if (dtype != FDMT_U8_I32 && dtype != FDMT_F32_F32 && dtype != FDMT_F32_F16STATE) return FDMT_ERR_INVALID_ARG;
  fdmt_batch_s *b = new (std::nothrow) fdmt_batch_s();
  if (b == nullptr) return FDMT_ERR_NO_MEMORY;
  b->n = n;
  b->dtype = dtype;
  b->prm = fdmt_batch_params{16, 2048, 0, 2000, 0, 0, 0};
  if (params != nullptr) {
    if (params->rows_per_item < 0 || params->tile < 0 || params->tile % 1024 != 0 ||
        params->blocks_per_sm < 0 || params->wait_ms < 0 || params->schedule < 0 || params->schedule > 2 ||
        params->fused_tile < 0 || params->fused_tile % 64 != 0 || params->smem_budget < 0 ||
        params->smem_budget > 227 * 1024) {
      delete b;
      return FDMT_ERR_INVALID_ARG;
    }
    if (params->rows_per_item) b->prm.rows_per_item = params->rows_per_item;
    if (params->tile) b->prm.tile = params->tile;
    if (params->blocks_per_sm) b->prm.blocks_per_sm = params->blocks_per_sm;
    if (params->wait_ms) b->prm.wait_ms = params->wait_ms;
    b->prm.schedule = params->schedule;
    b->prm.fused_tile = params->fused_tile;
    b->prm.smem_budget = params->smem_budget;
  }
  b->desc.assign(beams, beams + n);
  b->tabs.resize(n);
  b->beams.resize(n);
  b->ws_off.resize(n);
  b->ws_split.resize(n);
  std::vector<fdmt::InitOp> inits;
  std::vector<fdmt::RowOp> ops;
  size_t ws = 0;
  for (int i = 0; i < n; ++i) {
    const fdmt_beam_desc &d = beams[i];
    if (!(d.f_min > 0.0) || !(d.f_max > d.f_min) || d.nd < 1 || d.nt < 1 || (int64_t)d.nd > d.nt ||
        (d.nt * (int64_t)fdmt::in_elem(dtype)) % 16 != 0 || (d.nt * (int64_t)fdmt::st_elem(dtype)) % 16 != 0) {
      delete b;
      return FDMT_ERR_INVALID_ARG;
    }
    const std::string err = fdmt::build_tables(d.f_min, d.f_max, d.nf, d.nd, b->tabs[i]);
    if (!err.empty()) {
      delete b;
      return err.rfind("unsupported", 0) == 0 ? FDMT_ERR_UNSUPPORTED : FDMT_ERR_INVALID_ARG;
    }
    const fdmt::Tables &t = b->tabs[i];
    if (t.levels + 1 > fdmt::kMaxLevels) {
      delete b;
      return FDMT_ERR_UNSUPPORTED;
    }
    BeamDev &bd = b->beams[i];
    std::memset(&bd, 0, sizeof(bd));
    bd.nt = d.nt;
    bd.nf = d.nf;
    bd.nd = d.nd;
    bd.levels = t.levels;
    bd.init_off = (int32_t)inits.size();
    inits.insert(inits.end(), t.init.begin(), t.init.end());
    const int64_t base = (int64_t)ops.size();
    for (int l = 1; l <= t.levels; ++l) bd.ops_off[l] = base + t.ops_begin[l];
    for (int l = 0; l <= t.levels; ++l) bd.rows[l] = t.level_rows[l];
    ops.insert(ops.end(), t.ops.begin(), t.ops.end());
    // Ping-pong buffers of this beam: even levels, odd levels (< L).
    size_t even = 0, odd = 0;
    for (int l = 0; l < t.levels; ++l) {
      const size_t bytes = (size_t)t.level_rows[l] * (size_t)d.nt * fdmt::st_elem(dtype);
      if (l & 1) odd = std::max(odd, bytes); else even = std::max(even, bytes);
    }
    b->ws_off[i] = ws;
    b->ws_split[i] = (size_t)fdmt::rup((int64_t)even, 256);
    ws += b->ws_split[i] + (size_t)fdmt::rup((int64_t)odd, 256);
  }
  b->ws_bytes = ws;
  build_segments(b, -1, -1);
  b->segs_all = b->segs;
  if (b->total >= ((int64_t)1 << 62)) {
    delete b;
    return FDMT_ERR_UNSUPPORTED;
  }
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    delete b;
    return FDMT_ERR_CUDA;
  }
  int per_sm = 0, sms = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel_for(dtype),
                                                                fdmt::kBatchThreads, 0);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    delete b;
    return FDMT_ERR_CUDA;
  }
  if (b->prm.blocks_per_sm > 0) per_sm = std::min(per_sm, b->prm.blocks_per_sm);
  b->grid = per_sm * sms;
  e = upload_vec(inits, &b->d_inits);
  if (e == cudaSuccess) e = upload_vec(ops, &b->d_ops);
  if (e == cudaSuccess) e = upload_vec(b->segs, &b->d_segs);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&b->d_beams), sizeof(BeamDev) * n);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&b->d_counter), sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&b->d_done), sizeof(int) * (size_t)n * fdmt::kMaxLevels);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&b->d_status), sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(int));
  if (e != cudaSuccess) {
    batch_release(b);
    delete b;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? FDMT_ERR_NO_MEMORY : FDMT_ERR_CUDA;
  }
  if (b->prm.schedule == 1) {
    const int st = fdmt::fused_batch_create(b->desc, b->tabs, dtype, b->prm, &b->fused);
    if (st != FDMT_OK) {
      batch_release(b);
      delete b;
      return st;
    }
  }
  if (b->prm.schedule == 2) {
    // One fused plan per beam, each with its own slice of the workspace so
    // beams can run concurrently.
    fdmt_schedule_params sp{};
    sp.tile = b->prm.fused_tile;
    sp.smem_budget = b->prm.smem_budget;
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
      const fdmt_beam_desc &d = b->desc[i];
      fdmt_plan_t p = nullptr;
      int st = fdmt_plan_ex(d.f_min, d.f_max, d.nf, d.nt, d.nd, dtype, FDMT_SCHED_FUSED,
                            (sp.tile || sp.smem_budget) ? &sp : nullptr, &p);
      size_t ws = 0;
      if (st == FDMT_OK) st = fdmt_workspace_bytes(p, &ws);
      if (st != FDMT_OK) {
        if (p) fdmt_destroy(p);
        batch_release(b);
        delete b;
        return st;
      }
      b->plans.push_back(p);
      b->plan_ws_off.push_back(off);
      b->plan_ws.push_back(ws);
      off += (size_t)fdmt::rup((int64_t)ws, 256);
      b->order.push_back(i);
    }
    b->ws_bytes = off;
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
      return b->desc[x].nt * (int64_t)b->desc[x].nd > b->desc[y].nt * (int64_t)b->desc[y].nd;
    });
    bool ok = cudaEventCreateWithFlags(&b->forked, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; k < kLaunchStreams && ok; ++k) {
      cudaStream_t st = nullptr;
      cudaEvent_t ev = nullptr;
      ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
      if (ok) b->streams.push_back(st);
      ok = ok && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
      if (ok) b->joined.push_back(ev);
    }
    if (!ok) {
      cudaGetLastError();
      batch_release(b);
      delete b;
      return FDMT_ERR_CUDA;
    }
  }
  *out = b;
  return FDMT_OK;
}

void fdmt_destroy_batch(fdmt_batch_t batch) {
  if (batch == nullptr) return;
  batch_release(batch);
  delete batch;
}

int fdmt_batch_workspace_bytes(fdmt_batch_t batch, size_t *bytes) {
  if (batch == nullptr || bytes == nullptr) return FDMT_ERR_INVALID_ARG;
  *bytes = batch->fused ? fdmt::fused_batch_workspace(batch->fused) : batch->ws_bytes;  // launches: ws_bytes
  return FDMT_OK;
}

int fdmt_batch_drop_level(fdmt_batch_t batch, int32_t beam, int32_t level) {
  if (batch == nullptr) return FDMT_ERR_INVALID_ARG;
  if (!batch->plans.empty()) return FDMT_ERR_UNSUPPORTED;  // launches have no work list
  if (batch->fused) return fdmt::fused_batch_drop(batch->fused, level == -1 ? -1 : beam, level);
  if (level == -1) {
    batch->segs = batch->segs_all;
    int64_t total = 0;
    for (const Seg &s : batch->segs) total = s.first + (int64_t)s.rblocks * s.tiles;
    batch->total = total;
  } else {
    if (beam < 0 || beam >= batch->n || level < 0 || level > batch->tabs[beam].levels)
      return FDMT_ERR_INVALID_ARG;
    build_segments(batch, beam, level);
  }
  if (batch->d_segs) cudaFree(batch->d_segs);
  batch->d_segs = nullptr;
  if (upload_vec(batch->segs, &batch->d_segs) != cudaSuccess) return cudaGetLastError(), FDMT_ERR_CUDA;
  batch->key.clear();  // the recorded launch refers to the old list
  return FDMT_OK;
}

int fdmt_batch_levels(fdmt_batch_t batch, int32_t beam, int32_t *groups, int32_t *bounds, int32_t *sizes,
                      int32_t n) {
  if (batch == nullptr || groups == nullptr || beam < 0 || beam >= batch->n) return FDMT_ERR_INVALID_ARG;
  std::vector<int32_t> v, z;
  int32_t fused_groups = 0, fused_tile = 0;
  if (!batch->plans.empty() &&
      fdmt_schedule_info(batch->plans[beam], &fused_groups, nullptr, 0, &fused_tile) == FDMT_OK && fused_groups > 0) {
    // The beam's own fused plan: bounds and stored sizes of its launches.
    int64_t cnt = 0;
    fdmt_fused_tables(batch->plans[beam], 0, nullptr, 0, &cnt);
    std::vector<int32_t> tab((size_t)cnt);
    fdmt_fused_tables(batch->plans[beam], 0, tab.data(), cnt, &cnt);
    for (int64_t g = 0; g < cnt / 16; ++g) {
      if (g == 0) {
        v.push_back(tab[0]);
        z.push_back(tab[14]);
      }
      v.push_back(tab[16 * g + 1]);
      z.push_back(tab[16 * g + 15]);
    }
  } else if (batch->fused) {
    v = fdmt::fused_batch_bounds(batch->fused, beam);
    z = fdmt::fused_batch_sizes(batch->fused, beam);
  } else {
    v.push_back(0);
    for (int l = 0; l <= batch->tabs[beam].levels; ++l) v.push_back(l);
    z.assign(v.size(), (int32_t)fdmt::st_elem(batch->dtype));
    z[0] = (int32_t)fdmt::in_elem(batch->dtype);
    z.back() = 4;
  }
  *groups = (int32_t)v.size() - 1;
  if ((bounds != nullptr || sizes != nullptr) && n < (int32_t)v.size()) return FDMT_ERR_INVALID_ARG;
  if (bounds != nullptr) std::copy(v.begin(), v.end(), bounds);
  if (sizes != nullptr) std::copy(z.begin(), z.end(), sizes);
  return FDMT_OK;
}

int fdmt_execute_batch(fdmt_batch_t batch, const void *const *in, void *const *out, void *workspace,
                       size_t ws_bytes, void *stream) {
  if (batch == nullptr || in == nullptr || out == nullptr) return FDMT_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return cudaGetLastError(), FDMT_ERR_CUDA;
  if (dev != batch->device) return FDMT_ERR_INVALID_ARG;
  const size_t need = batch->fused ? fdmt::fused_batch_workspace(batch->fused) : batch->ws_bytes;
  if (need > 0 && (workspace == nullptr || ws_bytes < need)) return FDMT_ERR_WORKSPACE;
  if (workspace != nullptr && (reinterpret_cast<uintptr_t>(workspace) % 256) != 0) return FDMT_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<const void *> key;
  key.push_back(workspace);
  for (int i = 0; i < batch->n; ++i) {
    if (in[i] == nullptr || out[i] == nullptr || (reinterpret_cast<uintptr_t>(in[i]) & 15u) ||
        (reinterpret_cast<uintptr_t>(out[i]) & 15u))
      return FDMT_ERR_INVALID_ARG;
    key.push_back(in[i]);
    key.push_back(out[i]);
  }
  if (batch->fused) return fdmt::fused_batch_execute(batch->fused, in, out, workspace, s);
  if (!batch->plans.empty()) {
    // Fork: every stream waits for the caller's stream; beams largest first,
    // round robin over the streams; join: the caller's stream waits for all.
    cudaError_t e = cudaEventRecord(batch->forked, s);
    for (cudaStream_t st : batch->streams)
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, batch->forked, 0);
    if (e != cudaSuccess) return cudaGetLastError(), FDMT_ERR_CUDA;
    for (size_t j = 0; j < batch->order.size(); ++j) {
      const int i = batch->order[j];
      const int st = fdmt_execute(batch->plans[i], in[i], nullptr, out[i],
                                  static_cast<char *>(workspace) + batch->plan_ws_off[i], batch->plan_ws[i],
                                  batch->streams[j % batch->streams.size()]);
      if (st != FDMT_OK) return st;
    }
    for (size_t k = 0; k < batch->streams.size() && e == cudaSuccess; ++k) {
      e = cudaEventRecord(batch->joined[k], batch->streams[k]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, batch->joined[k], 0);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cudaGetLastError(), FDMT_ERR_CUDA;
    return FDMT_OK;
  }
  cudaError_t e = cudaSuccess;
  if (key != batch->key || batch->exec == nullptr) {
    // New pointers: write the per-beam pointers, then record the launch.
    for (int i = 0; i < batch->n; ++i) {
      BeamDev &bd = batch->beams[i];
      bd.in = in[i];
      bd.out = out[i];
      char *w = static_cast<char *>(workspace) + batch->ws_off[i];
      bd.buf[0] = w;
      bd.buf[1] = w + batch->ws_split[i];
    }
    e = cudaMemcpyAsync(batch->d_beams, batch->beams.data(), sizeof(BeamDev) * batch->n,
                        cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (batch->exec) cudaGraphExecDestroy(batch->exec);
    if (batch->graph) cudaGraphDestroy(batch->graph);
    batch->exec = nullptr;
    batch->graph = nullptr;
    cudaStream_t cap = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t le = launch_batch(batch, cap);
      e = cudaStreamEndCapture(cap, &batch->graph);
      if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&batch->exec, batch->graph, 0);
    if (cap) cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
      cudaGetLastError();
      batch->key.clear();
      return FDMT_ERR_CUDA;
    }
    batch->key = key;
  }
  int status = 0;
  e = cudaGraphLaunch(batch->exec, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, batch->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cudaGetLastError(), FDMT_ERR_CUDA;
  if (status != 0) {
    const int zero = 0;
    if (cudaMemcpy(batch->d_status, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
      return cudaGetLastError(), FDMT_ERR_CUDA;
    return FDMT_ERR_TIMEOUT;
  }
  return FDMT_OK;
}

}  // extern "C"
