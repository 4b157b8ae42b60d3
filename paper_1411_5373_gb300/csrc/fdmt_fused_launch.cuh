// Fused-schedule kernel and its launch (shared by the translation units that
// instantiate it: fdmt_fused_f32.cu for float32, fdmt_fused.cu for fp16
// state, fdmt_fused_u8.cu for uint8).  The schedule: fdmt_fused.h; the planner: fdmt_fused_plan.cpp.
//
// One block computes one cone for one time tile:
//   1. warp 0 issues TMA copies of the cone's base rows (or input channels)
//      into shared memory; out-of-range columns arrive as zeros, which is
//      the paper's copy rule for t < 0;
//   2. all threads wait on the mbarrier (bounded: on timeout the block sets
//      the plan's status word and returns instead of hanging);
//   3. the stages run: a cone that starts at the input walks level 1
//      straight from the staged samples (the Option-1 partial sums of
//      section 4 are running sums in registers); the other levels are
//      computed one (single) or two (pair) at a time, the level between the
//      two of a pair never stored; each warp runs its own list of row
//      pieces, lanes over time (conflict-free: consecutive lanes touch
//      consecutive words);
//   4. the group's top level is written to global memory, coalesced.

#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "fdmt_fused.h"
#include "fdmt_fused_dev.cuh"
#include "fdmt_internal.h"
#include "fdmt_tma.h"

namespace fdmt {

// Persistent blocks: block b handles items b, b + gridDim.x, ... where item
// = template * ntiles + tile.  Per item: wait for its staged rows, run the
// first stage (level 1 walked from the staged input, or the first single /
// pair stage over the staged base rows), stage the next item into S, run
// the remaining stages in Pa / Pb; the last writes global memory.  The next
// item's template and first copy descriptors are read while the current
// item computes.
// A launch that ends with the search keeps 32 sums per thread in flight in
// its search stage: it is compiled for two resident blocks per SM (more
// registers per thread).
// GEN: the plan holds stages with passed-up or one-term halves (Nf not a
// power of two); SCALE: channel weights multiply the input.  Each launch
// takes the variant it needs, so a kernel carries only its own stage code.
// MINB: the resident blocks per SM the register budget is set for.
template <class TI, class TB, class TO, class A, bool FROM_INPUT, bool R16, bool SEARCH, bool GEN, bool SCALE,
          int MINB = kFusedMinBlocks>
__global__ void __launch_bounds__(kFusedThreads, SEARCH ? 2 : MINB)
fused_kernel(const __grid_constant__ TmaMaps maps, TO *__restrict__ out, int64_t nt, int32_t W,
             int64_t ntiles, int64_t items, const FusedTemplate *__restrict__ tpls,
             const FusedLoad *__restrict__ loads, const FusedWalk *__restrict__ walks,
             const FusedOp *__restrict__ ops, const int32_t *__restrict__ stages,
             const float *__restrict__ w, int32_t box, int32_t cshift, int *__restrict__ status,
             const SearchArgs sa) {
  using TS = typename std::conditional<FROM_INPUT, TI, TB>::type;  // staged element type
  extern __shared__ __align__(128) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t bar = smem_u32(smem);

  int64_t item = blockIdx.x;
  if (item >= items) return;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  // item = tpl * ntiles + tile, advanced by gridDim.x without divisions.
  int64_t tile = (int64_t)blockIdx.x % ntiles, tpl = (int64_t)blockIdx.x / ntiles;
  const int64_t step_tile = (int64_t)gridDim.x % ntiles, step_tpl = (int64_t)gridDim.x / ntiles;
  auto advance = [&]() {
    tile += step_tile;
    tpl += step_tpl;
    if (tile >= ntiles) {
      tile -= ntiles;
      ++tpl;
    }
  };
  FusedTemplate tp = tpls[tpl];
  __syncthreads();
  int64_t T0_cur = tile * (int64_t)W;
  if (warp == 0) stage_item<TS>(smem, bar, maps.m, tp, loads, fetch_load(tp, loads, lane), T0_cur, box, cshift, lane);
  advance();  // (tpl, tile) of the next item from here on
  FusedTemplate tp_next = FusedTemplate{0, 0, 0, 0, 0, 0, 0, 0};
  if (item + gridDim.x < items) tp_next = tpls[tpl];
  DescStream ds;
  ds.slot = desc_slot(bar, tp, warp);
  ds_peek(ds, stages, &tp, 0, warp);
  uint32_t phase = 0;
  for (; item < items; item += gridDim.x) {
    const FusedTemplate cur = tp;
    const int64_t T0 = T0_cur;
    const int64_t next = item + gridDim.x;
    const int64_t T0_next = tile * (int64_t)W;
    FusedLoad ld_next = FusedLoad{0, 0, 0, 0};
    if (warp == 0 && next < items) ld_next = fetch_load(tp_next, loads, lane);
    if (!mbar_wait_bounded(bar, phase)) {
      // The copies did not complete in time: report it, give in-flight
      // copies one more bounded wait so none lands after the block exits.
      atomicExch(status, 1);
      mbar_wait_bounded(bar, phase);
      return;
    }
    phase ^= 1u;
    const int lim = (int)((nt - T0) < (int64_t)W ? (nt - T0) : (int64_t)W);
    item_first_stage<TI, TB, A, TO, R16, FROM_INPUT, SEARCH, GEN, SCALE>(
        bar, stages, cur, walks, ops, w, warp, lane, out, nt, T0, lim, ds, next < items ? &tp_next : nullptr);
    __syncthreads();  // S is no longer read: stage the next item into it
    if (next < items) {
      if (warp == 0) stage_item<TS>(smem, bar, maps.m, tp_next, loads, ld_next, T0_next, box, cshift, lane);
      tp = tp_next;
      advance();
      if (next + gridDim.x < items) tp_next = tpls[tpl];
      T0_cur = T0_next;
    }
    item_later_stages<A, TO, R16, SEARCH, GEN>(bar, stages, cur, ops, walks, warp, lane, out, nt, T0, lim, T0 / W,
                                               sa, ds, next < items ? &tp : nullptr);
    __syncthreads();  // Pa / Pb are reused by the next item
  }
}

namespace {

template <class TI, class TB, class TO, class A, bool FI, bool R16, bool SEARCH, bool GEN, bool SCALE,
          int MINB = kFusedMinBlocks>
cudaError_t launch_variant(const DeviceTables &dt, const FusedGroup &g, const void *base, int64_t base_rows,
                           void *dst, const float *w, int64_t nt, cudaStream_t s, const SearchArgs *sa) {
  auto kern = fused_kernel<TI, TB, TO, A, FI, R16, SEARCH, GEN, SCALE, MINB>;
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [&] {
    attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  });
  if (attr_err != cudaSuccess) return attr_err;
  using TS = typename std::conditional<FI, TI, TB>::type;
  TmaMaps maps;
  int32_t cshift = 0;
  if (!make_group_maps(maps.m, g, base, map_type<TS>(), sizeof(TS), (uint64_t)base_rows, (uint64_t)nt, &cshift))
    return cudaErrorInvalidValue;
  const int32_t box = g.box;
  const int64_t items = (int64_t)g.tpl_count * g.ntiles;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kFusedThreads, g.smem_bytes);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int64_t blocks = std::min<int64_t>(items, (int64_t)per_sm * sms);
  dt.prof->begin(s, FI ? K_FUSED_LOCAL : K_FUSED_CONE, g.lb * 100 + g.lt);
  kern<<<(unsigned)blocks, kFusedThreads, g.smem_bytes, s>>>(
      maps, static_cast<TO *>(dst), nt, g.W, g.ntiles, items, dt.f_tpls + g.tpl_begin, dt.f_loads,
      dt.f_walks, dt.f_ops, dt.f_stages, w, box, cshift, dt.status, sa ? *sa : SearchArgs{});
  dt.prof->end(s);
  return cudaGetLastError();
}

// The variant with or without pass-through stage code (GEN) and weights.
template <class TI, class TB, class TO, class A, bool FI, bool R16, bool SEARCH, int MINB>
cudaError_t launch_gen_scale(const DeviceTables &dt, const FusedGroup &g, const void *base, int64_t base_rows,
                             void *dst, const float *w, int64_t nt, cudaStream_t s, const SearchArgs *sa) {
  const bool gen = dt.fused->general;
  if constexpr (FI && std::is_floating_point<A>::value) {
    if (w != nullptr)
      return gen ? launch_variant<TI, TB, TO, A, FI, R16, SEARCH, true, true, MINB>(dt, g, base, base_rows, dst, w,
                                                                                    nt, s, sa)
                 : launch_variant<TI, TB, TO, A, FI, R16, SEARCH, false, true, MINB>(dt, g, base, base_rows, dst, w,
                                                                                     nt, s, sa);
  }
  return gen ? launch_variant<TI, TB, TO, A, FI, R16, SEARCH, true, false, MINB>(dt, g, base, base_rows, dst, w, nt,
                                                                                 s, sa)
             : launch_variant<TI, TB, TO, A, FI, R16, SEARCH, false, false, MINB>(dt, g, base, base_rows, dst, w, nt,
                                                                                  s, sa);
}

// The launch of one group, with the kernel variant the plan and the
// arguments need (weights only for float input from the input).  Float32
// sums whose shared memory leaves room for at most two blocks per SM take
// the variant compiled for two (more registers per thread: measured faster
// there; for integer and fp16-state sums it measured slower).
template <class TI, class TB, class TO, class A, bool FI, bool R16, bool SEARCH = false>
cudaError_t launch_group(const DeviceTables &dt, const FusedGroup &g, const void *base, int64_t base_rows,
                         void *dst, const float *w, int64_t nt, cudaStream_t s, const SearchArgs *sa = nullptr) {
  if constexpr (std::is_same<A, float>::value && !R16 && !SEARCH && kFusedMinBlocks > 2) {
    // blocks per SM that the shared memory admits
    int dev = 0, smem_sm = 0, reserved = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e != cudaSuccess) return e;
    if (smem_sm / (g.smem_bytes + reserved) <= 2)
      return launch_gen_scale<TI, TB, TO, A, FI, R16, SEARCH, 2>(dt, g, base, base_rows, dst, w, nt, s, sa);
  }
  return launch_gen_scale<TI, TB, TO, A, FI, R16, SEARCH, kFusedMinBlocks>(dt, g, base, base_rows, dst, w, nt, s,
                                                                           sa);
}

// The launches of a float plan (A the sums' type, R16: fp16-state rounding).
template <class TI, class TB, class TO, class A, bool R16>
cudaError_t run_fused_typed(const DeviceTables &dt, const void *in, const float *w, void *out,
                            void *const bufs[2], int64_t nt, cudaStream_t s, const SearchArgs *sa) {
  const FusedPlan &fp = *dt.fused;
  const int G = (int)fp.groups.size();
  for (int g = 0; g < G; ++g) {
    const FusedGroup &gr = fp.groups[g];
    const bool last = (g == G - 1);
    void *dst = last ? out : bufs[g & 1];
    cudaError_t e;
    if (last && gr.search_k > 0) {
      // The last launch ends with the boxcar search (a search needs at
      // least two merge levels, so a launch from the input walks level 1
      // into Pa before its top level goes to Pt).
      if (sa == nullptr) return cudaErrorInvalidValue;
      e = gr.from_input ? launch_group<TI, TB, TO, A, true, R16, true>(dt, gr, in, dt.nf, dst, w, nt, s, sa)
                        : launch_group<TI, TB, TO, A, false, R16, true>(dt, gr, bufs[(g - 1) & 1],
                                                                        dt.level_rows[gr.lb], dst, w, nt, s, sa);
    } else if (gr.from_input) {
      e = last ? launch_group<TI, TB, TO, A, true, R16>(dt, gr, in, dt.nf, dst, w, nt, s)
               : launch_group<TI, TB, TB, A, true, R16>(dt, gr, in, dt.nf, dst, w, nt, s);
    } else {
      const void *base = bufs[(g - 1) & 1];
      const int64_t rows = dt.level_rows[gr.lb];
      e = last ? launch_group<TI, TB, TO, A, false, R16>(dt, gr, base, rows, dst, w, nt, s)
               : launch_group<TI, TB, TB, A, false, R16>(dt, gr, base, rows, dst, w, nt, s);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

// uint8 input (fdmt_fused_u8.cu).
cudaError_t run_fused_u8(const DeviceTables &dt, const void *in, void *out, void *const bufs[2], int64_t nt,
                         cudaStream_t s, const SearchArgs *sa);
// float32 input and state (fdmt_fused_f32.cu).
cudaError_t run_fused_f32(const DeviceTables &dt, const void *in, const float *w, void *out, void *const bufs[2],
                          int64_t nt, cudaStream_t s, const SearchArgs *sa);

}  // namespace fdmt
