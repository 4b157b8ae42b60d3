// Fused-schedule kernel of the FDMT (cones of several merge levels per
// launch; planner in fdmt_fused_plan.cpp, layout in fdmt_fused.h).
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
template <class TI, class TB, class TO, class A, bool FROM_INPUT, bool R16, bool SEARCH>
__global__ void __launch_bounds__(kFusedThreads, SEARCH ? 2 : kFusedMinBlocks)
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
    item_first_stage<TI, TB, A, TO, R16, FROM_INPUT, SEARCH>(bar, stages, cur, walks, ops, w, warp, lane, out, nt,
                                                             T0, lim, ds, next < items ? &tp_next : nullptr);
    __syncthreads();  // S is no longer read: stage the next item into it
    if (next < items) {
      if (warp == 0) stage_item<TS>(smem, bar, maps.m, tp_next, loads, ld_next, T0_next, box, cshift, lane);
      tp = tp_next;
      advance();
      if (next + gridDim.x < items) tp_next = tpls[tpl];
      T0_cur = T0_next;
    }
    item_later_stages<A, TO, R16, SEARCH>(bar, stages, cur, ops, walks, warp, lane, out, nt, T0, lim, T0 / W, sa, ds,
                                          next < items ? &tp : nullptr);
    __syncthreads();  // Pa / Pb are reused by the next item
  }
}

// ---------------------------------------------------------------------------
// Host side: tensor maps and launches.

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Row-window map over a [rows][nt] matrix: boxes of `box` columns x 1 row.
bool make_map(CUtensorMap *m, const void *base, CUtensorMapDataType type, uint32_t elem,
              uint64_t rows, uint64_t nt, uint32_t box) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (fn == nullptr) return false;
  cuuint64_t dims[2] = {nt, rows};
  cuuint64_t strides[1] = {nt * elem};
  cuuint32_t boxd[2] = {box, 1};
  cuuint32_t es[2] = {1, 1};
  return fn(m, type, 2, const_cast<void *>(base), dims, strides, boxd, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Row-block map over a [rows][nt] matrix viewed as [rows][nt / chunk][chunk]
// (nt a multiple of chunk): boxes of chunk x kchunks x brows elements.
bool make_block_map(CUtensorMap *m, const void *base, CUtensorMapDataType type, uint32_t elem, uint64_t rows,
                    uint64_t nt, uint32_t chunk, uint32_t kchunks, uint32_t brows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (fn == nullptr) return false;
  cuuint64_t dims[3] = {chunk, nt / chunk, rows};
  cuuint64_t strides[2] = {(cuuint64_t)chunk * elem, nt * elem};
  cuuint32_t boxd[3] = {chunk, kchunks, brows};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(m, type, 3, const_cast<void *>(base), dims, strides, boxd, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool make_group_maps(CUtensorMap *maps, const FusedGroup &g, const void *base, CUtensorMapDataType type,
                     uint32_t elem, uint64_t rows, uint64_t nt, int32_t *cshift) {
  std::memset(maps, 0, sizeof(CUtensorMap) * (kMaxBlockP + 1));
  *cshift = 0;
  if (g.chunk > 0) {
    while ((1 << *cshift) < g.chunk) ++*cshift;
    for (int p = 0; p <= g.max_p && p <= kMaxBlockP; ++p)
      if (!make_block_map(&maps[p], base, type, elem, rows, nt, (uint32_t)g.chunk, (uint32_t)g.kchunks, 1u << p))
        return false;
    return true;
  }
  return make_map(&maps[0], base, type, elem, rows, nt, (uint32_t)g.box);
}

namespace {

template <class TI, class TB, class TO, class A, bool FI, bool R16, bool SEARCH = false>
cudaError_t launch_group(const DeviceTables &dt, const FusedGroup &g, const void *base, int64_t base_rows,
                         void *dst, const float *w, int64_t nt, cudaStream_t s, const SearchArgs *sa = nullptr) {
  auto kern = fused_kernel<TI, TB, TO, A, FI, R16, SEARCH>;
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

// uint8 input: launch-boundary states are int32 or, where the sums fit,
// uint16 (the group's in_size / out_size).
cudaError_t run_fused_u8(const DeviceTables &dt, const void *in, void *out, void *const bufs[2], int64_t nt,
                         cudaStream_t s, const SearchArgs *sa) {
  const FusedPlan &fp = *dt.fused;
  const int G = (int)fp.groups.size();
  for (int g = 0; g < G; ++g) {
    const FusedGroup &gr = fp.groups[g];
    void *dst = (g == G - 1) ? out : bufs[g & 1];
    const bool o16 = gr.out_size == 2, i16 = gr.in_size == 2;
    cudaError_t e;
    if (g == G - 1 && gr.search_k > 0) {
      if (sa == nullptr) return cudaErrorInvalidValue;
      if (gr.from_input) {
        e = launch_group<uint8_t, int32_t, int32_t, int32_t, true, false, true>(dt, gr, in, dt.nf, dst, nullptr,
                                                                                nt, s, sa);
      } else {
        const void *base = bufs[(g - 1) & 1];
        const int64_t rows = dt.level_rows[gr.lb];
        e = i16 ? launch_group<uint8_t, uint16_t, int32_t, int32_t, false, false, true>(dt, gr, base, rows, dst,
                                                                                        nullptr, nt, s, sa)
                : launch_group<uint8_t, int32_t, int32_t, int32_t, false, false, true>(dt, gr, base, rows, dst,
                                                                                       nullptr, nt, s, sa);
      }
    } else if (gr.from_input) {
      e = o16 ? launch_group<uint8_t, int32_t, uint16_t, int32_t, true, false>(dt, gr, in, dt.nf, dst, nullptr, nt, s)
              : launch_group<uint8_t, int32_t, int32_t, int32_t, true, false>(dt, gr, in, dt.nf, dst, nullptr, nt, s);
    } else {
      const void *base = bufs[(g - 1) & 1];
      const int64_t rows = dt.level_rows[gr.lb];
      if (i16 && o16)
        e = launch_group<uint8_t, uint16_t, uint16_t, int32_t, false, false>(dt, gr, base, rows, dst, nullptr, nt, s);
      else if (i16)
        e = launch_group<uint8_t, uint16_t, int32_t, int32_t, false, false>(dt, gr, base, rows, dst, nullptr, nt, s);
      else if (!o16)
        e = launch_group<uint8_t, int32_t, int32_t, int32_t, false, false>(dt, gr, base, rows, dst, nullptr, nt, s);
      else
        e = cudaErrorInvalidValue;  // sizes only grow with the level
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t run_fused(const DeviceTables &dt, int dtype, const void *in, const float *w, void *out,
                      void *const bufs[2], int64_t nt, cudaStream_t s, const SearchArgs *sa) {
  if (dt.fused == nullptr) return cudaErrorInvalidValue;
  switch (dtype) {
    case 0: return run_fused_u8(dt, in, out, bufs, nt, s, sa);
    case 1: return run_fused_typed<float, float, float, float, false>(dt, in, w, out, bufs, nt, s, sa);
    case 2: return run_fused_typed<float, __half, float, float, true>(dt, in, w, out, bufs, nt, s, sa);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fdmt
