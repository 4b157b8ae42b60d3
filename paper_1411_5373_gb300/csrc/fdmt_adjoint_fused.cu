// Fused-schedule kernel of the FDMT adjoint (pull cones of several
// transposed levels per launch; planner in fdmt_adjoint_plan.cpp, layout in
// fdmt_adjoint_fused.h).
//
// One block computes one cone for one time tile, persistent over items as
// the forward cone kernel: warp 0 stages the cone's level-lt gradient rows
// by TMA (zeros past Nt), every thread waits on the mbarrier (bounded: on
// timeout the block sets the plan's status word and returns), then the
// stages run level by level, each child row summing its run of parent rows
// in increasing row order; the last stage writes the owned level-lb rows,
// or the input gradient (the Option-1 transpose) in the launch that ends at
// level 0.  The next item's copies go out as soon as the first stage has
// read the staged rows.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "fdmt_adjoint_fused.h"
#include "fdmt_fused_dev.cuh"
#include "fdmt_internal.h"
#include "fdmt_tma.h"

namespace fdmt {

namespace {

// out_row[t] for t = t0 + lane + 32 k: written where the piece column is
// below `width` and 0 <= t < nt (bands tile time with their own offset, so
// t0 may be negative).
__device__ __forceinline__ void adj_store_global(float *__restrict__ out_row, int64_t t0,
                                                 const float (&v)[kLaneCols], int width, int64_t nt, int lane) {
  if (width == kPieceCols && t0 >= 0 && t0 + kPieceCols <= nt) {  // a whole piece inside [0, nt)
    float *p = out_row + t0 + lane;
#pragma unroll
    for (int k = 0; k < kLaneCols; ++k) p[32 * k] = v[k];
    return;
  }
#pragma unroll
  for (int k = 0; k < kLaneCols; ++k) {
    const int tau = lane + 32 * k;
    const int64_t t = t0 + tau;
    const bool ok = tau < width && t >= 0 && t < nt;
    stg_if(out_row + (ok ? t : 0), v[k], ok);
  }
}

// The ops of a stage two at a time, body(a, b, two) (b = a when the stage
// has an odd op left), so that each warp keeps the loads of two ops in
// flight.  Descriptor chunks as in for_ops.
template <class F>
__device__ __forceinline__ void for_op_pairs(const FusedOp *__restrict__ ops, int i0, int i1, DescStream &ds,
                                             int lane, F &&body) {
  const int4 *src = reinterpret_cast<const int4 *>(ops);
  int4 q = ds.q;
  if (!ds.ready) q = (2 * i0 + lane < 2 * i1) ? __ldg(src + 2 * i0 + lane) : make_int4(0, 0, 0, 0);
  ds.ready = false;
  for (int base = i0; base < i1; base += kDescChunk) {
    __syncwarp();  // every lane is done with the previous chunk
    sts_v4(ds.slot + 16u * (uint32_t)lane, q);
    __syncwarp();
    const int nb = base + kDescChunk;
    if (nb < i1) {
      if (2 * nb + lane < 2 * i1) q = __ldg(src + 2 * nb + lane);
    } else {
      ds_load_first(ds, ops, nullptr, lane);
    }
    const int n = min(kDescChunk, i1 - base);
    for (int k = 0; k < n; k += 2) {
      const bool two = k + 1 < n;
      const uint32_t sa = ds.slot + 32u * (uint32_t)k, sb = two ? sa + 32u : sa;
      const int4 a0 = lds_v4(sa), a1 = lds_v4(sa + 16u), b0 = lds_v4(sb), b1 = lds_v4(sb + 16u);
      body(FusedOp{a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w},
           FusedOp{b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w}, two);
    }
  }
  if (i0 >= i1) ds_load_first(ds, ops, nullptr, lane);
}

// One transposed level: each op sums its run of p2 parent rows (stride p1
// bytes; the upper half's stride includes the one-column shift per row).
template <int OUT>
__device__ __forceinline__ void adj_gather_stage(uint32_t sbase, const FusedOp *__restrict__ ops, int i0, int i1,
                                                 DescStream &ds, int lane, float *__restrict__ out, int64_t nt,
                                                 int64_t T0) {
  for_ops(ops, nullptr, i0, i1, ds, lane, [&](const FusedOp &op) {
    // the sum starts from the first row of the run and adds the others in
    // row order; runs of one to three rows (nearly all) are straight-line
    float v[kLaneCols];
    const uint32_t a0 = sbase + (uint32_t)op.p0;
    const uint32_t step = (uint32_t)op.p1;
    ld_piece<float, float>(v, a0, lane);
    if (op.p2 == 2) {
      float x[kLaneCols];
      ld_piece<float, float>(x, a0 + step, lane);
#pragma unroll
      for (int k = 0; k < kLaneCols; ++k) v[k] = __fadd_rn(v[k], x[k]);
    } else if (op.p2 == 3) {
      float x[kLaneCols], y[kLaneCols];
      ld_piece<float, float>(x, a0 + step, lane);
      ld_piece<float, float>(y, a0 + 2 * step, lane);
#pragma unroll
      for (int k = 0; k < kLaneCols; ++k) v[k] = __fadd_rn(__fadd_rn(v[k], x[k]), y[k]);
    } else if (op.p2 > 3) {
      uint32_t a = a0 + step;
      for (int j = 1; j < op.p2; ++j, a += step) {
        float x[kLaneCols];
        ld_piece<float, float>(x, a, lane);
#pragma unroll
        for (int k = 0; k < kLaneCols; ++k) v[k] = __fadd_rn(v[k], x[k]);
      }
    }
    if constexpr (OUT == kOutSmem)
      st_piece_smem<float, false>(sbase + (uint32_t)op.dst, v, op.width, lane);
    else
      adj_store_global(out + (int64_t)op.dst * nt, T0 + op.col, v, op.width, nt, lane);
  });
}

// Transpose of the Option-1 initialisation for one channel:
//   g_in[tau] = sum_{j < rows} sum_{i <= j} g0[j][tau + i]
// (j outer, i inner), scaled by the channel weight when w is given.  With
// `part`, each op also writes its piece's share of the weight gradient,
// sum_tau x[k][t] g_in[tau] (unscaled), summed in a fixed order: per lane
// over its columns, then a butterfly over the lanes; slot (channel, tile,
// piece).
__device__ __forceinline__ void adj_init_load_x(float (&xv)[kLaneCols], const FusedOp &op,
                                                const float *__restrict__ x, int64_t nt, int64_t T0, int lane) {
  const float *xrow = x + (int64_t)op.dst * nt;
  const int64_t t0 = T0 + op.col;
#pragma unroll
  for (int k = 0; k < kLaneCols; ++k) {
    const int tau = lane + 32 * k;
    const int64_t t = t0 + tau;
    xv[k] = (tau < op.width && t >= 0 && t < nt) ? __ldg(xrow + t) : 0.f;
  }
}

// FOLD: the op is kAdjInitF (level-0 values re-formed from level-1 runs).
template <bool FOLD>
__device__ __forceinline__ void adj_init_op(uint32_t sbase, const FusedOp &op, const float (&xv)[kLaneCols],
                                            int lane, float *__restrict__ out, int64_t nt, int64_t T0,
                                            const float *__restrict__ w, float *__restrict__ part,
                                            int64_t part_row) {
  // (j, i) = (0, 0) first, then the other terms in order
  float v[kLaneCols];
  if constexpr (FOLD) {
    // term (j, i) is level-0 row j at column tau + i: its run of level-1
    // rows summed in row order, as the gather would have stored it
    uint32_t pj = sbase + (uint32_t)op.p0;
    const uint32_t step = (uint32_t)op.p1, back = 4u * (uint32_t)(op.flags & 1);
    uint32_t runs = (uint32_t)op.flags >> 1;
    for (int j = 0; j < op.p2; ++j, runs >>= 4) {
      const int cnt = (int)(runs & 15u);
      for (int ii = 0; ii <= j; ++ii) {
        float r[kLaneCols];
        const uint32_t a = pj + 4u * (uint32_t)ii;
        ld_piece<float, float>(r, a, lane);
        for (int q = 1; q < cnt; ++q) {
          float y[kLaneCols];
          ld_piece<float, float>(y, a + (uint32_t)q * step, lane);
#pragma unroll
          for (int k = 0; k < kLaneCols; ++k) r[k] = __fadd_rn(r[k], y[k]);
        }
        if (j == 0) {
#pragma unroll
          for (int k = 0; k < kLaneCols; ++k) v[k] = r[k];
        } else {
#pragma unroll
          for (int k = 0; k < kLaneCols; ++k) v[k] = __fadd_rn(v[k], r[k]);
        }
      }
      pj += (uint32_t)cnt * step - back;
    }
  } else {
    ld_piece<float, float>(v, sbase + (uint32_t)op.p0, lane);
    for (int j = 1; j < op.p2; ++j) {
      const uint32_t row = sbase + (uint32_t)op.p0 + (uint32_t)(j * op.p1);
      for (int ii = 0; ii <= j; ++ii) {
        float y[kLaneCols];
        ld_piece<float, float>(y, row + (uint32_t)(4 * ii), lane);
#pragma unroll
        for (int k = 0; k < kLaneCols; ++k) v[k] = __fadd_rn(v[k], y[k]);
      }
    }
  }
  if (part != nullptr) {
    const int64_t t0 = T0 + op.col;
    float d = 0.f;
#pragma unroll
    for (int k = 0; k < kLaneCols; ++k) {
      const int tau = lane + 32 * k;
      const int64_t t = t0 + tau;
      const bool ok = tau < op.width && t >= 0 && t < nt;
      d = __fadd_rn(d, ok ? __fmul_rn(xv[k], v[k]) : 0.f);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) d = __fadd_rn(d, __shfl_xor_sync(0xffffffffu, d, off));
    if (lane == 0) part[(int64_t)op.dst * part_row + op.p3] = d;
  }
  if (w != nullptr) {
    const float wk = __ldg(w + op.dst);
#pragma unroll
    for (int k = 0; k < kLaneCols; ++k) v[k] = __fmul_rn(v[k], wk);
  }
  adj_store_global(out + (int64_t)op.dst * nt, T0 + op.col, v, op.width, nt, lane);
}

// The init stage takes its ops two at a time: the input samples of both
// (for the weight gradient) are requested before either op's sums, so the
// two loads' latencies overlap.
template <bool FOLD>
__device__ __forceinline__ void adj_init_stage(uint32_t sbase, const FusedOp *__restrict__ ops, int i0, int i1,
                                               DescStream &ds, int lane, float *__restrict__ out, int64_t nt,
                                               int64_t T0, const float *__restrict__ w, const float *__restrict__ x,
                                               float *__restrict__ part, int64_t part_row) {
  for_op_pairs(ops, i0, i1, ds, lane, [&](const FusedOp &a, const FusedOp &b, bool two) {
    float xa[kLaneCols], xb[kLaneCols];
    if (part != nullptr) {
      adj_init_load_x(xa, a, x, nt, T0, lane);
      if (two) adj_init_load_x(xb, b, x, nt, T0, lane);
    }
    adj_init_op<FOLD>(sbase, a, xa, lane, out, nt, T0, w, part, part_row);
    if (two) adj_init_op<FOLD>(sbase, b, xb, lane, out, nt, T0, w, part, part_row);
  });
}

// Persistent blocks over items = template * ntiles + tile, as the forward
// cone kernel.  INIT: the last stage is the initialisation transpose; it
// keeps two ops' input samples in flight, so it is compiled for two
// resident blocks per SM (more registers per thread).
template <bool INIT>
__global__ void __launch_bounds__(kFusedThreads, INIT ? 2 : kFusedMinBlocks)
adjoint_cone_kernel(const __grid_constant__ TmaMaps maps, float *__restrict__ out, int64_t nt, int32_t W,
                    int64_t ntiles, int64_t items, const FusedTemplate *__restrict__ tpls,
                    const FusedLoad *__restrict__ loads, const FusedOp *__restrict__ ops,
                    const int32_t *__restrict__ stages, const float *__restrict__ w, int32_t box,
                    int32_t cshift, int *__restrict__ status, const float *__restrict__ x,
                    float *__restrict__ part, int32_t pieces) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t bar = smem_u32(smem);

  int64_t item = blockIdx.x;
  if (item >= items) return;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
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
  if (warp == 0)
    stage_item<float>(smem, bar, maps.m, tp, loads, fetch_load(tp, loads, lane), T0_cur, box, cshift, lane);
  advance();
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
      atomicExch(status, 1);
      mbar_wait_bounded(bar, phase);
      return;
    }
    phase ^= 1u;
    {
      const StageRange r = ds_take(ds);
      if (cur.n_stages > 1) ds_peek(ds, stages, &cur, 1, warp);
      else ds_peek(ds, stages, next < items ? &tp_next : nullptr, 0, warp);
      if (!INIT && cur.n_stages == 1) adj_gather_stage<kOutGlobal>(bar, ops, r.i0, r.i1, ds, lane, out, nt, T0);
      else adj_gather_stage<kOutSmem>(bar, ops, r.i0, r.i1, ds, lane, out, nt, T0);
    }
    __syncthreads();  // S is no longer read: stage the next item into it
    if (next < items) {
      if (warp == 0) stage_item<float>(smem, bar, maps.m, tp_next, loads, ld_next, T0_next, box, cshift, lane);
      tp = tp_next;
      advance();
      if (next + gridDim.x < items) tp_next = tpls[tpl];
      T0_cur = T0_next;
    }
    for (int s = 1; s < cur.n_stages; ++s) {
      const StageRange r = ds_take(ds);
      if (s + 1 < cur.n_stages) ds_peek(ds, stages, &cur, s + 1, warp);
      else ds_peek(ds, stages, next < items ? &tp : nullptr, 0, warp);
      if (s == cur.n_stages - 1) {
        if (INIT) {
          float *const pt = part != nullptr ? part + (T0 / W) * pieces : nullptr;
          if (r.kind == kAdjInitF)
            adj_init_stage<true>(bar, ops, r.i0, r.i1, ds, lane, out, nt, T0, w, x, pt, ntiles * pieces);
          else
            adj_init_stage<false>(bar, ops, r.i0, r.i1, ds, lane, out, nt, T0, w, x, pt, ntiles * pieces);
        }
        else adj_gather_stage<kOutGlobal>(bar, ops, r.i0, r.i1, ds, lane, out, nt, T0);
      } else {
        adj_gather_stage<kOutSmem>(bar, ops, r.i0, r.i1, ds, lane, out, nt, T0);
        __syncthreads();
      }
    }
    __syncthreads();  // Pa / Pb are reused by the next item
  }
}

// The weight gradient from the init launch's partials: one warp per
// channel sums its (tile, piece) slots in a fixed order.
__global__ void __launch_bounds__(256)
adj_weights_finalize_kernel(const float *__restrict__ part, int32_t nf, int64_t per_channel,
                            float *__restrict__ gw) {
  const int lane = threadIdx.x & 31;
  const int64_t k = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (k >= nf) return;
  const float *p = part + k * per_channel;
  float d = 0.f;
  for (int64_t i = lane; i < per_channel; i += 32) d = __fadd_rn(d, p[i]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) d = __fadd_rn(d, __shfl_xor_sync(0xffffffffu, d, off));
  if (lane == 0) gw[k] = d;
}

template <bool INIT>
cudaError_t launch_adj_group(const DeviceTables &dt, const AdjGroup &g, const float *base, int64_t base_rows,
                             float *dst, const float *w, int64_t nt, cudaStream_t s, const float *x = nullptr,
                             float *part = nullptr) {
  auto kern = adjoint_cone_kernel<INIT>;
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [&] {
    attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  });
  if (attr_err != cudaSuccess) return attr_err;
  FusedGroup mg;  // the staged rows: row boxes of g.box samples or row blocks
  mg.box = g.box;
  mg.chunk = g.chunk;
  mg.kchunks = g.kchunks;
  mg.max_p = g.max_p;
  TmaMaps maps;
  int32_t cshift = 0;
  if (!make_group_maps(maps.m, mg, base, map_type<float>(), sizeof(float), (uint64_t)base_rows, (uint64_t)nt,
                       &cshift))
    return cudaErrorInvalidValue;
  const int64_t items = (int64_t)g.tpl_count * g.ntiles;
  if (items == 0) return cudaSuccess;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kFusedThreads, g.smem_bytes);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int64_t blocks = std::min<int64_t>(items, (int64_t)per_sm * sms);
  dt.prof->begin(s, K_ADJ_CONE, g.lb * 100 + g.lt);
  kern<<<(unsigned)blocks, kFusedThreads, g.smem_bytes, s>>>(maps, dst, nt, g.W, g.ntiles, items,
                                                            dt.a_tpls + g.tpl_begin, dt.a_loads, dt.a_ops,
                                                            dt.a_stages, w, g.box, cshift, dt.status, x, part,
                                                            g.pieces);
  dt.prof->end(s);
  return cudaGetLastError();
}

}  // namespace

cudaError_t run_adjoint_fused(const DeviceTables &dt, const float *grad_out, const float *w, float *grad_in,
                              void *const bufs[2], int64_t nt, cudaStream_t s, const float *x, float *part,
                              float *grad_w) {
  if (dt.adj_fused == nullptr) return cudaErrorInvalidValue;
  const AdjFusedPlan &ap = *dt.adj_fused;
  const int G = (int)ap.groups.size();
  for (int g = 0; g < G; ++g) {
    const AdjGroup &gr = ap.groups[g];
    const float *base = g == 0 ? grad_out : static_cast<const float *>(bufs[(g - 1) & 1]);
    float *dst = (g == G - 1) ? grad_in : static_cast<float *>(bufs[g & 1]);
    const int64_t rows = dt.level_rows[gr.lt];
    const cudaError_t e = gr.init ? launch_adj_group<true>(dt, gr, base, rows, dst, w, nt, s, x,
                                                           grad_w != nullptr ? part : nullptr)
                                  : launch_adj_group<false>(dt, gr, base, rows, dst, nullptr, nt, s);
    if (e != cudaSuccess) return e;
  }
  if (grad_w == nullptr) return cudaSuccess;
  const AdjGroup &gl = ap.groups.back();
  dt.prof->begin(s, K_ADJ_WFINAL, 0);
  adj_weights_finalize_kernel<<<(unsigned)((dt.nf + 7) / 8), 256, 0, s>>>(part, dt.nf, gl.ntiles * gl.pieces,
                                                                          grad_w);
  dt.prof->end(s);
  return cudaGetLastError();
}

}  // namespace fdmt
