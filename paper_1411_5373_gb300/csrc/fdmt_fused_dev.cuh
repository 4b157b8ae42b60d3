// Device-side building blocks of the fused-schedule kernels (single beam
// in fdmt_fused.cu, batches in fdmt_batch_fused.cu): mbarrier and TMA
// wrappers, shared-memory row adds, the Option-1 partial sums of a cone, the
// per-level op loops and the staging of one work item.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "fdmt_common.cuh"
#include "fdmt_fused.h"

namespace fdmt {

constexpr int kFusedWarps = kFusedBlockWarps;
constexpr int kFusedThreads = 32 * kFusedWarps;
constexpr int kWaitTries = 4000;            // x the suspend hint below: a ~2 s bound
constexpr uint32_t kSuspendHintNs = 500000;

// ---------------------------------------------------------------------------
// PTX helpers (mbarrier + TMA)

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

// try_wait with a suspend-time hint: a waiting thread sleeps in hardware
// until the phase completes or the hint elapses, instead of spinning.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(kSuspendHintNs)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity`; false if it did not complete in time.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  for (int i = 0; i < kWaitTries; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_row(uint32_t dst, const CUtensorMap *map, int32_t x,
                                             int32_t y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Row block: chunks [x, x + kchunks) of rows [y, y + 2^p) through a map of
// the [rows][nt / chunk][chunk] view whose box is (chunk, kchunks, 2^p).
__device__ __forceinline__ void tma_load_block(uint32_t dst, const CUtensorMap *map, int32_t x, int32_t y,
                                               uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// The tensor maps of a launch: row boxes use m[0]; row blocks use m[p] for
// copies of 2^p rows.
struct TmaMaps {
  CUtensorMap m[kMaxBlockP + 1];
};

template <bool R16>
__device__ __forceinline__ float round_state(float v) {
  if constexpr (R16) return __half2float(__float2half_rn(v));
  return v;
}
template <bool R16>
__device__ __forceinline__ int32_t round_state(int32_t v) { return v; }

template <class T> __device__ __forceinline__ T to_store(float v);
template <> __device__ __forceinline__ float to_store<float>(float v) { return v; }
template <> __device__ __forceinline__ __half to_store<__half>(float v) { return __float2half_rn(v); }
template <class T> __device__ __forceinline__ T to_store(int32_t v) { return v; }

// Ops of one level are shared out round-robin over the warps.  A warp
// fetches the descriptors of its next 32 ops with one load per lane and
// broadcasts them with shuffles, so descriptor latency is paid once per 32
// ops instead of once per op.
__device__ __forceinline__ FusedOp fetch_op(const FusedOp *__restrict__ ops, int idx, int end) {
  if (idx < end) return ops[idx];
  return FusedOp{0, 0, 0, 0};
}

__device__ __forceinline__ FusedOp bcast_op(const FusedOp &m, int k) {
  FusedOp o;
  o.dst = __shfl_sync(0xffffffffu, m.dst, k);
  o.lo = __shfl_sync(0xffffffffu, m.lo, k);
  o.hi = __shfl_sync(0xffffffffu, m.hi, k);
  o.width = __shfl_sync(0xffffffffu, m.width, k);
  return o;
}

// ---------------------------------------------------------------------------
// Row adds with explicit shared-memory accesses.  A lane handles columns
// lane, lane + 32, ...; four columns per trip with immediate offsets, so a
// trip costs 8 loads, 4 adds, 4 stores and three pointer bumps.  The asm
// statements are volatile and keep source order, so each trip issues all of
// its loads before its first add.

__device__ __forceinline__ float lds_f32(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ int32_t lds_s32(uint32_t a) {
  int32_t v;
  asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ float lds_h2f(uint32_t a) {
  unsigned short v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a) : "memory");
  return __half2float(__ushort_as_half(v));
}
__device__ __forceinline__ void sts_f32(uint32_t a, float v) {
  asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void sts_s32(uint32_t a, int32_t v) {
  asm volatile("st.shared.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

template <class TI, class A> __device__ __forceinline__ A load_input(uint32_t a);
template <> __device__ __forceinline__ float load_input<float, float>(uint32_t a) { return lds_f32(a); }
template <> __device__ __forceinline__ int32_t load_input<uint8_t, int32_t>(uint32_t a) {
  unsigned short v;
  asm volatile("ld.shared.u8 %0, [%1];" : "=h"(v) : "r"(a) : "memory");
  return (int32_t)v;
}

template <class T> struct Lds;
template <> struct Lds<float> {
  static __device__ __forceinline__ float get(uint32_t a) { return lds_f32(a); }
};
template <> struct Lds<int32_t> {
  static __device__ __forceinline__ int32_t get(uint32_t a) { return lds_s32(a); }
};
template <> struct Lds<__half> {
  static __device__ __forceinline__ float get(uint32_t a) { return lds_h2f(a); }
};
template <> struct Lds<uint16_t> {  // uint16-stored integer state
  static __device__ __forceinline__ int32_t get(uint32_t a) {
    unsigned short v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a) : "memory");
    return (int32_t)v;
  }
};
__device__ __forceinline__ void sts(uint32_t a, float v) { sts_f32(a, v); }
__device__ __forceinline__ void sts(uint32_t a, int32_t v) { sts_s32(a, v); }

// dst[tau] = lo[tau] + hi[tau] for tau in [0, width), all in shared memory.
template <class TSrc, class A, bool R16>
__device__ __forceinline__ void row_add_smem(uint32_t dst, uint32_t lo, uint32_t hi, int width, int lane) {
  constexpr uint32_t es = sizeof(TSrc), ed = sizeof(A);
  lo += lane * es;
  hi += lane * es;
  dst += lane * ed;
  int cnt = width > lane ? ((width - lane + 31) >> 5) : 0;
  for (; cnt >= 4; cnt -= 4) {
    const A a0 = Lds<TSrc>::get(lo), a1 = Lds<TSrc>::get(lo + 32 * es);
    const A a2 = Lds<TSrc>::get(lo + 64 * es), a3 = Lds<TSrc>::get(lo + 96 * es);
    const A b0 = Lds<TSrc>::get(hi), b1 = Lds<TSrc>::get(hi + 32 * es);
    const A b2 = Lds<TSrc>::get(hi + 64 * es), b3 = Lds<TSrc>::get(hi + 96 * es);
    sts(dst, round_state<R16>(acc_add(a0, b0)));
    sts(dst + 32 * ed, round_state<R16>(acc_add(a1, b1)));
    sts(dst + 64 * ed, round_state<R16>(acc_add(a2, b2)));
    sts(dst + 96 * ed, round_state<R16>(acc_add(a3, b3)));
    lo += 128 * es;
    hi += 128 * es;
    dst += 128 * ed;
  }
  for (; cnt > 0; --cnt) {
    const A a = Lds<TSrc>::get(lo), b = Lds<TSrc>::get(hi);
    sts(dst, round_state<R16>(acc_add(a, b)));
    lo += 32 * es;
    hi += 32 * es;
    dst += 32 * ed;
  }
}

// drow[tau] = lo[tau] + hi[tau] for tau in [0, lim): the top level, to global memory.
template <class TSrc, class TO, class A>
__device__ __forceinline__ void row_add_global(TO *drow, uint32_t lo, uint32_t hi, int lim, int lane) {
  constexpr uint32_t es = sizeof(TSrc);
  lo += lane * es;
  hi += lane * es;
  drow += lane;
  int cnt = lim > lane ? ((lim - lane + 31) >> 5) : 0;
  for (; cnt >= 4; cnt -= 4) {
    const A a0 = Lds<TSrc>::get(lo), a1 = Lds<TSrc>::get(lo + 32 * es);
    const A a2 = Lds<TSrc>::get(lo + 64 * es), a3 = Lds<TSrc>::get(lo + 96 * es);
    const A b0 = Lds<TSrc>::get(hi), b1 = Lds<TSrc>::get(hi + 32 * es);
    const A b2 = Lds<TSrc>::get(hi + 64 * es), b3 = Lds<TSrc>::get(hi + 96 * es);
    drow[0] = to_store<TO>(acc_add(a0, b0));
    drow[32] = to_store<TO>(acc_add(a1, b1));
    drow[64] = to_store<TO>(acc_add(a2, b2));
    drow[96] = to_store<TO>(acc_add(a3, b3));
    lo += 128 * es;
    hi += 128 * es;
    drow += 128;
  }
  for (; cnt > 0; --cnt) {
    const A a = Lds<TSrc>::get(lo), b = Lds<TSrc>::get(hi);
    drow[0] = to_store<TO>(acc_add(a, b));
    lo += 32 * es;
    hi += 32 * es;
    drow += 32;
  }
}

// Option-1 partial sums of one channel (section 4): row j of level 0 at
// column tau is x[tau] + x[tau - 1] + ... + x[tau - j], summed in that
// order; rows a..e are stored.  A lane handles columns lane, lane + 32, ...
// (`cnt` of them), four at a time so that four columns' loads are in
// flight together.
// E >= 0 fixes the last row at compile time (the loops unroll); E < 0
// takes e_rt.  SCALE multiplies each sample by the channel weight wk first.
template <class TI, class A, bool R16, bool SCALE, int E>
__device__ __forceinline__ void init_rows(uint32_t xa, uint32_t da, int a, int e_rt, int stride, int cnt,
                                          float wk) {
  constexpr uint32_t es = sizeof(TI), ed = sizeof(A);
  const int e = E >= 0 ? E : e_rt;
  const uint32_t rs = (uint32_t)stride * ed;
  auto in = [&](uint32_t addr) {
    A v = load_input<TI, A>(addr);
    if constexpr (SCALE) v = __fmul_rn(v, wk);
    return v;
  };
  for (; cnt >= 4; cnt -= 4) {
    A r0 = in(xa), r1 = in(xa + 32 * es), r2 = in(xa + 64 * es), r3 = in(xa + 96 * es);
    uint32_t d = da;
    if (a == 0) {
      sts(d, round_state<R16>(r0));
      sts(d + 32 * ed, round_state<R16>(r1));
      sts(d + 64 * ed, round_state<R16>(r2));
      sts(d + 96 * ed, round_state<R16>(r3));
      d += rs;
    }
#pragma unroll
    for (int i = 1; i <= e; ++i) {
      const uint32_t xi = xa - i * es;
      const A v0 = in(xi), v1 = in(xi + 32 * es), v2 = in(xi + 64 * es), v3 = in(xi + 96 * es);
      r0 = acc_add(r0, v0);
      r1 = acc_add(r1, v1);
      r2 = acc_add(r2, v2);
      r3 = acc_add(r3, v3);
      if (i >= a) {
        sts(d, round_state<R16>(r0));
        sts(d + 32 * ed, round_state<R16>(r1));
        sts(d + 64 * ed, round_state<R16>(r2));
        sts(d + 96 * ed, round_state<R16>(r3));
        d += rs;
      }
    }
    xa += 128 * es;
    da += 128 * ed;
  }
  for (; cnt > 0; --cnt) {
    A r = in(xa);
    uint32_t d = da;
    if (a == 0) {
      sts(d, round_state<R16>(r));
      d += rs;
    }
#pragma unroll
    for (int i = 1; i <= e; ++i) {
      r = acc_add(r, in(xa - i * es));
      if (i >= a) {
        sts(d, round_state<R16>(r));
        d += rs;
      }
    }
    xa += 32 * es;
    da += 32 * ed;
  }
}

// init_rows with the channel's last row (almost always 0..3) and the weight
// switch resolved to compile-time constants.
template <class TI, class A, bool R16, bool SCALE>
__device__ __forceinline__ void init_rows_any(uint32_t xa, uint32_t da, int a, int e, int stride, int cnt,
                                              float wk) {
  switch (e) {
    case 0: init_rows<TI, A, R16, SCALE, 0>(xa, da, a, e, stride, cnt, wk); break;
    case 1: init_rows<TI, A, R16, SCALE, 1>(xa, da, a, e, stride, cnt, wk); break;
    case 2: init_rows<TI, A, R16, SCALE, 2>(xa, da, a, e, stride, cnt, wk); break;
    case 3: init_rows<TI, A, R16, SCALE, 3>(xa, da, a, e, stride, cnt, wk); break;
    default: init_rows<TI, A, R16, SCALE, -1>(xa, da, a, e, stride, cnt, wk); break;
  }
}

// One level of ops in shared memory.  `first` holds the warp's first batch
// of descriptors (ops op0 + warp + 8 * lane), fetched ahead of time.
template <class TSrc, class A, bool R16>
__device__ __forceinline__ void level_in_smem(uint32_t sbase, const FusedOp *__restrict__ ops,
                                              int op0, int op1, int warp, int lane,
                                              const FusedOp &first) {
  for (int base = op0 + warp; base < op1; base += kFusedWarps * 32) {
    const FusedOp mine = (base == op0 + warp) ? first : fetch_op(ops, base + lane * kFusedWarps, op1);
    const int cnt = min(32, (op1 - base + kFusedWarps - 1) / kFusedWarps);
    for (int k = 0; k < cnt; ++k) {
      const FusedOp op = bcast_op(mine, k);
      row_add_smem<TSrc, A, R16>(sbase + op.dst, sbase + op.lo, sbase + op.hi, op.width, lane);
    }
  }
}

// The group's top level: the same adds, written to global memory.
template <class TSrc, class TO, class A>
__device__ __forceinline__ void level_to_global(uint32_t sbase, const FusedOp *__restrict__ ops,
                                                int op0, int op1, int warp, int lane, TO *out,
                                                int64_t nt, int64_t T0, int lim, const FusedOp &first) {
  for (int base = op0 + warp; base < op1; base += kFusedWarps * 32) {
    const FusedOp mine = (base == op0 + warp) ? first : fetch_op(ops, base + lane * kFusedWarps, op1);
    const int cnt = min(32, (op1 - base + kFusedWarps - 1) / kFusedWarps);
    for (int k = 0; k < cnt; ++k) {
      const FusedOp op = bcast_op(mine, k);
      row_add_global<TSrc, TO, A>(out + (int64_t)op.dst * nt + T0, sbase + op.lo, sbase + op.hi, lim, lane);
    }
  }
}

// Descriptors a block needs to start an item, fetched one item ahead: the
// template, the level boundaries (lane i holds the first op of level i) and
// the warp's first batch of first-stage descriptors.
struct ItemPrefetch {
  FusedTemplate tp;
  int bounds;
  FusedOp first_op;
  FusedInit first_init;
};

template <bool FROM_INPUT>
__device__ __forceinline__ ItemPrefetch prefetch_item(const FusedTemplate &tp,
                                                      const int32_t *__restrict__ level_ops,
                                                      const FusedOp *__restrict__ ops,
                                                      const FusedInit *__restrict__ inits, int warp,
                                                      int lane) {
  ItemPrefetch p;
  p.tp = tp;
  p.bounds = (lane <= p.tp.n_levels) ? level_ops[p.tp.level_begin + lane] : 0;
  p.first_op = FusedOp{0, 0, 0, 0};
  p.first_init = FusedInit{0, 0, 0, 0, 0, 0, 0, 0};
  if constexpr (FROM_INPUT) {
    const int my = warp + lane * kFusedWarps;
    if (my < p.tp.init_count) p.first_init = inits[p.tp.init_begin + my];
  } else {
    const int op0 = __shfl_sync(0xffffffffu, p.bounds, 0);
    const int op1 = __shfl_sync(0xffffffffu, p.bounds, 1);
    p.first_op = fetch_op(ops, op0 + warp + lane * kFusedWarps, op1);
  }
  return p;
}

__device__ __forceinline__ FusedLoad fetch_load(const FusedTemplate &tp, const FusedLoad *__restrict__ loads,
                                                int i) {
  if (i < tp.load_count) return loads[tp.load_begin + i];
  return FusedLoad{0, 0, 0, 0};
}

// Stage the rows of work item `item` into region S: warp 0 only; lane 0
// announces the bytes on the mbarrier, then the lanes issue the copies.
// `first` is load `lane` of the template, fetched ahead of time, so the
// copies go out without waiting on a descriptor read.  cshift > 0: row
// blocks of 2^cshift-element chunks; else row boxes of `box` elements.
template <class TS>
__device__ __forceinline__ void stage_item(unsigned char *smem, uint32_t bar, const CUtensorMap *maps,
                                           const FusedTemplate &tp, const FusedLoad *__restrict__ loads,
                                           const FusedLoad &first, int64_t T0, int32_t box, int32_t cshift,
                                           int lane) {
  // Order this block's earlier generic-proxy accesses of S before the
  // async-proxy copies that overwrite it.
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)tp.tx_bytes);
  __syncwarp();
  const uint32_t box_bytes = (uint32_t)box * (uint32_t)sizeof(TS);
  for (int i = lane; i < tp.load_count; i += 32) {
    const FusedLoad ld = (i == lane) ? first : loads[tp.load_begin + i];
    const int32_t x = (int32_t)(T0 + ld.xoff);
    const uint32_t dst = smem_u32(smem + ld.smem);
    if (cshift > 0) {
      tma_load_block(dst, maps + ld.nbox, x >> cshift, ld.row, bar);
    } else {
      for (int b = 0; b < ld.nbox; ++b) tma_load_row(dst + b * box_bytes, maps, x + b * box, ld.row, bar);
    }
  }
}

// First stage of a from-input item: the Option-1 partial sums of its
// channels (or column pieces of channels), one per warp in turn; `first`
// holds the warp's first batch of init descriptors.
template <class TI, class A, bool R16>
__device__ __forceinline__ void item_inits(uint32_t bar, const FusedInit *__restrict__ inits,
                                           const FusedTemplate &tp, const FusedInit &first,
                                           const float *__restrict__ w, int warp, int lane) {
  const FusedInit *__restrict__ ib = inits + tp.init_begin;
  for (int base = warp; base < tp.init_count; base += kFusedWarps * 32) {
    const int my = base + lane * kFusedWarps;
    FusedInit mine = first;
    if (base != warp) mine = (my < tp.init_count) ? ib[my] : FusedInit{0, 0, 0, 0, 0, 0, 0, 0};
    const int cnt = min(32, (tp.init_count - base + kFusedWarps - 1) / kFusedWarps);
    for (int k = 0; k < cnt; ++k) {
      const int x_smem = __shfl_sync(0xffffffffu, mine.x_smem, k);
      const int dst_smem = __shfl_sync(0xffffffffu, mine.dst_smem, k);
      const int a = __shfl_sync(0xffffffffu, mine.a, k);
      const int e = __shfl_sync(0xffffffffu, mine.e, k);
      const int width = __shfl_sync(0xffffffffu, mine.width, k);
      const int chan = __shfl_sync(0xffffffffu, mine.chan, k);
      const int stride = __shfl_sync(0xffffffffu, mine.dst_stride, k);
      const uint32_t xa = bar + x_smem + lane * (uint32_t)sizeof(TI);
      const uint32_t da = bar + dst_smem + lane * (uint32_t)sizeof(A);
      const int ncol = width > lane ? ((width - lane + 31) >> 5) : 0;
      bool scaled = false;
      if constexpr (std::is_floating_point<A>::value) {
        if (w != nullptr) {
          init_rows_any<TI, A, R16, true>(xa, da, a, e, stride, ncol, w[chan]);
          scaled = true;
        }
      }
      if (!scaled) init_rows_any<TI, A, R16, false>(xa, da, a, e, stride, ncol, 1.0f);
    }
  }
}

// First stage of an item staged from the state: its first merge level,
// read from the staged rows (to global memory if it is the only level).
template <class TB, class TO, class A, bool R16>
__device__ __forceinline__ void item_first_level(uint32_t bar, const FusedOp *__restrict__ ops,
                                                 const FusedTemplate &tp, int bounds, const FusedOp &first,
                                                 int warp, int lane, TO *out, int64_t nt, int64_t T0, int lim) {
  const int op0 = __shfl_sync(0xffffffffu, bounds, 0);
  const int op1 = __shfl_sync(0xffffffffu, bounds, 1);
  if (tp.n_levels == 1)
    level_to_global<TB, TO, A>(bar, ops, op0, op1, warp, lane, out, nt, T0, lim, first);
  else
    level_in_smem<TB, A, R16>(bar, ops, op0, op1, warp, lane, first);
}

// Levels lv0 .. nlev - 1 of an item (lane i of `bounds` holds the first op
// of level i), each level's first descriptor batch fetched while the
// previous level is computed; the last level goes to global memory.
template <class TO, class A, bool R16>
__device__ __forceinline__ void item_levels(uint32_t bar, const FusedOp *__restrict__ ops, int bounds, int lv0,
                                            int nlev, int warp, int lane, TO *out, int64_t nt, int64_t T0,
                                            int lim) {
  FusedOp pf = FusedOp{0, 0, 0, 0};
  if (lv0 < nlev)
    pf = fetch_op(ops, __shfl_sync(0xffffffffu, bounds, lv0) + warp + lane * kFusedWarps,
                  __shfl_sync(0xffffffffu, bounds, lv0 + 1));
  for (int lv = lv0; lv < nlev; ++lv) {
    const int op0 = __shfl_sync(0xffffffffu, bounds, lv);
    const int op1 = __shfl_sync(0xffffffffu, bounds, lv + 1);
    const FusedOp here = pf;
    if (lv + 1 < nlev)
      pf = fetch_op(ops, op1 + warp + lane * kFusedWarps, __shfl_sync(0xffffffffu, bounds, lv + 2));
    if (lv == nlev - 1) {
      level_to_global<A, TO, A>(bar, ops, op0, op1, warp, lane, out, nt, T0, lim, here);
    } else {
      level_in_smem<A, A, R16>(bar, ops, op0, op1, warp, lane, here);
      __syncthreads();
    }
  }
}

}  // namespace fdmt
