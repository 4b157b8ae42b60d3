// Device-side building blocks of the fused-schedule kernels (single beam
// in fdmt_fused.cu, batches in fdmt_batch_fused.cu): mbarrier and TMA
// wrappers, the staging of one work item, and its compute stages (level 1
// walked from the staged input, single levels and pairs of levels).
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <type_traits>

#include "fdmt_common.cuh"
#include "fdmt_fused.h"

namespace fdmt {

constexpr int kFusedWarps = kFusedBlockWarps;
constexpr int kFusedThreads = 32 * kFusedWarps;
#ifndef FDMT_MIN_BLOCKS
#define FDMT_MIN_BLOCKS 3
#endif
constexpr int kFusedMinBlocks = FDMT_MIN_BLOCKS;  // resident blocks per SM the register budget allows
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

// Predicated shared-memory loads (no branch): 0 where the predicate is off,
// and no shared-memory access is made for those lanes.
__device__ __forceinline__ float lds_f32_if(uint32_t a, bool p) {
  float v;
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\tmov.f32 %0, 0f00000000;\n\t"
               "@q ld.shared.f32 %0, [%1];\n\t}" : "=f"(v) : "r"(a), "r"((uint32_t)p) : "memory");
  return v;
}
__device__ __forceinline__ int32_t lds_s32_if(uint32_t a, bool p) {
  int32_t v;
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\tmov.s32 %0, 0;\n\t"
               "@q ld.shared.s32 %0, [%1];\n\t}" : "=r"(v) : "r"(a), "r"((uint32_t)p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t lds_u16_if(uint32_t a, bool p) {
  uint32_t v;
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\tmov.u32 %0, 0;\n\t"
               "@q ld.shared.u16 %0, [%1];\n\t}" : "=r"(v) : "r"(a), "r"((uint32_t)p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t lds_u8_if(uint32_t a, bool p) {
  uint32_t v;
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\tmov.u32 %0, 0;\n\t"
               "@q ld.shared.u8 %0, [%1];\n\t}" : "=r"(v) : "r"(a), "r"((uint32_t)p) : "memory");
  return v;
}
template <class T> struct LdsIf;
template <> struct LdsIf<float> {
  static __device__ __forceinline__ float get(uint32_t a, bool p) { return lds_f32_if(a, p); }
};
template <> struct LdsIf<int32_t> {
  static __device__ __forceinline__ int32_t get(uint32_t a, bool p) { return lds_s32_if(a, p); }
};
template <> struct LdsIf<__half> {
  static __device__ __forceinline__ float get(uint32_t a, bool p) {
    return __half2float(__ushort_as_half((unsigned short)lds_u16_if(a, p)));
  }
};
template <> struct LdsIf<uint16_t> {
  static __device__ __forceinline__ int32_t get(uint32_t a, bool p) { return (int32_t)lds_u16_if(a, p); }
};
template <> struct LdsIf<uint8_t> {
  static __device__ __forceinline__ int32_t get(uint32_t a, bool p) { return (int32_t)lds_u8_if(a, p); }
};

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

// ---------------------------------------------------------------------------
// Stages of a work item.  Each warp runs its own list of ops (the planner
// splits every stage into kFusedBlockWarps contiguous lists); lane l handles
// columns l, l + 32, ..., l + 32 (kLaneCols - 1) of an op's piece, so every
// shared-memory access of a warp touches 32 consecutive words (no bank
// conflicts).  Values that an op's reuse flags carry over stay in registers.

// Descriptors: every lane reads the same address (one broadcast request).
__device__ __forceinline__ FusedOp ld_op(const FusedOp *__restrict__ p) {
  const int4 a = __ldg(reinterpret_cast<const int4 *>(p));
  const int4 b = __ldg(reinterpret_cast<const int4 *>(p) + 1);
  return FusedOp{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
}
__device__ __forceinline__ FusedWalk ld_walk(const FusedWalk *__restrict__ p) {
  const int4 a = __ldg(reinterpret_cast<const int4 *>(p));
  const int4 b = __ldg(reinterpret_cast<const int4 *>(p) + 1);
  const int4 c = __ldg(reinterpret_cast<const int4 *>(p) + 2);
  return FusedWalk{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
}

__device__ __forceinline__ void sts_v4(uint32_t a, int4 v) {
  asm volatile("st.shared.v4.s32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}
__device__ __forceinline__ int4 lds_v4(uint32_t a) {
  int4 v;
  asm volatile("ld.shared.v4.s32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a)
               : "memory");
  return v;
}

// A warp's descriptor stream through the stages of its items.  The words
// of the stage that runs next (its kind and this warp's first and end op or
// walk) are requested one stage ahead; during the last chunk of a stage the
// first chunk of the next stage (or of the next item's first stage) comes
// into `q`, so a stage starts without a round trip to L2.
struct DescStream {
  uint32_t slot;      // the warp's slot in shared memory (kDescSlotBytes)
  int4 q;             // this lane's 16 bytes of the next stage's first chunk
  int kind, i0, i1;   // the next stage (kind < 0: none)
  bool ready;         // q holds that chunk
};

constexpr int kWalkChunk = kDescSlotBytes / 48;  // walks per chunk (48 bytes: three lanes each)

// Request the words of stage s of template tp (none if tp is null).
__device__ __forceinline__ void ds_peek(DescStream &ds, const int32_t *__restrict__ stages,
                                        const FusedTemplate *tp, int s, int warp) {
  ds.ready = false;
  if (tp == nullptr || s >= tp->n_stages) {
    ds.kind = -1;
    ds.i0 = ds.i1 = 0;
    return;
  }
  const int32_t *p = stages + tp->stage_begin + s * kStageWords;
  ds.kind = __ldg(p);
  ds.i0 = __ldg(p + 1 + warp);
  ds.i1 = __ldg(p + 2 + warp);
}

// Load the first chunk of the requested stage into q (walk or op layout).
__device__ __forceinline__ void ds_load_first(DescStream &ds, const FusedOp *__restrict__ ops,
                                              const FusedWalk *__restrict__ walks, int lane) {
  if (ds.ready || ds.kind < 0) return;
  const int k = ds.kind & kStageKindMask;
  int4 q = make_int4(0, 0, 0, 0);
  if (k == kStageWalk) {
    if (lane < 3 * kWalkChunk && 3 * ds.i0 + lane < 3 * ds.i1)
      q = __ldg(reinterpret_cast<const int4 *>(walks) + 3 * ds.i0 + lane);
  } else if (k != kStageSearch) {
    if (2 * ds.i0 + lane < 2 * ds.i1) q = __ldg(reinterpret_cast<const int4 *>(ops) + 2 * ds.i0 + lane);
  }
  ds.q = q;
  ds.ready = true;
}

// The stage about to run (the one requested last) as a range.
struct StageRange {
  int kind, i0, i1;
};
__device__ __forceinline__ StageRange ds_take(const DescStream &ds) { return StageRange{ds.kind, ds.i0, ds.i1}; }

// Runs body(op) for ops i0 .. i1 - 1 of this warp, in order.  The lanes
// copy the descriptors kDescChunk at a time (two lanes per 32-byte op) into
// the warp's slot; the next chunk's loads are in flight while the current
// chunk runs (for the last chunk: the next stage's first chunk), and every
// op is read back from the slot as a broadcast.  On entry ds.q holds the
// first chunk if ds.ready; ds's stage words are the next stage's.
template <class F>
__device__ __forceinline__ void for_ops(const FusedOp *__restrict__ ops, const FusedWalk *__restrict__ walks,
                                        int i0, int i1, DescStream &ds, int lane, F &&body) {
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
      ds_load_first(ds, ops, walks, lane);
    }
    const int n = min(kDescChunk, i1 - base);
    for (int k = 0; k < n; ++k) {
      const int4 a = lds_v4(ds.slot + 32u * (uint32_t)k), b = lds_v4(ds.slot + 32u * (uint32_t)k + 16u);
      body(FusedOp{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w});
    }
  }
  if (i0 >= i1) ds_load_first(ds, ops, walks, lane);
}

// The same for walks (48 bytes: three lanes per walk, kWalkChunk walks per
// slot).  A walk keeps many running sums in registers, so a later chunk's
// descriptors are fetched when it starts, and the next stage's first chunk
// once the last walk is done.
template <class F>
__device__ __forceinline__ void for_walks(const FusedWalk *__restrict__ walks, const FusedOp *__restrict__ ops,
                                          int i0, int i1, DescStream &ds, int lane, F &&body) {
  const int4 *src = reinterpret_cast<const int4 *>(walks);
  constexpr int kWords = 3 * kWalkChunk;  // 16-byte words per chunk
  bool first = ds.ready;
  int4 q0 = ds.q;
  ds.ready = false;
  for (int base = i0; base < i1; base += kWalkChunk) {
    __syncwarp();
    if (lane < kWords && 3 * base + lane < 3 * i1) sts_v4(ds.slot + 16u * (uint32_t)lane, first ? q0 : __ldg(src + 3 * base + lane));
    first = false;
    __syncwarp();
    const int n = min(kWalkChunk, i1 - base);
    for (int k = 0; k < n; ++k) {
      const uint32_t a = ds.slot + 48u * (uint32_t)k;
      const int4 x = lds_v4(a), y = lds_v4(a + 16u), z = lds_v4(a + 32u);
      body(FusedWalk{x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w, z.x, z.y, z.z, z.w});
    }
  }
  ds_load_first(ds, ops, walks, lane);
}

// C columns of a row piece from shared memory (columns >= width read nothing).
// kLaneCols columns of a row piece from shared memory.  The loads are
// unconditional (no branch or predicate between them): columns at or beyond
// the op's width read whatever lies there, which the planner keeps inside
// the block's shared memory (kOverRead bytes of slack after the last
// region), and those values never reach a stored column.
template <class TSrc, class A>
__device__ __forceinline__ void ld_piece(A (&v)[kLaneCols], uint32_t addr, int lane) {
  constexpr uint32_t es = sizeof(TSrc);
  addr += (uint32_t)lane * es;
#pragma unroll
  for (int k = 0; k < kLaneCols; ++k) v[k] = (A)Lds<TSrc>::get(addr + (uint32_t)(32 * k) * es);
}

// v[k] <- v at one column earlier (lane l takes lane l - 1's value; lane 0
// of the first column group takes `first`).
template <class A>
__device__ __forceinline__ void shift_one(A (&v)[kLaneCols], A first, int lane) {
  A s[kLaneCols];
#pragma unroll
  for (int k = 0; k < kLaneCols; ++k) s[k] = __shfl_sync(0xffffffffu, v[k], (lane + 31) & 31);
  v[0] = lane ? s[0] : first;
#pragma unroll
  for (int k = 1; k < kLaneCols; ++k) v[k] = lane ? s[k] : s[k - 1];
}

// Predicated stores (no branch): only columns below the limit are written.
__device__ __forceinline__ void sts_if(uint32_t a, float v, bool p) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.shared.f32 [%0], %1;\n\t}"
               ::"r"(a), "f"(v), "r"((uint32_t)p) : "memory");
}
__device__ __forceinline__ void sts_if(uint32_t a, int32_t v, bool p) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.shared.s32 [%0], %1;\n\t}"
               ::"r"(a), "r"(v), "r"((uint32_t)p) : "memory");
}
__device__ __forceinline__ void stg_if(float *g, float v, bool p) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.global.f32 [%0], %1;\n\t}"
               ::"l"(g), "f"(v), "r"((uint32_t)p) : "memory");
}
__device__ __forceinline__ void stg_if(int32_t *g, int32_t v, bool p) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.global.s32 [%0], %1;\n\t}"
               ::"l"(g), "r"(v), "r"((uint32_t)p) : "memory");
}
__device__ __forceinline__ void stg_if(__half *g, float v, bool p) {
  const unsigned short h = __half_as_ushort(__float2half_rn(v));
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.global.u16 [%0], %1;\n\t}"
               ::"l"(g), "h"(h), "r"((uint32_t)p) : "memory");
}
__device__ __forceinline__ void stg_if(uint16_t *g, int32_t v, bool p) {
  const unsigned short h = (unsigned short)v;
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.global.u16 [%0], %1;\n\t}"
               ::"l"(g), "h"(h), "r"((uint32_t)p) : "memory");
}

// Store an op's result: to shared memory (a stored level, rounded in
// fp16-state mode) or, for the top stage, to the global row at columns
// T0 + col + tau, tau < n.  A whole piece is stored without predicates.
template <class A, bool R16>
__device__ __forceinline__ void st_piece_smem(uint32_t addr, const A (&v)[kLaneCols], int width, int lane) {
  addr += (uint32_t)lane * sizeof(A);
  if (width >= kPieceCols) {
#pragma unroll
    for (int k = 0; k < kLaneCols; ++k) sts(addr + (uint32_t)(32 * k) * sizeof(A), round_state<R16>(v[k]));
  } else {
#pragma unroll
    for (int k = 0; k < kLaneCols; ++k)
      sts_if(addr + (uint32_t)(32 * k) * sizeof(A), round_state<R16>(v[k]), lane + 32 * k < width);
  }
}
template <class TO, class A>
__device__ __forceinline__ void st_piece_global(TO *__restrict__ drow, const A (&v)[kLaneCols], int n, int lane) {
  drow += lane;
  if (n >= kPieceCols) {
#pragma unroll
    for (int k = 0; k < kLaneCols; ++k) drow[32 * k] = to_store<TO>(v[k]);
  } else {
#pragma unroll
    for (int k = 0; k < kLaneCols; ++k) stg_if(drow + 32 * k, v[k], lane + 32 * k < n);
  }
}

// The top level of a searched launch into Pt, in the search layout (column c
// of a row at word c + 4 (c / 16)); it is the output level, never rounded.
template <class A>
__device__ __forceinline__ void st_piece_padded(uint32_t addr, const A (&v)[kLaneCols], int width, int lane) {
  addr += (uint32_t)(lane + 4 * (lane >> 4)) * sizeof(A);
#pragma unroll
  for (int k = 0; k < kLaneCols; ++k) sts_if(addr + (uint32_t)(40 * k) * sizeof(A), v[k], lane + 32 * k < width);
}

// One level per op: out = lo + hi (lo reused under kOpLoSame).
// Where a merge stage writes: shared memory (a stored level), global memory
// (the group's top level), or shared memory in the search layout (the top
// level of a launch that ends with the boxcar search).
enum : int { kOutSmem = 0, kOutGlobal = 1, kOutPadded = 2 };

// GEN: the stage has ops with a passed-up or one-term half (Nf not a power
// of two); without it those tests are compiled out of the loop.
template <class TSrc, class A, class TO, bool R16, int OUT, bool GEN>
__device__ __forceinline__ void stage_single(uint32_t sbase, const FusedOp *__restrict__ ops,
                                             const FusedWalk *__restrict__ walks, int i0, int i1, DescStream &ds,
                                             int lane, TO *__restrict__ out, int64_t nt, int64_t T0, int lim) {
  A lo[kLaneCols], hi[kLaneCols], v[kLaneCols];
#pragma unroll
  for (int k = 0; k < kLaneCols; ++k) lo[k] = (A)0;
  for_ops(ops, walks, i0, i1, ds, lane, [&](const FusedOp &op) {
    if (!(op.flags & kOpLoSame)) ld_piece<TSrc, A>(lo, sbase + op.p0, lane);
    if (GEN && (op.flags & kOpNoHi)) {  // no upper half: the lower row passes up
#pragma unroll
      for (int k = 0; k < kLaneCols; ++k) v[k] = lo[k];
    } else {
      ld_piece<TSrc, A>(hi, sbase + op.p1, lane);
#pragma unroll
      for (int k = 0; k < kLaneCols; ++k) v[k] = acc_add(lo[k], hi[k]);
    }
    if constexpr (OUT == kOutGlobal) {
      st_piece_global<TO, A>(out + (int64_t)op.dst * nt + T0 + op.col, v, min(op.width, lim - op.col), lane);
    } else if constexpr (OUT == kOutPadded) {
      st_piece_padded<A>(sbase + op.dst, v, op.width, lane);
    } else {
      st_piece_smem<A, R16>(sbase + op.dst, v, op.width, lane);
    }
  });
}

// Two levels per op: out = (s[p0] + s[p1]) + (s[p2] + s[p3]); the lower
// half sum is reused under kOpLoSame, the upper half sum is the previous
// one moved a column later under kOpHiShift.  The half sums belong to a
// level below the top, so fp16-state mode rounds them.
template <class TSrc, class A, class TO, bool R16, int OUT, bool GEN>
__device__ __forceinline__ void stage_pair(uint32_t sbase, const FusedOp *__restrict__ ops,
                                           const FusedWalk *__restrict__ walks, int i0, int i1, DescStream &ds,
                                           int lane, TO *__restrict__ out, int64_t nt, int64_t T0, int lim) {
  constexpr uint32_t es = sizeof(TSrc);
  A lp[kLaneCols], hp[kLaneCols], a[kLaneCols], b[kLaneCols];
#pragma unroll
  for (int k = 0; k < kLaneCols; ++k) lp[k] = hp[k] = (A)0;
  for_ops(ops, walks, i0, i1, ds, lane, [&](const FusedOp &op) {
    if (!(op.flags & kOpLoSame)) {
      ld_piece<TSrc, A>(a, sbase + op.p0, lane);
      if (GEN && (op.flags & kOpLoOne)) {
#pragma unroll
        for (int k = 0; k < kLaneCols; ++k) lp[k] = round_state<R16>(a[k]);
      } else {
        ld_piece<TSrc, A>(b, sbase + op.p1, lane);
#pragma unroll
        for (int k = 0; k < kLaneCols; ++k) lp[k] = round_state<R16>(acc_add(a[k], b[k]));
      }
    }
    A v[kLaneCols];
    if (GEN && (op.flags & kOpNoHi)) {  // no upper half: the lower part passes up
#pragma unroll
      for (int k = 0; k < kLaneCols; ++k) v[k] = lp[k];
    } else {
      const bool one = GEN && (op.flags & kOpHiOne) != 0;
      if (op.flags & kOpHiShift) {
        // column 0 of the new upper half sum (every lane reads the same words)
        const A h0 = (A)Lds<TSrc>::get(sbase + op.p2);
        const A first = round_state<R16>(one ? h0 : acc_add(h0, (A)Lds<TSrc>::get(sbase + op.p3)));
        shift_one<A>(hp, first, lane);
      } else {
        ld_piece<TSrc, A>(a, sbase + op.p2, lane);
        if (one) {
#pragma unroll
          for (int k = 0; k < kLaneCols; ++k) hp[k] = round_state<R16>(a[k]);
        } else {
          ld_piece<TSrc, A>(b, sbase + op.p3, lane);
#pragma unroll
          for (int k = 0; k < kLaneCols; ++k) hp[k] = round_state<R16>(acc_add(a[k], b[k]));
        }
      }
#pragma unroll
      for (int k = 0; k < kLaneCols; ++k) v[k] = acc_add(lp[k], hp[k]);
    }
    if constexpr (OUT == kOutGlobal) {
      st_piece_global<TO, A>(out + (int64_t)op.dst * nt + T0 + op.col, v, min(op.width, lim - op.col), lane);
    } else if constexpr (OUT == kOutPadded) {
      st_piece_padded<A>(sbase + op.dst, v, op.width, lane);
    } else {
      st_piece_smem<A, R16>(sbase + op.dst, v, op.width, lane);
    }
  });
  (void)es;
}

// Level 1 straight from the staged input (section 4: the Option-1 partial
// sums of level 0 and one merge).  The running sums plo = x_lo[tau] + ... +
// x_lo[tau - dl] and phi = x_hi[tau - dl] + ... + x_hi[tau - dl - j] are
// kept in registers in the oracle's order (each adds one earlier sample);
// when dl grows the upper sums move one column later (its first column is
// summed afresh by lane 0).  SCALE multiplies every sample by its channel's
// weight first.
template <class TI, class A, class TO, bool R16, bool SCALE, bool TOP, bool GEN>
__device__ __forceinline__ void stage_walk(uint32_t sbase, const FusedWalk *__restrict__ walks,
                                           const FusedOp *__restrict__ ops, int i0, int i1, DescStream &ds,
                                           int lane, const float *__restrict__ w, TO *__restrict__ out, int64_t nt,
                                           int64_t T0, int lim) {
  constexpr int32_t es = (int32_t)sizeof(TI);
  A plo[kLaneCols], phi[kLaneCols], v[kLaneCols];
  for_walks(walks, ops, i0, i1, ds, lane, [&](const FusedWalk &wk) {
    float wl = 1.0f, wh = 1.0f;
    if constexpr (SCALE) {
      wl = __ldg(w + wk.chan);
      wh = __ldg(w + wk.chan + 1);
    }
    const uint32_t xl = sbase + wk.x_lo, xh = sbase + wk.x_hi;
    // Sample of a channel `s` columns before column col (scaled).
    auto smp = [&](uint32_t base, int col, int s, float wt) -> A {
      A x = load_input<TI, A>(base + (uint32_t)((col - s) * es));
      if constexpr (SCALE) x = __fmul_rn(x, wt);
      return x;
    };
    const bool upper = !GEN || !(wk.flags & kWalkNoUpper);
    int dl = wk.dl0, j = wk.a - wk.dl0;
#pragma unroll
    for (int k = 0; k < kLaneCols; ++k) {
      const int col = lane + 32 * k;
      A s0 = smp(xl, col, 0, wl);
      for (int t = 1; t <= dl; ++t) s0 = acc_add(s0, smp(xl, col, t, wl));
      A s1 = A(0);
      if (upper) {
        s1 = smp(xh, col, dl, wh);
        for (int t = 1; t <= j; ++t) s1 = acc_add(s1, smp(xh, col, dl + t, wh));
      }
      plo[k] = s0;
      phi[k] = s1;
    }
    for (int r = wk.a; r <= wk.e; ++r) {
      if (r > wk.a && !upper) {
        // a single channel: row r is its Option-1 row r (dl = r)
        ++dl;
#pragma unroll
        for (int k = 0; k < kLaneCols; ++k) plo[k] = acc_add(plo[k], smp(xl, lane + 32 * k, dl, wl));
      } else if (r > wk.a) {
        if ((wk.bits >> (r - wk.a - 1)) & 1) {
          ++dl;
          // every lane sums column 0 (the same addresses: broadcast reads)
          A first = smp(xh, 0, dl, wh);
          for (int t = 1; t <= j; ++t) first = acc_add(first, smp(xh, 0, dl + t, wh));
#pragma unroll
          for (int k = 0; k < kLaneCols; ++k) plo[k] = acc_add(plo[k], smp(xl, lane + 32 * k, dl, wl));
          shift_one<A>(phi, first, lane);
        } else {
          ++j;
#pragma unroll
          for (int k = 0; k < kLaneCols; ++k) phi[k] = acc_add(phi[k], smp(xh, lane + 32 * k, dl + j, wh));
        }
      }
      if (upper) {
#pragma unroll
        for (int k = 0; k < kLaneCols; ++k) v[k] = acc_add(round_state<R16>(plo[k]), round_state<R16>(phi[k]));
      } else {
#pragma unroll
        for (int k = 0; k < kLaneCols; ++k) v[k] = round_state<R16>(plo[k]);
      }
      if constexpr (TOP) {
        st_piece_global<TO, A>(out + (int64_t)(wk.dst + r - wk.a) * nt + T0 + wk.col, v,
                               min(wk.width, lim - wk.col), lane);
      } else {
        st_piece_smem<A, R16>(sbase + wk.dst + (uint32_t)((r - wk.a) * wk.dst_row), v, wk.width, lane);
      }
    }
  });
}

// A warp's descriptor slot: the template's layout ends with the slots of
// the block's warps, then the over-read slack.
__device__ __forceinline__ uint32_t desc_slot(uint32_t sbase, const FusedTemplate &tp, int warp) {
  return sbase + (uint32_t)(tp.smem_bytes - kOverRead - kDescBytes + warp * kDescSlotBytes);
}

// Stage words of stage s of a template: kind, first op of warp w, first op
// of warp w + 1.
__device__ __forceinline__ StageRange stage_range(const int32_t *__restrict__ stages, int stage_begin, int s,
                                                  int warp) {
  const int32_t *p = stages + stage_begin + s * kStageWords;
  return StageRange{__ldg(p), __ldg(p + 1 + warp), __ldg(p + 2 + warp)};
}

// Stage s of an item; TSrc is the type of the stage's source rows (the
// staged base level for the first stage, the accumulator type after it).
// ds: this warp's descriptor stream (its next stage already requested).
// GEN: the plan may hold stages with passed-up or one-term halves (else
// only the code without those tests is compiled in).
template <class TSrc, class A, class TO, bool R16, int OUT, bool GEN = true>
__device__ __forceinline__ void run_merge_stage(const StageRange &r, uint32_t sbase, DescStream &ds,
                                                const FusedOp *__restrict__ ops, const FusedWalk *__restrict__ walks,
                                                int lane, TO *__restrict__ out, int64_t nt, int64_t T0, int lim) {
  const bool gen = GEN && (r.kind & kStageGeneral) != 0;
  if ((r.kind & kStageKindMask) == kStagePair) {
    if (gen) stage_pair<TSrc, A, TO, R16, OUT, true>(sbase, ops, walks, r.i0, r.i1, ds, lane, out, nt, T0, lim);
    else stage_pair<TSrc, A, TO, R16, OUT, false>(sbase, ops, walks, r.i0, r.i1, ds, lane, out, nt, T0, lim);
  } else {
    if (gen) stage_single<TSrc, A, TO, R16, OUT, true>(sbase, ops, walks, r.i0, r.i1, ds, lane, out, nt, T0, lim);
    else stage_single<TSrc, A, TO, R16, OUT, false>(sbase, ops, walks, r.i0, r.i1, ds, lane, out, nt, T0, lim);
  }
}

// ---------------------------------------------------------------------------
// Boxcar search of the top level (section 4.2, pulse profile) in the last
// launch.  For width w = 2^k the boxcar sum B_w[t] = A[t - w + 1] + ... +
// A[t] is built as the binary tree B_1 = A, B_2w[t] = B_w[t] + B_w[t - w];
// per (row, width) the largest value over the tile's own columns and the
// region where it first occurs are kept, to be resolved to a time by the
// search's finalize kernel, which recomputes the region from A.  Regions
// are 16 samples for widths 1 .. 16 and 256 samples for widths 32 .. 256,
// named by the time of their first sample.

constexpr int kSearchNoRegion = INT32_MIN;

__device__ __forceinline__ float search_lowest(float) { return -__int_as_float(0x7f800000); }
__device__ __forceinline__ int32_t search_lowest(int32_t) { return INT32_MIN; }
__device__ __forceinline__ float search_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ int32_t search_max(int32_t a, int32_t b) { return max(a, b); }

// Per (row, width) best of an item, one 64-bit word in shared memory
// reduced with atomicMax: the value's order-preserving bits above the
// complement of its region, so the maximum is the largest value and, among
// equal values, the earliest region.  0 = nothing seen.
__device__ __forceinline__ uint32_t search_order(float v) {
  const uint32_t b = __float_as_uint(v);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ uint32_t search_order(int32_t v) { return (uint32_t)v ^ 0x80000000u; }
__device__ __forceinline__ float search_value(uint32_t o, float) {
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}
__device__ __forceinline__ int32_t search_value(uint32_t o, int32_t) { return (int32_t)(o ^ 0x80000000u); }
__device__ __forceinline__ bool search_nan(float v) { return v != v; }
__device__ __forceinline__ bool search_nan(int32_t) { return false; }

// The key of the largest of x[16 .. 31] over the columns c0 + S (i - 16) in
// [lo, hi), with `region` (the time of the region's first sample); 0 when
// `use` is false or nothing qualifies.  NaN never qualifies (the transform
// of finite input is finite).
template <class A, int S>
__device__ __forceinline__ unsigned long long search_key(const A (&x)[32], bool use, int c0, int lo, int hi,
                                                         int region) {
  if (!use) return 0ull;
  A m;
  if (c0 >= lo && c0 + 15 * S < hi) {
    A t[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) t[i] = search_max(x[16 + i], x[24 + i]);
#pragma unroll
    for (int i = 0; i < 4; ++i) t[i] = search_max(t[i], t[i + 4]);
    m = search_max(search_max(t[0], t[2]), search_max(t[1], t[3]));
  } else {
    m = search_lowest(A());
    bool any = false;
#pragma unroll
    for (int i = 16; i < 32; ++i) {
      const int c = c0 + S * (i - 16);
      if (c >= lo && c < hi) {
        m = search_max(m, x[i]);
        any = true;
      }
    }
    if (!any) return 0ull;
  }
  if (search_nan(m)) return 0ull;
  return ((unsigned long long)search_order(m) << 32) | (uint32_t)(0x7fffffff - region);
}

// Joins the keys of a warp into the best words they name: lanes naming the
// same word are reduced in registers first (largest value, then earliest
// region), then one atomicMax per word.  Every lane of the warp calls it.
__device__ __forceinline__ void search_join_warp(unsigned long long key, uint32_t addr, int lane) {
  const unsigned group = __match_any_sync(0xffffffffu, addr);
  const uint32_t hi = (uint32_t)(key >> 32);
  const uint32_t mhi = __reduce_max_sync(group, hi);
  const uint32_t mlo = __reduce_max_sync(group, hi == mhi ? (uint32_t)key : 0u);
  if (lane == __ffs(group) - 1 && (mhi | mlo) != 0u) {
    const unsigned long long k = ((unsigned long long)mhi << 32) | mlo;
    asm volatile("atom.shared.max.u64 _, [%0], %1;" ::"r"(addr), "l"(k) : "memory");
  }
}

__device__ __forceinline__ int4 lds128(uint32_t a) {
  int4 v;
  asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a)
               : "memory");
  return v;
}
__device__ __forceinline__ void sts128(uint32_t a, int4 v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}

// The boxcar search of an item's top rows (Pt, search layout), all threads
// of the block together.  The stage's ops are the rows (dst = global row,
// p0 = the row in Pt, width = own columns W, col = history columns).
// Phase 1 takes (row, run of 16 columns) units, whole rows per wave, lane
// after lane along a row: a unit loads its run and the run before it, then
// (after a block barrier) writes the run's own columns to A, doubles four
// times in registers (widths 1 .. 16) and stores B_16 over its run in place
// (no later wave reads those rows).  Phase 2 takes (256-column group, row,
// residue) units over B_16 at stride 16 (widths 32 .. 256).  Each unit's
// best per width joins the row's best in shared memory (`best`, rows x
// widths words); the bests are written as the tile's partials.
template <class A, class TO>
__device__ __forceinline__ void stage_search_block(uint32_t sbase, const FusedOp *__restrict__ ops, int op0,
                                                   int op1, TO *__restrict__ out, int64_t nt, int64_t T0, int lim,
                                                   int64_t tile, const SearchArgs &sa) {
  const int tid = threadIdx.x, R = op1 - op0, nk = sa.nk;
  if (R <= 0) return;
  const uint32_t best = sbase + sa.q_off;
  for (int i = tid; i < R * nk; i += kFusedThreads)
    asm volatile("st.shared.u64 [%0], %1;" ::"r"(best + 8u * i), "l"(0ull) : "memory");
  const FusedOp op_first = ld_op(ops + op0);
  const int hist = op_first.col, n = op_first.width + hist, own_hi = hist + lim, runs = n >> 4;
  const int32_t t0 = (int32_t)(T0 - hist);  // time of window column 0
  const int per_wave = kFusedThreads / runs;  // whole rows per wave (runs <= kFusedThreads)
  __syncthreads();
  const int lane = tid & 31;
  for (int row0 = 0; row0 < R; row0 += per_wave) {
    const int ri = row0 + tid / runs, r = tid % runs;
    const bool valid = tid < per_wave * runs && ri < R;
    FusedOp op{};
    A x[32];
    uint32_t cur = 0;
    if (valid) {
      op = ld_op(ops + op0 + ri);
      cur = sbase + op.p0 + (uint32_t)(20 * r) * sizeof(A);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int4 hi = lds128(cur + 16u * v);
        const int4 lo = r > 0 ? lds128(cur - 80u + 16u * v) : make_int4(0, 0, 0, 0);
        const A *ph = reinterpret_cast<const A *>(&hi);
        const A *pl = reinterpret_cast<const A *>(&lo);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          x[16 + 4 * v + e] = ph[e];
          x[4 * v + e] = pl[e];
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) x[j] = A(0);
    }
    __syncthreads();  // the wave's rows are all loaded before any run is overwritten
    const int c0 = 16 * r;
    if (valid) {
      TO *arow = out + (int64_t)op.dst * nt + T0 - hist;
      if (c0 >= hist && c0 + 16 <= own_hi) {
        int4 *dv = reinterpret_cast<int4 *>(arow + c0);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          TO o[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) o[e] = to_store<TO>(x[16 + 4 * v + e]);
          dv[v] = *reinterpret_cast<const int4 *>(o);
        }
      } else {
#pragma unroll
        for (int e = 0; e < 16; ++e)
          if (c0 + e >= hist && c0 + e < own_hi) arow[c0 + e] = to_store<TO>(x[16 + e]);
      }
    }
    const bool owned = valid && c0 + 15 >= hist && c0 < own_hi;
    const uint32_t brow = best + 8u * (uint32_t)((valid ? ri : 0) * nk);
    search_join_warp(search_key<A, 1>(x, owned, c0, hist, own_hi, t0 + c0), brow, lane);
#pragma unroll
    for (int m = 1; m <= 4; ++m) {
      const int h = 1 << (m - 1);
#pragma unroll
      for (int j = 31; j >= (1 << m); --j) x[j] = acc_add(x[j], x[j - h]);
      if (m < nk) search_join_warp(search_key<A, 1>(x, owned, c0, hist, own_hi, t0 + c0), brow + 8u * m, lane);
    }
    if (nk > 5 && valid) {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        int4 o;
        A *po = reinterpret_cast<A *>(&o);
#pragma unroll
        for (int e = 0; e < 4; ++e) po[e] = x[16 + 4 * v + e];
        sts128(cur + 16u * v, o);
      }
    }
    __syncthreads();  // before the next wave (and phase 2) reads its rows
  }
  if (nk > 5) {
    const int groups = (n + 255) >> 8;
    const int U2 = R * groups * 16;
    for (int u0 = 0; u0 < U2; u0 += kFusedThreads) {
      const int u = u0 + tid;
      const int rho = u & 15, ri = (u >> 4) % R, g = (u >> 4) / R;
      const int base = 256 * g;
      // groups without an own column take no part (but every lane joins)
      const bool use = u < U2 && base + 256 > hist && base < own_hi;
      A x[32];
      uint32_t brow = best;
      if (use) {
        const FusedOp op = ld_op(ops + op0 + ri);
        const uint32_t row = sbase + op.p0;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int c = base + rho + 16 * (j - 16);
          x[j] = (c >= 0 && c < n) ? Lds<A>::get(row + (uint32_t)search_pidx(c) * sizeof(A)) : A(0);
        }
        brow = best + 8u * (uint32_t)(ri * nk);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) x[j] = A(0);
      }
#pragma unroll
      for (int m = 1; m <= 4; ++m) {
        const int h = 1 << (m - 1);
#pragma unroll
        for (int j = 31; j >= (1 << m); --j) x[j] = acc_add(x[j], x[j - h]);
        if (4 + m < nk)
          search_join_warp(search_key<A, 16>(x, use, base + rho, hist, own_hi, t0 + base), brow + 8u * (4 + m),
                           lane);
      }
    }
    __syncthreads();
  }
  // The row bests become the tile's partials.
  for (int i = tid; i < R * nk; i += kFusedThreads) {
    const int ri = i / nk, k = i - ri * nk;
    unsigned long long key;
    asm volatile("ld.shared.u64 %0, [%1];" : "=l"(key) : "r"(best + 8u * i) : "memory");
    const FusedOp op = ld_op(ops + op0 + ri);
    const int64_t slot = ((int64_t)op.dst * nk + k) * sa.nseg + tile;
    if (key == 0) {
      sa.part_r[slot] = kSearchNoRegion;
    } else {
      static_cast<A *>(sa.part_v)[slot] = search_value((uint32_t)(key >> 32), A());
      sa.part_r[slot] = 0x7fffffff - (int32_t)(uint32_t)key;
    }
  }
}

// The first stage of an item: level 1 walked from the staged input
// (FROM_INPUT) or the first single / pair stage over the staged base rows.
// TB is the staged base level's type and TO the type written to global
// memory when this stage is the top.  With SEARCH the stage before the
// search writes the top level into Pt instead.
// ds: the warp's descriptor stream, holding this item's first stage; it
// leaves holding the stage after it (this item's second, or the first of
// `next`, the template of the block's next item, if any).
// GEN as for run_merge_stage; SCALE: the input is multiplied by channel
// weights (float input only).
template <class TI, class TB, class A, class TO, bool R16, bool FROM_INPUT, bool SEARCH, bool GEN = true,
          bool SCALE = true>
__device__ __forceinline__ void item_first_stage(uint32_t sbase, const int32_t *__restrict__ stages,
                                                 const FusedTemplate &tp, const FusedWalk *__restrict__ walks,
                                                 const FusedOp *__restrict__ ops, const float *__restrict__ w,
                                                 int warp, int lane, TO *__restrict__ out, int64_t nt, int64_t T0,
                                                 int lim, DescStream &ds, const FusedTemplate *next) {
  ds.slot = desc_slot(sbase, tp, warp);
  const StageRange r = ds_take(ds);
  // (a walk keeps many sums in registers: its successor is requested after it)
  if (FROM_INPUT) ds_peek(ds, stages, nullptr, 0, warp);
  else if (tp.n_stages > 1) ds_peek(ds, stages, &tp, 1, warp);
  else ds_peek(ds, stages, next, 0, warp);
  const bool top = !SEARCH && tp.n_stages == 1;
  if constexpr (FROM_INPUT) {
    bool scaled = false;
    const bool gen = GEN && (r.kind & kStageGeneral) != 0;
    if constexpr (SCALE && std::is_floating_point<A>::value) {
      if (w != nullptr) {
        scaled = true;
        if (gen) {
          if (top) stage_walk<TI, A, TO, R16, true, true, true>(sbase, walks, ops, r.i0, r.i1, ds, lane, w, out, nt, T0, lim);
          else stage_walk<TI, A, TO, R16, true, false, true>(sbase, walks, ops, r.i0, r.i1, ds, lane, w, out, nt, T0, lim);
        } else {
          if (top) stage_walk<TI, A, TO, R16, true, true, false>(sbase, walks, ops, r.i0, r.i1, ds, lane, w, out, nt, T0, lim);
          else stage_walk<TI, A, TO, R16, true, false, false>(sbase, walks, ops, r.i0, r.i1, ds, lane, w, out, nt, T0, lim);
        }
      }
    }
    if (!scaled) {
      if (gen) {
        if (top) stage_walk<TI, A, TO, R16, false, true, true>(sbase, walks, ops, r.i0, r.i1, ds, lane, w, out, nt, T0, lim);
        else stage_walk<TI, A, TO, R16, false, false, true>(sbase, walks, ops, r.i0, r.i1, ds, lane, w, out, nt, T0, lim);
      } else {
        if (top) stage_walk<TI, A, TO, R16, false, true, false>(sbase, walks, ops, r.i0, r.i1, ds, lane, w, out, nt, T0, lim);
        else stage_walk<TI, A, TO, R16, false, false, false>(sbase, walks, ops, r.i0, r.i1, ds, lane, w, out, nt, T0, lim);
      }
    }
    if (tp.n_stages > 1) ds_peek(ds, stages, &tp, 1, warp);
    else ds_peek(ds, stages, next, 0, warp);
  } else if constexpr (SEARCH) {
    if (tp.n_stages == 2) run_merge_stage<TB, A, TO, R16, kOutPadded, GEN>(r, sbase, ds, ops, walks, lane, out, nt, T0, lim);
    else run_merge_stage<TB, A, TO, R16, kOutSmem, GEN>(r, sbase, ds, ops, walks, lane, out, nt, T0, lim);
  } else {
    if (top) run_merge_stage<TB, A, TO, R16, kOutGlobal, GEN>(r, sbase, ds, ops, walks, lane, out, nt, T0, lim);
    else run_merge_stage<TB, A, TO, R16, kOutSmem, GEN>(r, sbase, ds, ops, walks, lane, out, nt, T0, lim);
  }
}

// Stages 1 .. n - 1 of an item (sources in Pa / Pb), a block barrier after
// each stage but the last; the last writes global memory (with SEARCH: the
// one before it writes Pt and the last is the search).
// ds as for item_first_stage: it enters holding stage 1 and leaves holding
// the first stage of `next` (null: none).
template <class A, class TO, bool R16, bool SEARCH, bool GEN = true>
__device__ __forceinline__ void item_later_stages(uint32_t sbase, const int32_t *__restrict__ stages,
                                                  const FusedTemplate &tp, const FusedOp *__restrict__ ops,
                                                  const FusedWalk *__restrict__ walks, int warp, int lane,
                                                  TO *__restrict__ out, int64_t nt, int64_t T0, int lim, int64_t tile,
                                                  const SearchArgs &sa, DescStream &ds, const FusedTemplate *next) {
  ds.slot = desc_slot(sbase, tp, warp);
  for (int s = 1; s < tp.n_stages; ++s) {
    const StageRange r = ds_take(ds);
    if (s + 1 < tp.n_stages) ds_peek(ds, stages, &tp, s + 1, warp);
    else ds_peek(ds, stages, next, 0, warp);
    if constexpr (SEARCH) {
      if (s == tp.n_stages - 1) {
        // every thread: the whole stage's rows (warp 0's first to the end)
        const int32_t *p = stages + tp.stage_begin + s * kStageWords;
        stage_search_block<A, TO>(sbase, ops, __ldg(p + 1), __ldg(p + kStageWords - 1), out, nt, T0, lim, tile, sa);
      } else {
        if (s == tp.n_stages - 2) run_merge_stage<A, A, TO, R16, kOutPadded, GEN>(r, sbase, ds, ops, walks, lane, out, nt, T0, lim);
        else run_merge_stage<A, A, TO, R16, kOutSmem, GEN>(r, sbase, ds, ops, walks, lane, out, nt, T0, lim);
        __syncthreads();
      }
    } else {
      if (s == tp.n_stages - 1) {
        run_merge_stage<A, A, TO, R16, kOutGlobal, GEN>(r, sbase, ds, ops, walks, lane, out, nt, T0, lim);
      } else {
        run_merge_stage<A, A, TO, R16, kOutSmem, GEN>(r, sbase, ds, ops, walks, lane, out, nt, T0, lim);
        __syncthreads();
      }
    }
  }
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

}  // namespace fdmt
