// Batched FDMT of independent beams with the fused schedule in ONE
// persistent launch (contracts in include/fdmt.h, fdmt_plan_batch with
// schedule = 1).
//
// Each beam is planned as in the single-beam fused schedule: level groups
// (lb, lt] whose work items are cones (a row range of a band of level lt and
// a time tile, section 4's addition rule unrolled down to level lb).  The
// items of all beams form one list in group-major order: every beam's first
// group (from the input), then every beam's second group, and so on.  A
// block takes the next item from a global counter; an item of group g > 0
// needs every item of group g - 1 of its beam done (a per-(beam, group)
// counter).  Producers precede their consumers in the list and a block only
// waits before it starts an item, never inside one, so a wait can only run
// out if a producer is missing; each wait is bounded by the global timer,
// and one that runs out stops the launch through a status word.
//
// Staged rows are read by TMA (the async proxy) from state other blocks
// wrote with ordinary stores: the waiting thread acquires the producer
// counter and the copying lanes issue a proxy fence before their copies.
// While an item computes, the next item's rows are staged into the same
// buffer early when it belongs to the same (beam, group) segment (same
// shared-memory layout, producers already done); otherwise they are staged
// once the current item is complete.
#include "fdmt_batch_fused.h"

#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fdmt_fused.h"
#include "fdmt_fused_dev.cuh"
#include "fdmt_tma.h"

namespace fdmt {
namespace {

constexpr int kMaxGroups = 16;
constexpr int kMapsPerSeg = kMaxBlockP + 1;

// One (beam, level group) of the work list.
struct BSeg {
  int64_t first;  // first global item
  int64_t nt;
  void *out;      // the group's top level: the beam's output or a workspace buffer
  int32_t beam, group, from_input, ntpl;
  int32_t ntiles, W, tpl_begin, box;  // tpl_begin: global template index
  int32_t cshift, map, need, done_idx;
  int32_t dep_idx, in_size, out_size;  // bytes per staged / written sample
  int32_t s_end;  // end of the group's staging region in shared memory
};

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int find_seg(const BSeg *__restrict__ segs, int nsegs, int64_t item, int from) {
  int s = from;
  while (s + 1 < nsegs && segs[s + 1].first <= item) ++s;
  return s;
}

// Staged sample types: the input for the first group, else the state
// (uint16 for integer levels stored narrow).
template <class TI, class TB>
__device__ __forceinline__ void stage_seg_item(unsigned char *smem, uint32_t bar, const BSeg *__restrict__ sg,
                                               const CUtensorMap *__restrict__ maps, const FusedTemplate &tp,
                                               const FusedLoad *__restrict__ loads, const FusedLoad &first,
                                               int64_t T0, int lane) {
  const CUtensorMap *m = maps + sg->map;
  if (sg->from_input)
    stage_item<TI>(smem, bar, m, tp, loads, first, T0, sg->box, sg->cshift, lane);
  else if (std::is_same<TB, int32_t>::value && sg->in_size == 2)
    stage_item<uint16_t>(smem, bar, m, tp, loads, first, T0, sg->box, sg->cshift, lane);
  else
    stage_item<TB>(smem, bar, m, tp, loads, first, T0, sg->box, sg->cshift, lane);
}

// The first stage of an item with the segment's runtime types: the input
// or the staged base level (uint16 for narrow integer state) in, the
// group's top type out when it is the only stage.
// GEN: some beam's plan has pass-through stages (as for the single-beam
// kernel); the batch has no channel weights.
template <class TI, class TB, class A, bool GEN>
__device__ __forceinline__ void batch_first_stage(bool from_input, bool i16, bool o16, uint32_t bar,
                                                  const int32_t *__restrict__ stages, const FusedTemplate &tp,
                                                  const FusedWalk *__restrict__ walks, const FusedOp *__restrict__ ops,
                                                  int warp, int lane, void *out, int64_t nt, int64_t T0, int lim,
                                                  DescStream &ds, const FusedTemplate *next) {
  TB *o = static_cast<TB *>(out);
  if constexpr (std::is_same<TB, int32_t>::value) {
    uint16_t *o_16 = static_cast<uint16_t *>(out);
    if (from_input) {
      if (o16)
        item_first_stage<TI, TB, A, uint16_t, false, true, false, GEN, false>(
            bar, stages, tp, walks, ops, nullptr, warp, lane, o_16, nt, T0, lim, ds, next);
      else
        item_first_stage<TI, TB, A, TB, false, true, false, GEN, false>(bar, stages, tp, walks, ops, nullptr, warp,
                                                                        lane, o, nt, T0, lim, ds, next);
    } else if (i16 && o16) {
      item_first_stage<TI, uint16_t, A, uint16_t, false, false, false, GEN, false>(
          bar, stages, tp, walks, ops, nullptr, warp, lane, o_16, nt, T0, lim, ds, next);
    } else if (i16) {
      item_first_stage<TI, uint16_t, A, TB, false, false, false, GEN, false>(bar, stages, tp, walks, ops, nullptr,
                                                                             warp, lane, o, nt, T0, lim, ds, next);
    } else {
      item_first_stage<TI, TB, A, TB, false, false, false, GEN, false>(bar, stages, tp, walks, ops, nullptr, warp,
                                                                       lane, o, nt, T0, lim, ds, next);
    }
  } else {
    if (from_input)
      item_first_stage<TI, TB, A, TB, false, true, false, GEN, false>(bar, stages, tp, walks, ops, nullptr, warp,
                                                                      lane, o, nt, T0, lim, ds, next);
    else
      item_first_stage<TI, TB, A, TB, false, false, false, GEN, false>(bar, stages, tp, walks, ops, nullptr, warp,
                                                                       lane, o, nt, T0, lim, ds, next);
  }
}

template <class TI, class TB, class A, bool GEN>
__global__ void __launch_bounds__(kFusedThreads, kFusedMinBlocks)
batch_fused_kernel(const BSeg *__restrict__ segs, int nsegs, int64_t total, const CUtensorMap *__restrict__ maps,
                   const FusedTemplate *__restrict__ tpls, const FusedLoad *__restrict__ loads,
                   const FusedWalk *__restrict__ walks, const FusedOp *__restrict__ ops,
                   const int32_t *__restrict__ stages, unsigned long long *__restrict__ counter,
                   int *__restrict__ done, int *__restrict__ status, uint64_t wait_ns) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t bar = smem_u32(smem);
  // Block-wide scalars in the 128-byte barrier slot, after the mbarrier.
  volatile long long *s_item = reinterpret_cast<volatile long long *>(smem + 16);
  volatile long long *s_next = reinterpret_cast<volatile long long *>(smem + 24);
  volatile int *s_ok = reinterpret_cast<volatile int *>(smem + 32);
  volatile int *s_early = reinterpret_cast<volatile int *>(smem + 36);

  // Item indices come from the global counter one item ahead: while item i
  // computes, the block already knows item i + 1 (its descriptors and copies
  // are prepared) and fetches the index of item i + 2.
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    *s_item = (long long)atomicAdd(counter, 1ull);
    *s_next = (long long)atomicAdd(counter, 1ull);
  }
  __syncthreads();
  int64_t item = *s_item;
  int64_t next = *s_next;
  if (item >= total) return;
  int si = find_seg(segs, nsegs, item, 0);
  FusedTemplate cur;
  {
    const int32_t local = (int32_t)(item - segs[si].first);
    cur = tpls[segs[si].tpl_begin + local / segs[si].ntiles];
  }
  uint32_t phase = 0;
  bool staged = false;  // this item's copies were issued while the previous item computed
  DescStream ds;
  ds.slot = desc_slot(smem_u32(smem), cur, warp);
  ds_peek(ds, stages, &cur, 0, warp);
  // The previous item's completion, published off the critical path: by
  // thread 32 while the block waits for the next item's copies, or by
  // thread 0 before it waits for producers (so that it never waits on
  // itself).
  int pending = -1;
  auto publish = [&]() {
    __threadfence();
    atomicAdd(done + pending, 1);
  };
  for (;;) {
    const BSeg *sg = segs + si;
    const int32_t ntiles = sg->ntiles, W = sg->W;
    const bool from_input = sg->from_input != 0;
    const int64_t nt = sg->nt;
    const int64_t T0 = (int64_t)((int32_t)(item - sg->first) % ntiles) * W;
    // The next item: its segment, template and (warp 0) copy descriptors.
    int nsi = si;
    FusedTemplate tpn = FusedTemplate{0, 0, 0, 0, 0, 0, 0, 0};
    int32_t nl = 0;
    if (next < total) {
      nsi = find_seg(segs, nsegs, next, si);
      nl = (int32_t)(next - segs[nsi].first);
      tpn = tpls[segs[nsi].tpl_begin + nl / segs[nsi].ntiles];
    }
    // The next item's copies go out during this item when its producers are
    // done (always within the same segment; else its previous group's
    // counter says so) and its staging region fits inside this item's,
    // which is free once the first stage has run.
    if (threadIdx.x == 0) {
      int e = 0;
      if (next < total) {
        const BSeg &ns = segs[nsi];
        if (nsi == si) e = 1;
        else if (ns.s_end <= sg->s_end && (ns.group == 0 || ld_acquire(done + ns.dep_idx) >= ns.need)) e = 1;
      }
      *s_early = e;
    }
    FusedLoad ldn = FusedLoad{0, 0, 0, 0};
    if (warp == 0 && next < total) ldn = fetch_load(tpn, loads, lane);
    if (!staged) {
      // The item's producers: every item of the previous group of its beam.
      if (threadIdx.x == 0) {
        if (pending >= 0) publish();
        int ok = 1;
        if (sg->group > 0) {
          const int *d = done + sg->dep_idx;
          const int need = sg->need;
          const uint64_t t0 = global_ns();
          while (ld_acquire(d) < need) {
            if (*(volatile int *)status != 0 || global_ns() - t0 > wait_ns) {
              atomicExch(status, 1);
              ok = 0;
              break;
            }
            __nanosleep(256);
          }
        }
        *s_ok = ok;
      }
      pending = -1;
      __syncthreads();
      if (!*s_ok) return;
      if (warp == 0) {
        // Rows written by other blocks with generic stores, read by TMA.
        asm volatile("fence.proxy.async.global;" ::: "memory");
        stage_seg_item<TI, TB>(smem, bar, sg, maps, cur, loads, fetch_load(cur, loads, lane), T0, lane);
      }
    }
    long long nn = 0;  // the item after next
    if (threadIdx.x == 0) nn = (long long)atomicAdd(counter, 1ull);
    if (threadIdx.x == 32 && pending >= 0) publish();
    pending = -1;
    if (!mbar_wait_bounded(bar, phase)) {
      atomicExch(status, 1);
      mbar_wait_bounded(bar, phase);
      return;
    }
    phase ^= 1u;
    const int lim = (int)((nt - T0) < (int64_t)W ? (nt - T0) : (int64_t)W);
    // Integer state stored as uint16 on either side of this group.
    constexpr bool kNarrow = std::is_same<TB, int32_t>::value;
    const bool i16 = kNarrow && sg->in_size == 2, o16 = kNarrow && sg->out_size == 2;
    const FusedTemplate tp = cur;
    batch_first_stage<TI, TB, A, GEN>(from_input, i16, o16, bar, stages, tp, walks, ops, warp, lane, sg->out, nt, T0,
                                 lim, ds, next < total ? &tpn : nullptr);
    __syncthreads();  // the staged rows are no longer read; s_early is visible
    const bool early = *s_early != 0;
    if (early && warp == 0) {
      const BSeg *nsg = segs + nsi;
      // rows written by other blocks with generic stores, read by TMA
      if (nsi != si) asm volatile("fence.proxy.async.global;" ::: "memory");
      stage_seg_item<TI, TB>(smem, bar, nsg, maps, tpn, loads, ldn, (int64_t)(nl % nsg->ntiles) * nsg->W, lane);
    }
    if (next < total) cur = tpn;
    const SearchArgs no_search{};
    if (kNarrow && o16)
      item_later_stages<A, uint16_t, false, false, GEN>(bar, stages, tp, ops, walks, warp, lane,
                                                        static_cast<uint16_t *>(sg->out), nt, T0, lim, 0, no_search,
                                                        ds, next < total ? &tpn : nullptr);
    else
      item_later_stages<A, TB, false, false, GEN>(bar, stages, tp, ops, walks, warp, lane, static_cast<TB *>(sg->out),
                                                  nt, T0, lim, 0, no_search, ds, next < total ? &tpn : nullptr);
    if (threadIdx.x == 0) *s_next = nn;
    __syncthreads();  // all of this item's stores are issued; Pa / Pb are free; s_next is visible
    pending = sg->done_idx;
    if (next >= total) {
      if (threadIdx.x == 0) publish();
      return;
    }
    item = next;
    si = nsi;
    next = *s_next;
    staged = early;
  }
}

template <class TI, class TB, class A>
void *kernel_ptr(bool gen) {
  return gen ? reinterpret_cast<void *>(batch_fused_kernel<TI, TB, A, true>)
             : reinterpret_cast<void *>(batch_fused_kernel<TI, TB, A, false>);
}

// The kernel variant of a batch: its input type, and whether any beam's plan
// has pass-through stages.
void *kernel_for(int dtype, bool gen) {
  return dtype == FDMT_U8_I32 ? kernel_ptr<uint8_t, int32_t, int32_t>(gen) : kernel_ptr<float, float, float>(gen);
}

int64_t rup(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

}  // namespace

struct FusedBatch {
  int n = 0, dtype = 0, device = -1;
  fdmt_batch_params prm{};
  std::vector<fdmt_beam_desc> desc;
  std::vector<FusedPlan> plans;
  std::vector<std::vector<int32_t>> level_rows;
  std::vector<std::vector<int32_t>> tpl_base;  // [beam][group] global index of the group's first template
  std::vector<size_t> ws_off;
  size_t ws_bytes = 0;
  std::vector<BSeg> segs;
  int64_t total = 0;
  int smem_bytes = 0, grid = 0;
  bool general = false;  // some beam's plan has pass-through stages
  // device
  FusedTemplate *d_tpls = nullptr;
  FusedLoad *d_loads = nullptr;
  FusedWalk *d_walks = nullptr;
  FusedOp *d_ops = nullptr;
  int32_t *d_lops = nullptr;
  BSeg *d_segs = nullptr;
  CUtensorMap *d_maps = nullptr;
  unsigned long long *d_counter = nullptr;
  int *d_done = nullptr;
  int *d_status = nullptr;
  // recorded launch for one set of pointers
  std::vector<const void *> key;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

void release(FusedBatch *fb) {
  if (fb->exec) cudaGraphExecDestroy(fb->exec);
  if (fb->graph) cudaGraphDestroy(fb->graph);
  void *ptrs[] = {fb->d_tpls, fb->d_loads, fb->d_walks, fb->d_ops, fb->d_lops, fb->d_segs,
                  fb->d_maps, fb->d_counter, fb->d_done, fb->d_status};
  for (void *p : ptrs)
    if (p) cudaFree(p);
}

template <class T>
cudaError_t upload(const std::vector<T> &v, T **dst) {
  *dst = nullptr;
  if (v.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(dst), v.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// Group-major work list, leaving out (drop_beam, drop_group).
void build_segments(FusedBatch *fb, int drop_beam, int drop_group) {
  size_t max_g = 0;
  for (const FusedPlan &fp : fb->plans) max_g = std::max(max_g, fp.groups.size());
  fb->segs.clear();
  int64_t first = 0;
  for (size_t g = 0; g < max_g; ++g)
    for (int b = 0; b < fb->n; ++b) {
      const FusedPlan &fp = fb->plans[b];
      if (g >= fp.groups.size() || (b == drop_beam && (int)g == drop_group)) continue;
      const FusedGroup &gr = fp.groups[g];
      BSeg s{};
      s.first = first;
      s.nt = fb->desc[b].nt;
      s.beam = b;
      s.group = (int32_t)g;
      s.from_input = gr.from_input ? 1 : 0;
      s.ntpl = gr.tpl_count;
      s.ntiles = (int32_t)gr.ntiles;
      s.W = gr.W;
      s.tpl_begin = fb->tpl_base[b][g];
      s.box = gr.box;
      s.in_size = gr.in_size;
      s.out_size = gr.out_size;
      s.s_end = gr.s_end;
      s.map = (int32_t)(fb->segs.size() * kMapsPerSeg);
      s.done_idx = b * kMaxGroups + (int32_t)g;
      if (g > 0) {
        const FusedGroup &pg = fp.groups[g - 1];
        s.need = (int32_t)((int64_t)pg.tpl_count * pg.ntiles);
        s.dep_idx = b * kMaxGroups + (int32_t)g - 1;
      }
      fb->segs.push_back(s);
      first += (int64_t)gr.tpl_count * gr.ntiles;
    }
  fb->total = first;
}

}  // namespace

int fused_batch_create(const std::vector<fdmt_beam_desc> &desc, const std::vector<Tables> &tabs, int dtype,
                       const fdmt_batch_params &prm, FusedBatch **out) {
  *out = nullptr;
  if (dtype != FDMT_U8_I32 && dtype != FDMT_F32_F32) return FDMT_ERR_UNSUPPORTED;
  FusedBatch *fb = new (std::nothrow) FusedBatch();
  if (fb == nullptr) return FDMT_ERR_NO_MEMORY;
  fb->n = (int)desc.size();
  fb->dtype = dtype;
  fb->prm = prm;
  fb->desc = desc;
  fb->plans.resize(fb->n);
  fb->level_rows.resize(fb->n);
  fb->tpl_base.resize(fb->n);
  fb->ws_off.resize(fb->n);
  const int32_t in_size = dtype == FDMT_U8_I32 ? 1 : 4;
  FusedParams fpar;
  fpar.narrow = (dtype == FDMT_U8_I32);
  fpar.W = prm.fused_tile;
  fpar.smem_budget = prm.smem_budget > 0 ? prm.smem_budget : 72 * 1024;
  std::vector<FusedTemplate> tpls;
  std::vector<FusedLoad> loads;
  std::vector<FusedWalk> walks;
  std::vector<FusedOp> ops;
  std::vector<int32_t> lops;
  size_t ws = 0;
  for (int b = 0; b < fb->n; ++b) {
    FusedPlan &fp = fb->plans[b];
    int same = -1;  // an earlier beam of the same shape: its programme is reused
    for (int c = 0; c < b && same < 0; ++c)
      if (desc[c].f_min == desc[b].f_min && desc[c].f_max == desc[b].f_max && desc[c].nf == desc[b].nf &&
          desc[c].nt == desc[b].nt && desc[c].nd == desc[b].nd)
        same = c;
    if (same >= 0) {
      fp = fb->plans[same];
    } else if (!plan_fused(tabs[b], desc[b].nt, 4, in_size, fpar, fp).empty() ||
               fp.groups.size() > kMaxGroups) {
      delete fb;
      return FDMT_ERR_UNSUPPORTED;
    }
    fb->level_rows[b] = tabs[b].level_rows;
    fb->general |= fp.general;
    const int32_t t_off = (int32_t)tpls.size(), l_off = (int32_t)loads.size();
    const int32_t w_off = (int32_t)walks.size(), o_off = (int32_t)ops.size();
    const int32_t lo_off = (int32_t)lops.size();
    for (FusedTemplate tp : fp.tpls) {
      tp.load_begin += l_off;
      tp.walk_begin += w_off;
      tp.stage_begin += lo_off;
      tpls.push_back(tp);
    }
    loads.insert(loads.end(), fp.loads.begin(), fp.loads.end());
    walks.insert(walks.end(), fp.walks.begin(), fp.walks.end());
    ops.insert(ops.end(), fp.ops.begin(), fp.ops.end());
    // Stage words: the kind, then indices into the walks (kind 0) or ops.
    for (size_t i = 0; i < fp.stages.size(); i += kStageWords) {
      lops.push_back(fp.stages[i]);
      const int32_t off = (fp.stages[i] & kStageKindMask) == kStageWalk ? w_off : o_off;
      for (int32_t k = 1; k < kStageWords; ++k) lops.push_back(fp.stages[i + k] + off);
    }
    for (const FusedGroup &g : fp.groups) {
      fb->tpl_base[b].push_back(t_off + g.tpl_begin);
      fb->smem_bytes = std::max(fb->smem_bytes, g.smem_bytes);
    }
    fb->ws_off[b] = ws;
    ws += (size_t)rup((int64_t)fp.ws_bytes, 256);
  }
  fb->ws_bytes = ws;
  if (tpls.size() >= ((size_t)1 << 31) || ops.size() >= ((size_t)1 << 31)) {
    delete fb;
    return FDMT_ERR_UNSUPPORTED;
  }
  build_segments(fb, -1, -1);
  cudaError_t e = cudaGetDevice(&fb->device);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel_for(dtype, fb->general), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             fb->smem_bytes);
  int per_sm = 0, sms = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel_for(dtype, fb->general), kFusedThreads,
                                                      fb->smem_bytes);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, fb->device);
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    delete fb;
    return FDMT_ERR_CUDA;
  }
  if (prm.blocks_per_sm > 0) per_sm = std::min(per_sm, prm.blocks_per_sm);
  fb->grid = per_sm * sms;
  e = upload(tpls, &fb->d_tpls);
  if (e == cudaSuccess) e = upload(loads, &fb->d_loads);
  if (e == cudaSuccess) e = upload(walks, &fb->d_walks);
  if (e == cudaSuccess) e = upload(ops, &fb->d_ops);
  if (e == cudaSuccess) e = upload(lops, &fb->d_lops);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&fb->d_counter), sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&fb->d_done), sizeof(int) * (size_t)fb->n * kMaxGroups);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&fb->d_status), sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(fb->d_status, 0, sizeof(int));
  if (e != cudaSuccess) {
    release(fb);
    delete fb;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? FDMT_ERR_NO_MEMORY : FDMT_ERR_CUDA;
  }
  *out = fb;
  return FDMT_OK;
}

void fused_batch_destroy(FusedBatch *fb) {
  if (fb == nullptr) return;
  release(fb);
  delete fb;
}

size_t fused_batch_workspace(const FusedBatch *fb) { return fb->ws_bytes; }

std::vector<int32_t> fused_batch_sizes(const FusedBatch *fb, int b) {
  std::vector<int32_t> v;
  const FusedPlan &fp = fb->plans[b];
  if (fp.groups.empty()) return v;
  v.push_back(fp.groups.front().in_size);
  for (const FusedGroup &g : fp.groups) v.push_back(g.out_size);
  return v;
}

std::vector<int32_t> fused_batch_bounds(const FusedBatch *fb, int b) {
  std::vector<int32_t> v;
  const FusedPlan &fp = fb->plans[b];
  if (fp.groups.empty()) return v;
  v.push_back(fp.groups.front().lb);
  for (const FusedGroup &g : fp.groups) v.push_back(g.lt);
  return v;
}

int fused_batch_drop(FusedBatch *fb, int beam, int group) {
  if (group == -1) {
    build_segments(fb, -1, -1);
  } else {
    if (beam < 0 || beam >= fb->n || group < 0 || group >= (int)fb->plans[beam].groups.size())
      return FDMT_ERR_INVALID_ARG;
    build_segments(fb, beam, group);
  }
  fb->key.clear();  // the recorded launch refers to the old list
  return FDMT_OK;
}

int fused_batch_execute(FusedBatch *fb, const void *const *in, void *const *out, void *workspace,
                        cudaStream_t s) {
  std::vector<const void *> key;
  key.push_back(workspace);
  for (int i = 0; i < fb->n; ++i) {
    key.push_back(in[i]);
    key.push_back(out[i]);
  }
  cudaError_t e = cudaSuccess;
  if (key != fb->key || fb->exec == nullptr) {
    // New pointers or a new work list: segment outputs and tensor maps,
    // then record the launch.
    std::vector<CUtensorMap> maps(fb->segs.size() * kMapsPerSeg);
    const uint32_t in_elem = fb->dtype == FDMT_U8_I32 ? 1 : 4;
    const CUtensorMapDataType in_type = fb->dtype == FDMT_U8_I32 ? map_type<uint8_t>() : map_type<float>();
    const CUtensorMapDataType st_type = fb->dtype == FDMT_U8_I32 ? map_type<int32_t>() : map_type<float>();
    for (size_t k = 0; k < fb->segs.size(); ++k) {
      BSeg &sg = fb->segs[k];
      const int b = sg.beam, g = sg.group;
      const FusedPlan &fp = fb->plans[b];
      const FusedGroup &gr = fp.groups[g];
      char *w = static_cast<char *>(workspace) + fb->ws_off[b];
      void *bufs[2] = {w, w + fp.ws_split};
      sg.out = (g + 1 == (int)fp.groups.size()) ? out[b] : bufs[g & 1];
      const void *base = g == 0 ? in[b] : bufs[(g - 1) & 1];
      const uint64_t rows = g == 0 ? (uint64_t)fb->desc[b].nf : (uint64_t)fb->level_rows[b][gr.lb];
      int32_t cshift = 0;
      const bool narrow_in = fb->dtype == FDMT_U8_I32 && gr.in_size == 2;
      if (!make_group_maps(&maps[k * kMapsPerSeg], gr, base,
                           g == 0 ? in_type : (narrow_in ? map_type<uint16_t>() : st_type),
                           g == 0 ? in_elem : (uint32_t)gr.in_size,
                           rows, (uint64_t)fb->desc[b].nt, &cshift)) {
        fb->key.clear();
        return FDMT_ERR_INVALID_ARG;
      }
      sg.cshift = cshift;
    }
    if (fb->d_segs) cudaFree(fb->d_segs);
    if (fb->d_maps) cudaFree(fb->d_maps);
    fb->d_segs = nullptr;
    fb->d_maps = nullptr;
    e = upload(fb->segs, &fb->d_segs);
    if (e == cudaSuccess) e = upload(maps, &fb->d_maps);
    if (fb->exec) cudaGraphExecDestroy(fb->exec);
    if (fb->graph) cudaGraphDestroy(fb->graph);
    fb->exec = nullptr;
    fb->graph = nullptr;
    cudaStream_t cap = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t le = cudaMemsetAsync(fb->d_counter, 0, sizeof(unsigned long long), cap);
      if (le == cudaSuccess) le = cudaMemsetAsync(fb->d_done, 0, sizeof(int) * (size_t)fb->n * kMaxGroups, cap);
      if (le == cudaSuccess) {
        const int nsegs = (int)fb->segs.size();
        const uint64_t wait_ns = (uint64_t)fb->prm.wait_ms * 1000000ull;
        void *args[] = {&fb->d_segs, (void *)&nsegs, &fb->total, &fb->d_maps, &fb->d_tpls, &fb->d_loads,
                        &fb->d_walks, &fb->d_ops, &fb->d_lops, &fb->d_counter, &fb->d_done, &fb->d_status,
                        (void *)&wait_ns};
        le = cudaLaunchKernel(kernel_for(fb->dtype, fb->general), dim3(fb->grid), dim3(kFusedThreads), args,
                              (size_t)fb->smem_bytes, cap);
      }
      e = cudaStreamEndCapture(cap, &fb->graph);
      if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&fb->exec, fb->graph, 0);
    if (cap) cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fb->key.clear();
      return FDMT_ERR_CUDA;
    }
    fb->key = key;
  }
  int status = 0;
  e = cudaGraphLaunch(fb->exec, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, fb->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cudaGetLastError(), FDMT_ERR_CUDA;
  if (status != 0) {
    const int zero = 0;
    if (cudaMemcpy(fb->d_status, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
      return cudaGetLastError(), FDMT_ERR_CUDA;
    return FDMT_ERR_TIMEOUT;
  }
  return FDMT_OK;
}

}  // namespace fdmt
