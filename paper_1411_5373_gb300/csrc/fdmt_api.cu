// C ABI of the FDMT library (declarations and contracts in include/fdmt.h).
//
// Argument checking, plan ownership (host tables + device tables), workspace
// layout and dispatch to the kernel launchers.  No entry point except
// fdmt_plan allocates device memory.
#include <cuda_runtime.h>

#include <climits>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>

#include "../../include/fdmt.h"
#include "fdmt_internal.h"
#include "fdmt_tables.h"

using fdmt::DeviceTables;
using fdmt::Tables;

struct fdmt_plan_s {
  double f_min = 0, f_max = 0;
  int32_t nf = 0, nd = 0, dtype = 0;
  int64_t nt = 0;
  uint32_t flags = 0;
  int device = -1;
  Tables host;
  DeviceTables dev;
  fdmt::Profiler prof;
  fdmt::FusedPlan fused;
  bool has_fused = false;
  fdmt::AdjFusedPlan adj_fused;  // fused adjoint (fused float plans)
  bool has_adj_fused = false;
  size_t adj_part_off = 0;       // its weight-gradient partials in the adjoint workspace
  size_t ws_bytes = 0;      // forward workspace
  size_t adj_ws_bytes = 0;  // adjoint workspace
  size_t ws_split = 0;      // offset of the second ping-pong buffer (forward)
  size_t adj_ws_split = 0;
  size_t fused_ws_bytes = 0;  // forward workspace of the fused schedule
  size_t fused_ws_split = 0;
  // Boxcar search in the last fused launch: widths, partial slots per
  // (row, width) and where the partials sit in the forward workspace.
  int32_t search_k = 0, search_nseg = 0;
  size_t part_off = 0, part_bytes = 0;
  // Input mapping (d_min pre-shift, descending channel order): the mapped
  // input (forward) or the mapped gradient and input (adjoint) follow the
  // schedule's own workspace.
  bool mapped = false;
  int32_t d_min = 0, descending = 0;
  std::vector<int32_t> in_shift;
  size_t map_off = 0, map_bytes = 0;          // forward
  size_t adj_map_off = 0, adj_map_bytes = 0;  // adjoint (two float planes)
};

namespace {

constexpr size_t kAlign = 256;

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

size_t input_elem(int dtype) { return dtype == FDMT_U8_I32 ? 1 : 4; }
size_t state_elem(int dtype) { return dtype == FDMT_F32_F16STATE ? 2 : 4; }

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Ping-pong split of a workspace holding levels [0, last] (last < L) with the
// given element size: even levels at offset 0, odd levels after them.
void pingpong_sizes(const Tables &t, int64_t nt, size_t elem, int last, size_t *split, size_t *total) {
  size_t even = 0, odd = 0;
  for (int l = 0; l <= last; ++l) {
    const size_t b = (size_t)t.level_rows[l] * (size_t)nt * elem;
    if (l & 1) odd = b > odd ? b : odd; else even = b > even ? b : even;
  }
  *split = round_up(even, kAlign);
  *total = *split + round_up(odd, kAlign);
}

// Adjoint workspace: step k of the transposed programme (two levels per
// step from level L down, one for a last odd level) writes buffer k % 2.
void adjoint_ws_sizes(const Tables &t, int64_t nt, size_t *split, size_t *total) {
  size_t sz[2] = {0, 0};
  int k = 0;
  for (int l = t.levels; l >= 1; l -= (l >= 2 ? 2 : 1), ++k) {
    const int child = l >= 2 ? l - 2 : l - 1;
    const size_t b = (size_t)t.level_rows[child] * (size_t)nt * sizeof(float);
    sz[k & 1] = b > sz[k & 1] ? b : sz[k & 1];
  }
  *split = round_up(sz[0], kAlign);
  *total = *split + round_up(sz[1], kAlign);
}

template <class T>
cudaError_t upload(const std::vector<T> &v, T **dst) {
  *dst = nullptr;
  if (v.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(dst), v.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

void profile_release(fdmt::Profiler &pr) {
  for (cudaEvent_t e : pr.start) cudaEventDestroy(e);
  for (cudaEvent_t e : pr.stop) cudaEventDestroy(e);
  pr.start.clear();
  pr.stop.clear();
  pr.kernel.clear();
  pr.level.clear();
  pr.next = 0;
}

void free_device(fdmt_plan_s *p) {
  DeviceTables &d = p->dev;
  void *ptrs[] = {d.init, d.ops, d.adj, d.adj2, d.adj2_terms, d.status, d.f_tpls, d.f_loads, d.f_walks,
                  d.f_ops, d.f_stages, d.in_shift, d.a_tpls, d.a_loads, d.a_ops, d.a_stages};
  for (void *q : ptrs)
    if (q) cudaFree(q);
  d.init = nullptr;
  d.ops = nullptr;
  d.adj = nullptr;
  d.adj2 = nullptr;
  d.adj2_terms = nullptr;
  d.status = nullptr;
  d.f_tpls = nullptr;
  d.f_loads = nullptr;
  d.f_walks = nullptr;
  d.f_ops = nullptr;
  d.f_stages = nullptr;
  d.in_shift = nullptr;
  d.a_tpls = nullptr;
  d.a_loads = nullptr;
  d.a_ops = nullptr;
  d.a_stages = nullptr;
}

int check_exec_common(fdmt_plan_t plan, void *workspace, size_t ws_bytes, size_t need) {
  if (plan == nullptr) return FDMT_ERR_INVALID_ARG;
  if (plan->flags & FDMT_PLAN_HOST_ONLY) return FDMT_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return FDMT_ERR_CUDA;
  if (dev != plan->device) return FDMT_ERR_INVALID_ARG;
  if (need > 0 && (workspace == nullptr || ws_bytes < need)) return FDMT_ERR_WORKSPACE;
  if (workspace != nullptr && (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0)
    return FDMT_ERR_INVALID_ARG;
  return FDMT_OK;
}

}  // namespace

extern "C" {

int fdmt_plan(double f_min, double f_max, int32_t nf, int64_t nt, int32_t nd, int32_t dtype,
              uint32_t flags, fdmt_plan_t *out) {
  return fdmt_plan_ex(f_min, f_max, nf, nt, nd, dtype, flags, nullptr, out);
}

int fdmt_plan_ex(double f_min, double f_max, int32_t nf, int64_t nt, int32_t nd, int32_t dtype,
                 uint32_t flags, const fdmt_schedule_params *params, fdmt_plan_t *out) {
  return fdmt_plan_curve(f_min, f_max, nf, nt, nd, dtype, flags, nullptr, params, out);
}

int fdmt_plan_curve(double f_min, double f_max, int32_t nf, int64_t nt, int32_t nd, int32_t dtype,
                    uint32_t flags, const fdmt_curve_params *curve, const fdmt_schedule_params *params,
                    fdmt_plan_t *out) {
  if (out == nullptr) return FDMT_ERR_INVALID_ARG;
  const double gamma = curve != nullptr ? curve->gamma : -2.0;
  if (!std::isfinite(gamma) || gamma == 0.0) return FDMT_ERR_INVALID_ARG;
  const int32_t d_min = curve != nullptr ? curve->d_min : 0;
  const int32_t descending = curve != nullptr ? curve->descending : 0;
  if (d_min < 0 || d_min > (1 << 30) || descending < 0 || descending > 1) return FDMT_ERR_INVALID_ARG;
  *out = nullptr;
  if (dtype != FDMT_U8_I32 && dtype != FDMT_F32_F32 && dtype != FDMT_F32_F16STATE)
    return FDMT_ERR_INVALID_ARG;
  if (flags & ~(uint32_t)(FDMT_PLAN_HOST_ONLY | FDMT_SCHED_FUSED)) return FDMT_ERR_INVALID_ARG;
  if (!std::isfinite(f_min) || !std::isfinite(f_max) || !(f_min > 0.0) || !(f_max > f_min))
    return FDMT_ERR_INVALID_ARG;
  if (nf < 2) return FDMT_ERR_INVALID_ARG;
  if (nd < 1 || nt < 1 || (int64_t)nd > nt) return FDMT_ERR_INVALID_ARG;
  if ((nt * (int64_t)input_elem(dtype)) % 16 != 0 || (nt * (int64_t)state_elem(dtype)) % 16 != 0)
    return FDMT_ERR_INVALID_ARG;
  if (nt > ((int64_t)1 << 40)) return FDMT_ERR_INVALID_ARG;

  fdmt_plan_s *p = new (std::nothrow) fdmt_plan_s();
  if (p == nullptr) return FDMT_ERR_NO_MEMORY;
  p->f_min = f_min;
  p->f_max = f_max;
  p->nf = nf;
  p->nd = nd;
  p->nt = nt;
  p->dtype = dtype;
  p->flags = flags;
  const std::string err = fdmt::build_tables(f_min, f_max, nf, nd, p->host, gamma);
  if (!err.empty()) {
    delete p;
    return err.rfind("unsupported", 0) == 0 ? FDMT_ERR_UNSUPPORTED : FDMT_ERR_INVALID_ARG;
  }
  const Tables &t = p->host;
  const int L = t.levels;
  pingpong_sizes(t, nt, state_elem(dtype), L - 1, &p->ws_split, &p->ws_bytes);
  adjoint_ws_sizes(t, nt, &p->adj_ws_split, &p->adj_ws_bytes);
  if (flags & FDMT_SCHED_FUSED) {
    if (nt >= ((int64_t)1 << 31) - ((int64_t)1 << 22)) {  // TMA coordinates are int32
      delete p;
      return FDMT_ERR_UNSUPPORTED;
    }
    fdmt::FusedParams fparams;
    fparams.narrow = (dtype == FDMT_U8_I32);
    if (params != nullptr) {
      if (params->tile < 0 || params->tile % 64 != 0 || params->smem_budget < 0 ||
          params->smem_budget > 227 * 1024 || params->n_bounds < 0 || params->n_bounds > 32 ||
          params->staging < 0 || params->staging > 2 || params->state16 < 0 || params->state16 > 1 ||
          params->search_widths < 0 || params->search_widths > fdmt::kSearchMaxWidths) {
        delete p;
        return FDMT_ERR_INVALID_ARG;
      }
      // The search's int32 window sums of uint8 input must not overflow:
      // |B_w| <= 2^(K-1) * 255 * (nf + nd - 1).
      if (params->search_widths > 0 && dtype == FDMT_U8_I32 &&
          (255LL * (nf + nd - 1)) << (params->search_widths - 1) > (long long)INT32_MAX) {
        delete p;
        return FDMT_ERR_UNSUPPORTED;
      }
      fparams.search_k = params->search_widths;
      fparams.W = params->tile;
      fparams.staging = params->staging;
      if (params->state16 == 1) fparams.narrow = false;
      if (params->smem_budget > 0) fparams.smem_budget = params->smem_budget;
      for (int32_t i = 0; i < params->n_bounds; ++i) fparams.bounds.push_back(params->bounds[i]);
      for (int32_t i = 0; i + 1 < params->n_bounds; ++i) {
        fparams.group_W.push_back(params->group_tile[i]);
        fparams.group_budget.push_back(params->group_budget[i]);
      }
    }
    const std::string ferr = fdmt::plan_fused(t, nt, (int32_t)state_elem(dtype),
                                              (int32_t)input_elem(dtype), fparams, p->fused);
    if (!ferr.empty()) {
      delete p;
      return FDMT_ERR_UNSUPPORTED;
    }
    p->has_fused = true;
    p->fused_ws_bytes = p->fused.ws_bytes;
    p->fused_ws_split = p->fused.ws_split;
    if (fparams.search_k > 0) {
      // Partials of the last launch's search: a value (up to 8 bytes) and a
      // region (4 bytes) per (row, width, tile), after the level states.
      p->search_k = fparams.search_k;
      p->search_nseg = (int32_t)p->fused.groups.back().ntiles;
      const size_t slots = (size_t)nd * (size_t)p->search_k * (size_t)p->search_nseg;
      p->part_off = round_up(p->fused_ws_bytes, kAlign);
      p->part_bytes = round_up(slots * (sizeof(int64_t) + sizeof(int32_t)), kAlign);
      p->fused_ws_bytes = p->part_off + p->part_bytes;
    }
    if (params != nullptr && (params->adjoint_schedule < 0 || params->adjoint_schedule > 2 ||
                              (params->adjoint_schedule != 2 && (params->adjoint_tile || params->adjoint_smem_budget ||
                                                                 params->adjoint_n_bounds)))) {
      delete p;
      return FDMT_ERR_INVALID_ARG;
    }
    if (dtype != FDMT_U8_I32 && (params == nullptr || params->adjoint_schedule != 1)) {
      fdmt::AdjParams ap;
      if (params != nullptr) {
        if (params->adjoint_tile < 0 ||
            params->adjoint_tile % 64 != 0 || params->adjoint_smem_budget < 0 ||
            params->adjoint_smem_budget > 227 * 1024 || params->adjoint_n_bounds < 0 ||
            params->adjoint_n_bounds > 32) {
          delete p;
          return FDMT_ERR_INVALID_ARG;
        }
        if (params->adjoint_tile > 0) {
          ap.W = params->adjoint_tile;
          ap.init_wide = false;
        }
        if (params->adjoint_smem_budget > 0) {
          ap.smem_budget = params->adjoint_smem_budget;
          ap.grow_budget = false;
        }
        for (int32_t i = 0; i < params->adjoint_n_bounds; ++i) ap.bounds.push_back(params->adjoint_bounds[i]);
        for (int32_t i = 0; i + 1 < params->adjoint_n_bounds; ++i) {
          if (params->adjoint_group_tile[i] < 0 || params->adjoint_group_tile[i] % 64 != 0 ||
              params->adjoint_group_budget[i] < 0 || params->adjoint_group_budget[i] > 227 * 1024) {
            delete p;
            return FDMT_ERR_INVALID_ARG;
          }
          ap.group_W.push_back(params->adjoint_group_tile[i]);
          ap.group_budget.push_back(params->adjoint_group_budget[i]);
        }
      }
      const std::string aerr = fdmt::plan_adjoint_fused(t, nt, ap, p->adj_fused);
      if (!aerr.empty()) {
        // explicit adjoint parameters that do not fit are an error; the
        // defaults fall back to the plain adjoint
        if (params != nullptr && (params->adjoint_tile || params->adjoint_smem_budget || params->adjoint_n_bounds)) {
          delete p;
          return aerr.rfind("unsupported", 0) == 0 ? FDMT_ERR_UNSUPPORTED : FDMT_ERR_INVALID_ARG;
        }
      } else {
        p->has_adj_fused = true;
        // the same two ping-pong buffers serve both adjoints
        const size_t b0 = round_up(p->adj_fused.buf_bytes[0], kAlign);
        const size_t b1 = round_up(p->adj_fused.buf_bytes[1], kAlign);
        const size_t second = p->adj_ws_bytes - p->adj_ws_split;
        p->adj_ws_split = std::max(p->adj_ws_split, b0);
        p->adj_ws_bytes = p->adj_ws_split + std::max(second, b1);
        p->adj_part_off = round_up(p->adj_ws_bytes, kAlign);
        p->adj_ws_bytes = p->adj_part_off + round_up((size_t)p->adj_fused.part_slots * sizeof(float), kAlign);
      }
    }
  }

  p->d_min = d_min;
  p->descending = descending;
  p->mapped = d_min > 0 || descending != 0;
  if (p->mapped) {
    p->in_shift = fdmt::input_shifts(f_min, f_max, nf, d_min, gamma);
    p->map_off = round_up(p->has_fused ? p->fused_ws_bytes : p->ws_bytes, kAlign);
    p->map_bytes = round_up((size_t)nf * (size_t)nt * input_elem(dtype), kAlign);
    p->adj_map_off = round_up(p->adj_ws_bytes, kAlign);
    p->adj_map_bytes = 2 * round_up((size_t)nf * (size_t)nt * sizeof(float), kAlign);
  }

  DeviceTables &d = p->dev;
  d.nf = nf;
  d.nd = nd;
  d.descending = descending;
  d.levels = L;
  d.max_sweep = t.max_sweep;
  d.level_rows.assign(t.level_rows.begin(), t.level_rows.end());
  d.ops_begin.assign(t.ops_begin.begin(), t.ops_begin.end());
  d.adj_begin.assign(t.adj_begin.begin(), t.adj_begin.end());
  d.adj2_begin.assign(t.adj2_begin.begin(), t.adj2_begin.end());
  d.prof = &p->prof;

  if (!(flags & FDMT_PLAN_HOST_ONLY)) {
    if (cudaGetDevice(&p->device) != cudaSuccess) {
      delete p;
      return FDMT_ERR_CUDA;
    }
    cudaError_t e = upload(t.init, &d.init);
    if (e == cudaSuccess) e = upload(t.ops, &d.ops);
    if (e == cudaSuccess) e = upload(t.adj, &d.adj);
    if (e == cudaSuccess) e = upload(t.adj2, &d.adj2);
    if (e == cudaSuccess) e = upload(t.adj2_terms, &d.adj2_terms);
    if (e == cudaSuccess) e = upload(std::vector<int>{0}, &d.status);
    if (e == cudaSuccess && p->mapped) e = upload(p->in_shift, &d.in_shift);
    if (e == cudaSuccess && p->has_fused) {
      d.fused = &p->fused;
      e = upload(p->fused.tpls, &d.f_tpls);
      if (e == cudaSuccess) e = upload(p->fused.loads, &d.f_loads);
      if (e == cudaSuccess) e = upload(p->fused.walks, &d.f_walks);
      if (e == cudaSuccess) e = upload(p->fused.ops, &d.f_ops);
      if (e == cudaSuccess) e = upload(p->fused.stages, &d.f_stages);
    }
    if (e == cudaSuccess && p->has_adj_fused) {
      d.adj_fused = &p->adj_fused;
      e = upload(p->adj_fused.tpls, &d.a_tpls);
      if (e == cudaSuccess) e = upload(p->adj_fused.loads, &d.a_loads);
      if (e == cudaSuccess) e = upload(p->adj_fused.ops, &d.a_ops);
      if (e == cudaSuccess) e = upload(p->adj_fused.stages, &d.a_stages);
    }
    if (e != cudaSuccess) {
      free_device(p);
      delete p;
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? FDMT_ERR_NO_MEMORY : FDMT_ERR_CUDA;
    }
  }
  *out = p;
  return FDMT_OK;
}

void fdmt_destroy(fdmt_plan_t plan) {
  if (plan == nullptr) return;
  profile_release(plan->prof);
  free_device(plan);
  delete plan;
}

int fdmt_workspace_bytes(fdmt_plan_t plan, size_t *bytes) {
  if (plan == nullptr || bytes == nullptr) return FDMT_ERR_INVALID_ARG;
  *bytes = plan->mapped ? plan->map_off + plan->map_bytes
                        : (plan->has_fused ? plan->fused_ws_bytes : plan->ws_bytes);
  return FDMT_OK;
}

int fdmt_adjoint_workspace_bytes(fdmt_plan_t plan, size_t *bytes) {
  if (plan == nullptr || bytes == nullptr) return FDMT_ERR_INVALID_ARG;
  if (plan->dtype == FDMT_U8_I32) return FDMT_ERR_UNSUPPORTED;
  *bytes = plan->mapped ? plan->adj_map_off + plan->adj_map_bytes : plan->adj_ws_bytes;
  return FDMT_OK;
}

namespace {
// Where the last fused launch of a searching plan writes its partials.
fdmt::SearchArgs search_args(const fdmt_plan_s *plan, void *workspace) {
  fdmt::SearchArgs sa{};
  const size_t slots = (size_t)plan->nd * (size_t)plan->search_k * (size_t)plan->search_nseg;
  char *base = static_cast<char *>(workspace) + plan->part_off;
  sa.part_v = base;
  sa.part_r = reinterpret_cast<int *>(base + slots * sizeof(int64_t));
  sa.nk = plan->search_k;
  sa.nseg = plan->search_nseg;
  sa.q_off = (uint32_t)plan->fused.groups.back().q_off;
  sa.q_row = (uint32_t)plan->fused.groups.back().q_row;
  return sa;
}
}  // namespace

int fdmt_execute(fdmt_plan_t plan, const void *in, const float *weights, void *out,
                 void *workspace, size_t ws_bytes, void *stream) {
  size_t need = 0;
  if (plan != nullptr) fdmt_workspace_bytes(plan, &need);
  int st = check_exec_common(plan, workspace, ws_bytes, need);
  if (st != FDMT_OK) return st;
  if (in == nullptr || out == nullptr || !aligned16(in) || !aligned16(out)) return FDMT_ERR_INVALID_ARG;
  if (weights != nullptr && plan->dtype == FDMT_U8_I32) return FDMT_ERR_INVALID_ARG;
  cudaError_t e = cudaSuccess;
  if (plan->mapped) {
    // The transform reads the mapped input (channels ascending, d_min pre-shift).
    void *mapped = static_cast<char *>(workspace) + plan->map_off;
    e = fdmt::map_input(plan->dev, plan->dtype, in, mapped, plan->nt, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return FDMT_ERR_CUDA;
    }
    in = mapped;
  }
  if (plan->has_fused) {
    void *bufs[2] = {workspace, workspace ? static_cast<char *>(workspace) + plan->fused_ws_split : nullptr};
    fdmt::SearchArgs sa{};
    if (plan->search_k > 0) sa = search_args(plan, workspace);
    e = fdmt::run_fused(plan->dev, plan->dtype, in, weights, out, bufs, plan->nt,
                        static_cast<cudaStream_t>(stream), plan->search_k > 0 ? &sa : nullptr);
  } else {
    void *bufs[2] = {workspace, static_cast<char *>(workspace) + plan->ws_split};
    e = fdmt::run_plain(plan->dev, plan->dtype, in, weights, out, bufs, plan->nt,
                        static_cast<cudaStream_t>(stream));
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FDMT_ERR_CUDA;
  }
  return FDMT_OK;
}

int fdmt_execute_search_workspace_bytes(fdmt_plan_t plan, int32_t n_widths, size_t *bytes) {
  if (plan == nullptr || bytes == nullptr || n_widths < 1 || n_widths > 13) return FDMT_ERR_INVALID_ARG;
  size_t ws = 0;
  fdmt_workspace_bytes(plan, &ws);
  if (plan->search_k == n_widths) {
    *bytes = ws;  // the partials are part of the transform's workspace
    return FDMT_OK;
  }
  size_t sws = 0;
  const int st = fdmt_search_workspace_bytes(plan->nd, plan->nt, n_widths, &sws);
  if (st != FDMT_OK) return st;
  *bytes = round_up(ws, kAlign) + sws;
  return FDMT_OK;
}

int fdmt_execute_search(fdmt_plan_t plan, const void *in, const float *weights, void *out, int32_t n_widths,
                        void *peak, int32_t *time, void *workspace, size_t ws_bytes, void *stream) {
  size_t need = 0;
  int st = fdmt_execute_search_workspace_bytes(plan, n_widths, &need);
  if (st != FDMT_OK) return st;
  if (peak == nullptr || time == nullptr) return FDMT_ERR_INVALID_ARG;
  if (workspace == nullptr || ws_bytes < need) return FDMT_ERR_WORKSPACE;
  if (plan->search_k != n_widths) {
    // No search in the plan's last launch for these widths: the transform,
    // then the standalone search over its output.
    size_t ws = 0;
    fdmt_workspace_bytes(plan, &ws);
    st = fdmt_execute(plan, in, weights, out, workspace, ws_bytes, stream);
    if (st != FDMT_OK) return st;
    const size_t off = round_up(ws, kAlign);
    const int64_t bound = plan->dtype == FDMT_U8_I32 ? 255LL * (plan->nf + plan->nd - 1) : 0;
    return fdmt_search(out, plan->dtype, plan->nd, plan->nt, n_widths, bound, peak, time,
                       static_cast<char *>(workspace) + off, ws_bytes - off, stream);
  }
  // The last launch writes A and the per-tile partials; the finalize step
  // resolves each (row, width) to its first time from A.
  st = fdmt_execute(plan, in, weights, out, workspace, ws_bytes, stream);
  if (st != FDMT_OK) return st;
  const fdmt::SearchArgs sa = search_args(plan, workspace);
  cudaError_t e = fdmt::search_finalize(plan->dtype, false, out, plan->nd, plan->nt, plan->search_k, plan->search_nseg,
                                        sa.part_v, sa.part_r, peak, time, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FDMT_ERR_CUDA;
  }
  return FDMT_OK;
}

int fdmt_execute_host(fdmt_plan_t plan, const void *host_in, const float *host_weights,
                      void *host_out, void *dev_in, float *dev_weights, void *dev_out,
                      void *workspace, size_t ws_bytes, void *stream) {
  if (plan == nullptr || host_in == nullptr || host_out == nullptr) return FDMT_ERR_INVALID_ARG;
  if (host_weights != nullptr && dev_weights == nullptr) return FDMT_ERR_INVALID_ARG;
  size_t need = 0;
  fdmt_workspace_bytes(plan, &need);
  int st = check_exec_common(plan, workspace, ws_bytes, need);
  if (st != FDMT_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t in_bytes = (size_t)plan->nf * (size_t)plan->nt * input_elem(plan->dtype);
  const size_t out_bytes = (size_t)plan->nd * (size_t)plan->nt * 4;
  if (cudaMemcpyAsync(dev_in, host_in, in_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return cudaGetLastError(), FDMT_ERR_CUDA;
  if (host_weights != nullptr &&
      cudaMemcpyAsync(dev_weights, host_weights, (size_t)plan->nf * sizeof(float),
                      cudaMemcpyHostToDevice, s) != cudaSuccess)
    return cudaGetLastError(), FDMT_ERR_CUDA;
  st = fdmt_execute(plan, dev_in, host_weights ? dev_weights : nullptr, dev_out, workspace,
                    ws_bytes, stream);
  if (st != FDMT_OK) return st;
  if (cudaMemcpyAsync(host_out, dev_out, out_bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return cudaGetLastError(), FDMT_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return cudaGetLastError(), FDMT_ERR_CUDA;
  return FDMT_OK;
}

int fdmt_adjoint(fdmt_plan_t plan, const float *grad_out, const float *in, const float *weights,
                 float *grad_in, float *grad_weights, void *workspace, size_t ws_bytes,
                 void *stream) {
  if (plan != nullptr && plan->dtype == FDMT_U8_I32) return FDMT_ERR_UNSUPPORTED;
  size_t need = 0;
  if (plan != nullptr) fdmt_adjoint_workspace_bytes(plan, &need);
  int st = check_exec_common(plan, workspace, ws_bytes, need);
  if (st != FDMT_OK) return st;
  if (grad_out == nullptr || grad_in == nullptr || !aligned16(grad_out) || !aligned16(grad_in))
    return FDMT_ERR_INVALID_ARG;
  if (grad_weights != nullptr && (in == nullptr || !aligned16(in))) return FDMT_ERR_INVALID_ARG;
  void *bufs[2] = {workspace, static_cast<char *>(workspace) + plan->adj_ws_split};
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  float *g_path = grad_in;
  const float *in_path = in;
  if (plan->mapped) {
    // Gradient with respect to the mapped input, then mapped back; the
    // weight gradient pairs it with the mapped input.
    const size_t plane = plan->adj_map_bytes / 2;
    g_path = reinterpret_cast<float *>(static_cast<char *>(workspace) + plan->adj_map_off);
    float *in_m = reinterpret_cast<float *>(static_cast<char *>(workspace) + plan->adj_map_off + plane);
    if (grad_weights != nullptr) {
      e = fdmt::map_input(plan->dev, plan->dtype, in, in_m, plan->nt, cs);
      in_path = in_m;
    }
  }
  if (e == cudaSuccess) {
    if (plan->has_adj_fused) {
      float *part = reinterpret_cast<float *>(static_cast<char *>(workspace) + plan->adj_part_off);
      e = fdmt::run_adjoint_fused(plan->dev, grad_out, weights, g_path, bufs, plan->nt, cs, in_path, part,
                                  grad_weights);
    } else {
      e = fdmt::run_adjoint_plain(plan->dev, grad_out, in_path, weights, g_path, grad_weights, bufs, plan->nt, cs);
    }
  }
  if (e == cudaSuccess && plan->mapped) e = fdmt::unmap_grad(plan->dev, g_path, grad_in, plan->nt, cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FDMT_ERR_CUDA;
  }
  return FDMT_OK;
}

int fdmt_profile_enable(fdmt_plan_t plan, int32_t capacity) {
  if (plan == nullptr || capacity < 0) return FDMT_ERR_INVALID_ARG;
  if (plan->flags & FDMT_PLAN_HOST_ONLY) return FDMT_ERR_INVALID_ARG;
  profile_release(plan->prof);
  fdmt::Profiler &pr = plan->prof;
  for (int32_t i = 0; i < capacity; ++i) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
      if (a) cudaEventDestroy(a);
      profile_release(pr);
      cudaGetLastError();
      return FDMT_ERR_CUDA;
    }
    pr.start.push_back(a);
    pr.stop.push_back(b);
  }
  pr.kernel.assign(capacity, -1);
  pr.level.assign(capacity, -1);
  pr.next = 0;
  return FDMT_OK;
}

int fdmt_profile_read(fdmt_plan_t plan, int32_t *kernel_ids, int32_t *levels, float *ms,
                      int32_t n, int64_t *launches) {
  if (plan == nullptr || launches == nullptr) return FDMT_ERR_INVALID_ARG;
  fdmt::Profiler &pr = plan->prof;
  *launches = pr.next;
  if (!pr.on()) return FDMT_OK;
  const int64_t cap = (int64_t)pr.start.size();
  const int64_t have = pr.next < cap ? pr.next : cap;
  if (have > 0 && (kernel_ids == nullptr || levels == nullptr || ms == nullptr)) return FDMT_ERR_INVALID_ARG;
  const int64_t first = pr.next - have;
  int64_t written = 0;
  for (int64_t j = 0; j < have && written < n; ++j) {
    const size_t i = (size_t)((first + j) % cap);
    if (cudaEventSynchronize(pr.stop[i]) != cudaSuccess) return cudaGetLastError(), FDMT_ERR_CUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, pr.start[i], pr.stop[i]) != cudaSuccess)
      return cudaGetLastError(), FDMT_ERR_CUDA;
    kernel_ids[written] = pr.kernel[i];
    levels[written] = pr.level[i];
    ms[written] = t;
    ++written;
  }
  pr.next = 0;
  return FDMT_OK;
}

int fdmt_device_status(fdmt_plan_t plan, void *stream) {
  if (plan == nullptr || (plan->flags & FDMT_PLAN_HOST_ONLY)) return FDMT_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int v = 0;
  if (cudaMemcpyAsync(&v, plan->dev.status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return cudaGetLastError(), FDMT_ERR_CUDA;
  if (v == 0) return FDMT_OK;
  const int zero = 0;
  if (cudaMemcpyAsync(plan->dev.status, &zero, sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return cudaGetLastError(), FDMT_ERR_CUDA;
  return FDMT_ERR_TIMEOUT;
}

int fdmt_schedule_info(fdmt_plan_t plan, int32_t *groups, int32_t *bounds, int32_t n, int32_t *tile) {
  if (plan == nullptr || groups == nullptr || tile == nullptr) return FDMT_ERR_INVALID_ARG;
  if (!plan->has_fused) {
    *groups = 0;
    *tile = 0;
    return FDMT_OK;
  }
  const std::vector<fdmt::FusedGroup> &g = plan->fused.groups;
  *groups = (int32_t)g.size();
  *tile = plan->fused.W;
  if (bounds != nullptr) {
    if (n < (int32_t)g.size() + 1) return FDMT_ERR_INVALID_ARG;
    bounds[0] = 0;
    for (size_t i = 0; i < g.size(); ++i) bounds[i + 1] = g[i].lt;
  }
  return FDMT_OK;
}

int fdmt_fused_tables(fdmt_plan_t plan, int32_t kind, int32_t *dst, int64_t n, int64_t *count) {
  if (plan == nullptr || count == nullptr) return FDMT_ERR_INVALID_ARG;
  const fdmt::FusedPlan &f = plan->fused;
  std::vector<int32_t> v;
  switch (kind) {
    case 0:
      for (const fdmt::FusedGroup &g : f.groups) {
        const int32_t row[16] = {g.lb, g.lt, g.from_input ? 1 : 0, g.tpl_begin, g.tpl_count,
                                 g.smem_bytes, (int32_t)g.ntiles, g.W, g.s_end, g.pa_end, g.box,
                                 g.chunk, g.kchunks, g.max_p, g.in_size, g.out_size};
        v.insert(v.end(), row, row + 16);
      }
      break;
    case 1:
      for (const fdmt::FusedTemplate &x : f.tpls) {
        const int32_t row[8] = {x.load_begin, x.load_count, x.walk_begin, x.walk_count,
                                x.stage_begin, x.n_stages, x.tx_bytes, x.smem_bytes};
        v.insert(v.end(), row, row + 8);
      }
      break;
    case 2:
      for (const fdmt::FusedLoad &x : f.loads) v.insert(v.end(), {x.row, x.smem, x.xoff, x.nbox});
      break;
    case 3:
      for (const fdmt::FusedWalk &x : f.walks)
        v.insert(v.end(), {x.dst, x.dst_row, x.x_lo, x.x_hi, x.width, x.col, x.a, x.e, x.dl0, x.bits, x.chan,
                           x.flags});
      break;
    case 4:
      for (const fdmt::FusedOp &x : f.ops)
        v.insert(v.end(), {x.dst, x.p0, x.p1, x.p2, x.p3, x.width, x.flags, x.col});
      break;
    case 5:
      v = f.stages;
      break;
    case 6:
      v = {f.W, f.state_size, f.input_size, f.acc_size, fdmt::kOverRead, fdmt::kDescBytes};
      break;
    case 7:
      // cost-model inputs per group: HBM KiB, shared-memory pipe kilo-slots,
      // items, ops (thousands), resident blocks, modelled microseconds
      for (const fdmt::FusedGroup &g : f.groups) {
        const int32_t row[6] = {(int32_t)(g.hbm_bytes / 1024), (int32_t)(g.smem_traffic / 128 / 1000),
                                (int32_t)(g.tpl_count * g.ntiles), (int32_t)(g.ops / 1000),
                                (int32_t)g.block_slots, (int32_t)(g.seconds * 1e6)};
        v.insert(v.end(), row, row + 6);
      }
      break;
    case 10:
      // fused adjoint launches: lt, lb, init, W, box, tpl_begin, tpl_count,
      // smem_bytes, s_end, pa_end, ntiles, modelled HBM KiB, row-block
      // chunk, chunks per row, log2 of the largest row block
      for (const fdmt::AdjGroup &g : plan->adj_fused.groups) {
        const int32_t row[15] = {g.lt, g.lb, g.init ? 1 : 0, g.W, g.box, g.tpl_begin, g.tpl_count, g.smem_bytes,
                                 g.s_end, g.pa_end, (int32_t)g.ntiles, (int32_t)(g.hbm_bytes / 1024),
                                 g.chunk, g.kchunks, g.max_p};
        v.insert(v.end(), row, row + 15);
      }
      break;
    case 11:
      for (const fdmt::FusedTemplate &x : plan->adj_fused.tpls) {
        const int32_t row[8] = {x.load_begin, x.load_count, x.walk_begin, x.walk_count,
                                x.stage_begin, x.n_stages, x.tx_bytes, x.smem_bytes};
        v.insert(v.end(), row, row + 8);
      }
      break;
    case 12:
      for (const fdmt::FusedLoad &x : plan->adj_fused.loads) v.insert(v.end(), {x.row, x.smem, x.xoff, x.nbox});
      break;
    case 13:
      for (const fdmt::FusedOp &x : plan->adj_fused.ops)
        v.insert(v.end(), {x.dst, x.p0, x.p1, x.p2, x.p3, x.width, x.flags, x.col});
      break;
    case 14:
      v = plan->adj_fused.stages;
      break;
    default:
      return FDMT_ERR_INVALID_ARG;
  }
  *count = (int64_t)v.size();
  if (dst != nullptr) {
    if (n < (int64_t)v.size()) return FDMT_ERR_INVALID_ARG;
    std::memcpy(dst, v.data(), v.size() * sizeof(int32_t));
  }
  return FDMT_OK;
}

const char *fdmt_kernel_name(int32_t kernel_id) {
  switch (kernel_id) {
    case fdmt::K_INIT: return "init";
    case fdmt::K_MERGE: return "merge";
    case fdmt::K_ADJ_MERGE: return "adjoint_merge";
    case fdmt::K_ADJ_INIT: return "adjoint_init";
    case fdmt::K_WEIGHTS: return "weights_epilogue";
    case fdmt::K_FUSED_LOCAL: return "fused_local";
    case fdmt::K_FUSED_CONE: return "fused_cone";
    case fdmt::K_ADJ_MERGE2: return "adjoint_merge2";
    case fdmt::K_MAP_INPUT: return "map_input";
    case fdmt::K_UNMAP_GRAD: return "unmap_grad";
    case fdmt::K_FFT_FORWARD: return "fft_forward";
    case fdmt::K_FFT_MERGE: return "fft_merge";
    case fdmt::K_FFT_INVERSE: return "fft_inverse";
    case fdmt::K_ADJ_CONE: return "adjoint_cone";
    case fdmt::K_ADJ_WFINAL: return "adjoint_weights_finalize";
    default: return "unknown";
  }
}

const char *fdmt_error_string(int status) {
  switch (status) {
    case FDMT_OK: return "ok";
    case FDMT_ERR_INVALID_ARG: return "invalid argument";
    case FDMT_ERR_UNSUPPORTED: return "unsupported configuration";
    case FDMT_ERR_CUDA: return "CUDA error";
    case FDMT_ERR_NO_MEMORY: return "out of memory";
    case FDMT_ERR_TIMEOUT: return "device wait timed out";
    case FDMT_ERR_WORKSPACE: return "workspace missing or too small";
    default: return "unknown status";
  }
}

int fdmt_num_levels(fdmt_plan_t plan, int32_t *levels) {
  if (plan == nullptr || levels == nullptr) return FDMT_ERR_INVALID_ARG;
  *levels = plan->host.levels;
  return FDMT_OK;
}

int fdmt_band_rows(fdmt_plan_t plan, int32_t level, int32_t *rows_out, int32_t n) {
  if (plan == nullptr || rows_out == nullptr) return FDMT_ERR_INVALID_ARG;
  if (level < 0 || level > plan->host.levels) return FDMT_ERR_INVALID_ARG;
  const std::vector<int32_t> &r = plan->host.band_rows[level];
  if (n < (int32_t)r.size()) return FDMT_ERR_INVALID_ARG;
  std::memcpy(rows_out, r.data(), r.size() * sizeof(int32_t));
  return FDMT_OK;
}

int fdmt_plan_shape(fdmt_plan_t plan, int32_t *nf, int64_t *nt, int32_t *nd, int32_t *dtype) {
  if (plan == nullptr) return FDMT_ERR_INVALID_ARG;
  if (nf != nullptr) *nf = plan->nf;
  if (nt != nullptr) *nt = plan->nt;
  if (nd != nullptr) *nd = plan->nd;
  if (dtype != nullptr) *dtype = plan->dtype;
  return FDMT_OK;
}

int fdmt_input_map(fdmt_plan_t plan, int32_t *shift, int32_t n, int32_t *descending) {
  if (plan == nullptr) return FDMT_ERR_INVALID_ARG;
  if (shift != nullptr) {
    if (n < plan->nf) return FDMT_ERR_INVALID_ARG;
    for (int32_t k = 0; k < plan->nf; ++k) shift[k] = plan->mapped ? plan->in_shift[(size_t)k] : 0;
  }
  if (descending != nullptr) *descending = plan->descending;
  return FDMT_OK;
}

int fdmt_band_dl(fdmt_plan_t plan, int32_t level, int32_t band, int32_t *dl_out, int32_t n) {
  if (plan == nullptr || dl_out == nullptr) return FDMT_ERR_INVALID_ARG;
  if (level < 1 || level > plan->host.levels) return FDMT_ERR_INVALID_ARG;
  if (band < 0 || band >= fdmt::bands_at(plan->nf, level)) return FDMT_ERR_INVALID_ARG;
  const std::vector<int32_t> &d = plan->host.dl[level][band];
  if (n < (int32_t)d.size()) return FDMT_ERR_INVALID_ARG;
  std::memcpy(dl_out, d.data(), d.size() * sizeof(int32_t));
  return FDMT_OK;
}

}  // extern "C"

namespace fdmt {

// Read-only view of a plan for entry points defined in other files.
bool plan_view(fdmt_plan_t plan, PlanView *v) {
  if (plan == nullptr || v == nullptr) return false;
  v->dev = &plan->dev;
  v->dtype = plan->dtype;
  v->nt = plan->nt;
  v->device = plan->device;
  v->host_only = (plan->flags & FDMT_PLAN_HOST_ONLY) != 0;
  v->ws_bytes = plan->ws_bytes;
  v->ws_split = plan->ws_split;
  v->mapped = plan->mapped;
  return true;
}

}  // namespace fdmt
