// Internal interfaces between the C-ABI layer and the kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "fdmt_adjoint_fused.h"
#include "fdmt_fused.h"
#include "fdmt_tables.h"

namespace fdmt {

// Kernel identifiers reported by the launch profiler (enum fdmt_kernel_id).
enum KernelId : int32_t {
  K_INIT = 0,
  K_MERGE = 1,
  K_ADJ_MERGE = 2,
  K_ADJ_INIT = 3,
  K_WEIGHTS = 4,
  K_FUSED_LOCAL = 5,
  K_FUSED_CONE = 6,
  K_ADJ_MERGE2 = 7,
  K_MAP_INPUT = 8,
  K_UNMAP_GRAD = 9,
  K_FFT_FORWARD = 10,
  K_FFT_MERGE = 11,
  K_FFT_INVERSE = 12,
  K_ADJ_CONE = 13,
  K_ADJ_WFINAL = 14,
};

// Optional per-launch timing: a ring of CUDA event pairs recorded around
// every kernel launch of a plan.  Created by fdmt_profile_enable; recording
// costs two event records per launch and no device memory.
struct Profiler {
  std::vector<cudaEvent_t> start, stop;
  std::vector<int32_t> kernel, level;
  int64_t next = 0;     // total launches recorded since enable / last read
  bool on() const { return !start.empty(); }
  void begin(cudaStream_t s, int32_t k, int32_t l) {
    if (!on()) return;
    const size_t i = (size_t)(next % (int64_t)start.size());
    kernel[i] = k;
    level[i] = l;
    cudaEventRecord(start[i], s);
  }
  void end(cudaStream_t s) {
    if (!on()) return;
    const size_t i = (size_t)(next % (int64_t)start.size());
    cudaEventRecord(stop[i], s);
    ++next;
  }
};

// Device copies of the delay tables of one plan (owned by the plan).
struct DeviceTables {
  int32_t nf = 0, nd = 0, levels = 0, max_sweep = 0;
  std::vector<int64_t> level_rows;  // host copy, [0 .. levels]
  std::vector<int64_t> ops_begin;   // host copy, [l] offset into ops
  std::vector<int64_t> adj_begin;   // host copy, [l] offset into adj (children at level l)
  InitOp *init = nullptr;           // device, nf entries
  RowOp *ops = nullptr;             // device, all levels
  AdjOp *adj = nullptr;             // device, all levels
  std::vector<int64_t> adj2_begin;  // host copy, [l] offset into adj2 (children at level l, parents l + 2)
  AdjRun *adj2 = nullptr;           // device, composed transposed level pairs
  AdjTerm *adj2_terms = nullptr;
  Profiler *prof = nullptr;         // owned by the plan; never null after fdmt_plan
  int *status = nullptr;            // device word: nonzero after a bounded wait gave up
  // Input mapping (null / 0 unless the plan has a d_min pre-shift or
  // descending channel order): per-channel delay s_k, device, nf entries.
  int32_t *in_shift = nullptr;
  int32_t descending = 0;
  // Fused schedule (null unless the plan was made with FDMT_SCHED_FUSED).
  const FusedPlan *fused = nullptr;
  FusedTemplate *f_tpls = nullptr;
  FusedLoad *f_loads = nullptr;
  FusedWalk *f_walks = nullptr;
  FusedOp *f_ops = nullptr;
  int32_t *f_stages = nullptr;
  // Fused adjoint (null unless the plan has one).
  const AdjFusedPlan *adj_fused = nullptr;
  FusedTemplate *a_tpls = nullptr;
  FusedLoad *a_loads = nullptr;
  FusedOp *a_ops = nullptr;
  int32_t *a_stages = nullptr;
};

// What other translation units may read of a plan (see plan_view).
struct PlanView {
  const DeviceTables *dev = nullptr;
  int32_t dtype = 0;
  int64_t nt = 0;
  int device = -1;
  bool host_only = false;
  size_t ws_bytes = 0;  // forward workspace the plain schedule needs
  size_t ws_split = 0;  // offset of its second ping-pong buffer
  bool mapped = false;  // input mapping in front of the transform
};

}  // namespace fdmt

struct fdmt_plan_s;

namespace fdmt {

bool plan_view(fdmt_plan_s *plan, PlanView *v);

// Plain schedule: init + one launch per level.  bufs[0] holds even levels,
// bufs[1] odd levels (< L); level L is written to `out`.
cudaError_t run_plain(const DeviceTables &dt, int dtype, const void *in, const float *w, void *out,
                      void *const bufs[2], int64_t nt, cudaStream_t s);

// Fused schedule: one launch per group of levels (fdmt_fused.h); bufs hold
// the intermediate level states between groups.  A plan whose last launch
// ends with the boxcar search needs `sa` (the partials it writes).
cudaError_t run_fused(const DeviceTables &dt, int dtype, const void *in, const float *w, void *out,
                      void *const bufs[2], int64_t nt, cudaStream_t s, const SearchArgs *sa = nullptr);

// The boxcar search's finalize step (fdmt_search.cu) over partials
// part_v / part_r laid out as (row, width, segment): per row and width the
// largest value and the first time it occurs, recomputed from A.  wide =
// the partial values are int64 (else float or int32 as A).
cudaError_t search_finalize(int dtype, bool wide, const void *A, int32_t nd, int64_t nt, int32_t nk, int32_t nseg,
                            const void *part_v, const int *part_r, void *peak, int32_t *time, cudaStream_t s);

// Transposed transform in float32; bufs as above (levels 0 .. L-1).
// grad_in = w .* FDMT^T(grad_out); grad_w[k] = <in[k], FDMT^T(grad_out)[k]> if grad_w.
cudaError_t run_adjoint_plain(const DeviceTables &dt, const float *grad_out, const float *in,
                              const float *w, float *grad_in, float *grad_w, void *const bufs[2],
                              int64_t nt, cudaStream_t s);

// Fused adjoint (fdmt_adjoint_fused.cu): grad_in = w .* FDMT^T(grad_out)
// (w may be null); with grad_w, also grad_w[k] = <x[k], FDMT^T(grad_out)[k]>
// through the init launch's partials in `part` (dt.adj_fused->part_slots
// floats).  bufs hold the levels between launches (buf_bytes).
cudaError_t run_adjoint_fused(const DeviceTables &dt, const float *grad_out, const float *w, float *grad_in,
                              void *const bufs[2], int64_t nt, cudaStream_t s, const float *x, float *part,
                              float *grad_w);

// Weight gradient and scaling after an unscaled adjoint:
//   grad_w[k] = <in[k], g[k]>, then g[k] *= w[k] (w may be null: no scaling).
cudaError_t run_weights_epilogue(const DeviceTables &dt, const float *in, const float *w, float *grad_in,
                                 float *grad_w, int64_t nt, cudaStream_t s);

// Input mapping (fdmt_map.cu): out[k] = raw[src(k)] delayed by s_k, and its
// transpose for the gradient.  Both as dt.in_shift / dt.descending say.
cudaError_t map_input(const DeviceTables &dt, int dtype, const void *raw, void *out, int64_t nt, cudaStream_t s);
cudaError_t unmap_grad(const DeviceTables &dt, const float *g, float *grad, int64_t nt, cudaStream_t s);

}  // namespace fdmt
