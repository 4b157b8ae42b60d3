// Batched FDMT with the fused schedule: every beam's cone programme (the
// single-beam fused schedule of fdmt_fused_plan.cpp) runs in ONE persistent
// launch; see fdmt_batch_fused.cu.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <vector>

#include "../../include/fdmt.h"
#include "fdmt_tables.h"

namespace fdmt {

struct FusedBatch;

// Plans the fused programme of every beam (tables already built) with the
// given tile (0 = per launch by the planner) and shared-memory budget per
// block.  Returns an FDMT status.
int fused_batch_create(const std::vector<fdmt_beam_desc> &desc, const std::vector<Tables> &tabs, int dtype,
                       const fdmt_batch_params &prm, FusedBatch **out);
void fused_batch_destroy(FusedBatch *fb);
size_t fused_batch_workspace(const FusedBatch *fb);
// Test hook: leave out the work items of (beam, level group); group -1
// restores the full work list.
int fused_batch_drop(FusedBatch *fb, int beam, int group);
int fused_batch_execute(FusedBatch *fb, const void *const *in, void *const *out, void *workspace,
                        cudaStream_t s);
// Level boundaries of beam b's programme: 0 = b0 < ... < b_G = L, and the
// bytes per sample stored at each.
std::vector<int32_t> fused_batch_bounds(const FusedBatch *fb, int b);
std::vector<int32_t> fused_batch_sizes(const FusedBatch *fb, int b);

}  // namespace fdmt
