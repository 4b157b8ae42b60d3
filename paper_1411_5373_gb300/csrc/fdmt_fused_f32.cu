// The fused-schedule launches for float32 input and state, in a translation
// unit of their own so that the kernel variants compile in parallel.
#include "fdmt_fused_launch.cuh"

namespace fdmt {

cudaError_t run_fused_f32(const DeviceTables &dt, const void *in, const float *w, void *out, void *const bufs[2],
                          int64_t nt, cudaStream_t s, const SearchArgs *sa) {
  return run_fused_typed<float, float, float, float, false>(dt, in, w, out, bufs, nt, s, sa);
}

}  // namespace fdmt
