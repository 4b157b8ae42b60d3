// The fused-schedule launches for uint8 input (int32 sums; launch-boundary
// states stored as uint16 where the sums fit), in a translation unit of
// their own so that the kernel variants compile in parallel.
#include "fdmt_fused_launch.cuh"

namespace fdmt {

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

}  // namespace fdmt
