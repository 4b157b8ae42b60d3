// Host side of the fused schedule: tensor maps, the launches of fp16-state
// plans and the dispatch over the input types (the kernel and the launch
// logic: fdmt_fused_launch.cuh; float32 launches: fdmt_fused_f32.cu; uint8
// launches: fdmt_fused_u8.cu).
#include "fdmt_fused_launch.cuh"

namespace fdmt {

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

cudaError_t run_fused(const DeviceTables &dt, int dtype, const void *in, const float *w, void *out,
                      void *const bufs[2], int64_t nt, cudaStream_t s, const SearchArgs *sa) {
  if (dt.fused == nullptr) return cudaErrorInvalidValue;
  switch (dtype) {
    case 0: return run_fused_u8(dt, in, out, bufs, nt, s, sa);
    case 1: return run_fused_f32(dt, in, w, out, bufs, nt, s, sa);
    case 2: return run_fused_typed<float, __half, float, float, true>(dt, in, w, out, bufs, nt, s, sa);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fdmt
