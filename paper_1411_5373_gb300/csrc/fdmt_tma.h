// Host-side TMA tensor maps of the fused schedule (shared by the single-beam
// and the batched launches).
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>

#include <cstdint>

#include "fdmt_fused.h"

namespace fdmt {

template <class T> CUtensorMapDataType map_type();
template <> inline CUtensorMapDataType map_type<float>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT32; }
template <> inline CUtensorMapDataType map_type<int32_t>() { return CU_TENSOR_MAP_DATA_TYPE_INT32; }
template <> inline CUtensorMapDataType map_type<__half>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT16; }
template <> inline CUtensorMapDataType map_type<uint8_t>() { return CU_TENSOR_MAP_DATA_TYPE_UINT8; }
template <> inline CUtensorMapDataType map_type<uint16_t>() { return CU_TENSOR_MAP_DATA_TYPE_UINT16; }

// Fills maps[0 .. kMaxBlockP] for the rows group g stages from `base`, a
// [rows][nt] matrix of `elem`-byte samples: one 2-D row-box map in maps[0],
// or row-block maps of 2^p rows in maps[p].  *cshift = log2 of the chunk for
// row blocks, else 0.  False if the driver rejects a map (alignment, sizes).
bool make_group_maps(CUtensorMap *maps, const FusedGroup &g, const void *base, CUtensorMapDataType type,
                     uint32_t elem, uint64_t rows, uint64_t nt, int32_t *cshift);

}  // namespace fdmt
