// Host-side encoding of TMA tensor maps (cuTensorMapEncodeTiled reached
// through the runtime's driver entry point, so the library does not link
// libcuda directly).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace lbk {

inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Tiled map of rank 2..5 with unit element strides and zero fill outside the
// tensor; optional shared-memory swizzle.
inline bool encode_tiled(CUtensorMap* map, CUtensorMapDataType dt, int rank, void* base,
                         const uint64_t* dims, const uint64_t* strides_bytes,
                         const uint32_t* box,
                         CUtensorMapSwizzle swizzle = CU_TENSOR_MAP_SWIZZLE_NONE) {
  auto fn = tensor_map_encoder();
  if (!fn) return false;
  const uint32_t es[5] = {1, 1, 1, 1, 1};
  return fn(map, dt, rank, base, dims, strides_bytes, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

inline CUtensorMapDataType pop_tensor_type(int storage) {
  return storage == 3 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                      : (storage == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                      : CU_TENSOR_MAP_DATA_TYPE_FLOAT32);
}

}  // namespace lbk
