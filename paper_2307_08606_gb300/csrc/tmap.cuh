// Driver entry point for building TMA tensor maps (cuTensorMapEncodeTiled),
// fetched through the runtime so that the library has no link-time dependency
// on libcuda.  Shared by the tensor-core kernels (tc.cu, gram_tc.cu).
#pragma once
#include <cuda.h>

namespace sadmm {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// nullptr if the driver does not provide it
EncodeTiledFn tensor_map_encoder();

}  // namespace sadmm
