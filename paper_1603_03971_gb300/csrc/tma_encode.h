// The driver's tensor-map encoder (cuTensorMapEncodeTiled), looked up once
// through the runtime's driver entry-point query so that librtm does not link
// libcuda directly. NULL when the driver does not provide it.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

namespace rtm {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn tma_encoder();

}  // namespace rtm
