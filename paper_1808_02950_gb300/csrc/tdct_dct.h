// tdct_dct.h -- launcher of the exact-DCT comparison codec (tdct_dct.cu).
#pragma once
#include <cuda_runtime.h>

#include "tdct_kernels.cuh"

namespace tdct {
cudaError_t launch_dct_codec(const PlaneDesc& P, int precision, float* coef,
                             unsigned long long* sse, cudaStream_t s);
}  // namespace tdct
