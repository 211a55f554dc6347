// tdct_dct_tc.h -- the exact-DCT comparison codec in BF16 on the tensor cores
// (tdct_dct_tc.cu; internal interface).
#pragma once
#include <cuda_runtime.h>

#include "tdct_kernels.cuh"

namespace tdct {

// Upload the bf16 weight tables of every r with `split` terms per weight (1:
// bf16 numerics; 3: FP32-level accuracy), once per device, synchronously:
// call outside stream capture before the first launch.
cudaError_t dct_tc_prepare(int split, const uint16_t** tables);

// One u8 plane, retention P.r: SSE into *sse (accumulated), the
// reconstruction into P.recon if set, the FP32 coefficients Y (raster order,
// [nby][nbx][8][8]) into coef if set.  status: the device status word.
cudaError_t launch_dct_tc(const PlaneDesc& P, int split, float* coef, int* status,
                          unsigned long long* sse, cudaStream_t s);

}  // namespace tdct
