// tdct_tc.h -- launcher of the tensor-core forward variant (tdct_tc.cu).
#pragma once
#include <cuda_runtime.h>

#include "tdct_kernels.cuh"

namespace tdct {
// One launch over every unit of `tab` (u8 planes whose rows are 16-byte
// aligned, W % 16 == 0, H % 8 == 0); R is the r-class, r_exact the retention.
template <int R>
cudaError_t launch_codec_tc(const PlaneTable& tab, const CodecParams& cp, int r_exact,
                            unsigned long long* sse, cudaStream_t s);
// Write the fp16 B matrices of every r to the device (once per device,
// synchronous; call outside stream capture before the first launch).
cudaError_t tc_prepare(const uint16_t** table);
}  // namespace tdct
