// tdct_sweep.h -- the zonal sweep of §6.1 (every r = 1..64) from one read of
// each plane (internal interface; entry points in tdct_abi.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "tdct_kernels.cuh"

namespace tdct {

// A unit of the sweep is 32 consecutive blocks of one block-row (8 rows x
// 256 samples): descriptors passed to launch_sweep carry chunks =
// ceil(nbx / 32) and unit prefix sums over that unit.
constexpr int kSweepUnitBlocks = 32;

// Per-plane SSE for every retention r = 1..64 (d_sse[64 * slot + r - 1],
// accumulated: zero it first) of u8 planes.  dct = false: T1 with the exact
// integer codec of the fused kernels; dct = true: the orthonormal DCT-II
// (C row-major, FP32 arithmetic).
cudaError_t launch_sweep(const PlaneTable& tab, bool dct, const float C[64],
                         unsigned long long* d_sse, cudaStream_t s);

}  // namespace tdct
