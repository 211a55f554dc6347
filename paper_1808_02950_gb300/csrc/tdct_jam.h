// tdct_jam.h -- the 16x16 / 32x32 block codec with the JAM transforms of T1
// (internal interface).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "tdct_kernels.cuh"

namespace tdct {

struct JamParams {
  int32_t q[32];     // q_i = L / n_i
  long long L2;      // L^2 (the rounding bias of the doubled inverse)
  long long limit;   // 256 * 2 L^2: values at or above clamp to 255
  int32_t hiw;       // 128 * 2 L^2: the centring shift of u8 samples
  uint32_t magic;    // floor(a / (2 L^2)) == umulhi(a, magic) >> shift for 0 <= a < limit
  int32_t shift;
  int32_t magic16;   // floor(a / (2 L^2)) == mulhi(a, magic16) >> 16 for 0 <= a <= limit
  int32_t r;         // retained coefficients, 1..B^2
  int32_t aligned;   // bit 0: image rows 16-byte aligned, bit 1: reconstruction rows
};

// SSE of one plane (u8 or int16) coded with B x B blocks, B = 16 or 32, into
// *sse (accumulated); the reconstruction is written when P.recon is set.
cudaError_t launch_jam_codec(int B, const PlaneDesc& P, const JamParams& jp,
                             unsigned long long* sse, cudaStream_t s);

}  // namespace tdct
