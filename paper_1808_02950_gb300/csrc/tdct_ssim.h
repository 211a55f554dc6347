// tdct_ssim.h -- batched mean SSIM of u8 plane pairs (internal interface).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace tdct {

constexpr int kSsimWin = 11;    // window side (Wang et al. 2004)
constexpr int kSsimBand = 512;  // output rows per unit of work (measured: 2.5 % faster than 128)
constexpr int kSsimStrip = 64;  // output columns per unit of work (two per lane)

// One plane pair.  Outputs are the window positions: (H - 10) x (W - 10).
struct SsimDesc {
  const uint8_t* x;
  const uint8_t* y;
  int64_t xpitch, ypitch;
  int64_t unit_begin;  // exclusive prefix of units over the batch
  int32_t H, W;
  int32_t strips, bands;  // ceil((W - 10) / 64), ceil((H - 10) / 512)
  int32_t slot, pad_;
};

// The separable window w = g g^T (g: 11 taps, standard deviation 1.5, unit
// sum) and the constants C1 = (0.01 L)^2, C2 = (0.03 L)^2, L = 255.
struct SsimParams {
  float g[kSsimWin];
  float C1, C2;
};

// Sum of SSIM over every window position of each plane into d_out[slot]
// (zeroed here), then the mean.  d_descs: device array of n descriptors.
cudaError_t launch_ssim(const SsimDesc* d_descs, int n, int64_t total_units,
                        const SsimParams& sp, double* d_out, cudaStream_t s);

}  // namespace tdct
