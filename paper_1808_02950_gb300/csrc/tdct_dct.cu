// tdct_dct.cu -- the exact-DCT comparison codec (§6.1 with the DCT of §2).
//
// C[k][j] = c_k cos(pi (2j+1) k / 16), c_0 = sqrt(1/8), c_k = 1/2 (the
// orthonormal DCT-II; the matrix printed in §2 is 2C).  The constants are
// computed on the host in FP64 with std::cos and rounded once.
//
// Per block: Y = C X C^T (rows, then columns), zonal mask of the first r
// zig-zag coefficients, X' = C^T Y' C, round half away from zero, clamp, SSE.
//   FP32: FP32 arithmetic.  The 8-point transforms use the even/odd split of
//         the DCT (C[k][7-l] = (-1)^k C[k][l]): 8 additions, then products on
//         the sums (even k, factorised further) or differences (odd k), and
//         the mirror image for the inverse.  Kernels are compiled per r-class:
//         coefficients outside the class are never formed (as in the integer
//         path), the exact r is applied by a mask.  u8 planes without the
//         coefficient output run two blocks per lane as FP32 pairs
//         (dct_fp32_pair_kernel); int16 planes and the coefficient output one
//         block per lane.
//   BF16: constants, inputs and every inter-stage value rounded to bf16,
//         products accumulated in FP32 -- the numerics of chaining bf16 GEMMs
//         with FP32 accumulation -- as direct 8-term products in the order of
//         the definition (pre-adding pixel pairs would change those numerics).
// When the coefficients are requested, all 64 are formed (class 64) and the
// warp's 32 blocks are written through shared memory as contiguous stores.
#include <cmath>
#include <cstring>

#include "tdct_classes.h"
#include "tdct_dct.cuh"
#include "tdct_dct.h"

namespace tdct {

// the u8 FP32 r-class kernels are instantiated in tdct_dct_cls_*.cu
#define TDCT_DCT_EXTERN(R)                                                                  \
  extern template cudaError_t launch_dct<R, 0, false, false>(                               \
      const PlaneDesc&, const DctParams&, float*, unsigned long long*, cudaStream_t, int);
TDCT_FOR_EACH_CLASS(TDCT_DCT_EXTERN)
#undef TDCT_DCT_EXTERN

namespace {
float to_bf16_float(float v) {
  // round to nearest even on the top 16 bits (finite inputs)
  uint32_t u;
  std::memcpy(&u, &v, 4);
  u += 0x7fffu + ((u >> 16) & 1u);
  u &= 0xffff0000u;
  float o;
  std::memcpy(&o, &u, 4);
  return o;
}

template <int DT, bool BF>
cudaError_t dispatch_dct(int r, const PlaneDesc& P, const DctParams& dp, float* coef,
                         unsigned long long* sse, cudaStream_t s, int grid) {
  // coefficients requested (all 64 formed), bf16 numerics or int16 residual
  // planes: one kernel for every r; u8 FP32: the r-class kernel
  if (coef) return launch_dct<64, DT, BF, true>(P, dp, coef, sse, s, grid);
  if constexpr (BF || DT == 1) {
    return launch_dct<64, DT, BF, false>(P, dp, coef, sse, s, grid);
  } else {
    switch (r_class(r)) {
#define TDCT_DCT_CASE(R) \
  case R:                \
    return launch_dct<R, DT, false, false>(P, dp, coef, sse, s, grid);
      TDCT_FOR_EACH_CLASS(TDCT_DCT_CASE)
#undef TDCT_DCT_CASE
      default:
        return cudaErrorInvalidValue;
    }
  }
}
}  // namespace

cudaError_t launch_dct_codec(const PlaneDesc& P, int precision, float* coef,
                             unsigned long long* sse, cudaStream_t s) {
  DctParams dp;
  for (int k = 0; k < 8; ++k)
    for (int j = 0; j < 8; ++j) {
      const double ck = k == 0 ? std::sqrt(1.0 / 8.0) : std::sqrt(2.0 / 8.0);
      const double v = ck * std::cos(M_PI * (2.0 * j + 1.0) * k / 16.0);
      dp.C[8 * k + j] = precision == 1 ? to_bf16_float((float)v) : (float)v;
    }
  dp.r = P.r;
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t nb = (int64_t)P.nbx * P.nby;
  int64_t grid = (nb + 127) / 128;
  if (grid > (int64_t)sms * 16) grid = (int64_t)sms * 16;
  if (grid < 1) grid = 1;
  const bool bf = precision == 1;
  if (P.dtype == 0)
    return bf ? dispatch_dct<0, true>(P.r, P, dp, coef, sse, s, (int)grid)
              : dispatch_dct<0, false>(P.r, P, dp, coef, sse, s, (int)grid);
  return bf ? dispatch_dct<1, true>(P.r, P, dp, coef, sse, s, (int)grid)
            : dispatch_dct<1, false>(P.r, P, dp, coef, sse, s, (int)grid);
}

}  // namespace tdct
