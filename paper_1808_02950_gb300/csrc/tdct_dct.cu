// tdct_dct.cu -- the exact-DCT comparison codec (§6.1 with the DCT of §2).
//
// C[k][j] = c_k cos(pi (2j+1) k / 16), c_0 = sqrt(1/8), c_k = 1/2 (the
// orthonormal DCT-II; the matrix printed in §2 is 2C).  The constants are
// computed on the host in FP64 with std::cos and rounded once.
//
// Per block: Y = C X C^T (rows, then columns), zonal mask of the first r
// zig-zag coefficients, X' = C^T Y' C, round half away from zero, clamp, SSE.
//   FP32: FP32 constants, every product and sum in FP32 (fmaf).
//   BF16: constants, inputs and every inter-stage value rounded to bf16,
//         products accumulated in FP32 -- the numerics of chaining bf16 GEMMs
//         with FP32 accumulation.
// Both are direct 8-term dot products, in the index order of the definition.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>

#include "tdct_dct.h"

namespace tdct {

struct DctParams {
  float C[64];
  int32_t r;
};

template <bool BF>
__device__ __forceinline__ float rnd(float v) {
  if constexpr (BF) return __bfloat162float(__float2bfloat16_rn(v));
  else return v;
}

template <int DT, bool BF>
__global__ void __launch_bounds__(128) dct_codec_kernel(const PlaneDesc P, const DctParams dp,
                                                        float* __restrict__ coef,
                                                        unsigned long long* __restrict__ sse_out) {
  const int64_t nb = (int64_t)P.nbx * P.nby;
  unsigned long long acc = 0;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int by = (int)(b / P.nbx), bx = (int)(b - (int64_t)by * P.nbx);
    const bool full = (by * 8 + 8 <= P.H) && ((bx + 1) * 8 <= P.W);
    RowWords<DT> rw;
    load_block<DT>(P, by, bx, full && (P.vec16 & 1), rw);
    float x[64];
    {
      uint32_t xi[64];
#pragma unroll
      for (int k = 0; k < 8; ++k) unpack_row<DT>(rw, k, xi + 8 * k);
#pragma unroll
      for (int p = 0; p < 64; ++p) x[p] = (float)(int32_t)xi[p];
    }
    // rows: t[k][j] = sum_l x[k][l] C[j][l]
    float t[64];
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float a = 0.f;
#pragma unroll
        for (int l = 0; l < 8; ++l) a = fmaf(x[8 * k + l], dp.C[8 * j + l], a);
        t[8 * k + j] = rnd<BF>(a);
      }
    // columns: y[i][j] = sum_k C[i][k] t[k][j]
    float y[64];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float a = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) a = fmaf(dp.C[8 * i + k], t[8 * k + j], a);
        y[8 * i + j] = a;
      }
    if (coef) {
      float* dst = coef + b * 64;
#pragma unroll
      for (int p = 0; p < 64; ++p) dst[p] = y[p];
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) y[8 * i + j] = zz_index(i, j) < dp.r ? rnd<BF>(y[8 * i + j]) : 0.f;
    // v[k][j] = sum_i C[i][k] y[i][j]
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float a = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) a = fmaf(dp.C[8 * i + k], y[8 * i + j], a);
        t[8 * k + j] = rnd<BF>(a);
      }
    // x'[k][l] = sum_j v[k][j] C[j][l]
    int32_t out[64];
    const float lo = DT == 0 ? 0.f : -255.f;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int l = 0; l < 8; ++l) {
        float a = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) a = fmaf(t[8 * k + j], dp.C[8 * j + l], a);
        const float v = fminf(fmaxf(roundf(a), lo), 255.f);  // roundf: half away from zero
        out[8 * k + l] = (int32_t)v;
        const int32_t d = (int32_t)x[8 * k + l] - out[8 * k + l];
        const bool valid = full || ((by * 8 + k) < P.H && (bx * 8 + l) < P.W);
        s += valid ? (uint32_t)(d * d) : 0u;
      }
    acc += s;
    if (P.recon) store_block<DT>(P, by, bx, full && (P.vec16 & 2), out);
  }
  acc = warp_sum_u64(acc);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(sse_out, acc);
}

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
  if (P.dtype == 0) {
    if (bf) dct_codec_kernel<0, true><<<(unsigned)grid, 128, 0, s>>>(P, dp, coef, sse);
    else dct_codec_kernel<0, false><<<(unsigned)grid, 128, 0, s>>>(P, dp, coef, sse);
  } else {
    if (bf) dct_codec_kernel<1, true><<<(unsigned)grid, 128, 0, s>>>(P, dp, coef, sse);
    else dct_codec_kernel<1, false><<<(unsigned)grid, 128, 0, s>>>(P, dp, coef, sse);
  }
  return cudaGetLastError();
}

}  // namespace tdct
