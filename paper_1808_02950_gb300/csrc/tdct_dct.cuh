// tdct_dct.cuh -- kernel template of the exact-DCT comparison codec (see tdct_dct.cu).
#pragma once
#include <cuda_bf16.h>

#include "tdct_classes.h"
#include "tdct_kernels.cuh"

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

// Columns j that hold a kept coefficient for class R, and rows i likewise.
__host__ __device__ constexpr bool col_needed(int R, int j) {
  for (int i = 0; i < 8; ++i)
    if (kept(R, i, j)) return true;
  return false;
}

// 8-point forward DCT, outputs y[k] for `want(k)`; even/odd split.
template <typename F>
__device__ __forceinline__ void dct8_fwd(const float x[8], float y[8], const float* C, F want) {
  float s[4], d[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    s[m] = x[m] + x[7 - m];
    d[m] = x[m] - x[7 - m];
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (!want(k)) continue;
    const float* v = (k & 1) ? d : s;
    float a = v[0] * C[8 * k];
#pragma unroll
    for (int m = 1; m < 4; ++m) a = fmaf(v[m], C[8 * k + m], a);
    y[k] = a;
  }
}

// 8-point inverse DCT x[l] = sum_k C[k][l] y[k] over the k with has(k).
template <typename F>
__device__ __forceinline__ void dct8_inv(const float y[8], float x[8], const float* C, F has) {
  float e[4], o[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    float ae = 0.f, ao = 0.f;
#pragma unroll
    for (int k = 0; k < 8; k += 2)
      if (has(k)) ae = fmaf(y[k], C[8 * k + m], ae);
#pragma unroll
    for (int k = 1; k < 8; k += 2)
      if (has(k)) ao = fmaf(y[k], C[8 * k + m], ao);
    e[m] = ae;
    o[m] = ao;
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    x[m] = e[m] + o[m];
    x[7 - m] = e[m] - o[m];
  }
}

// floor(t) for |t| < 2^22 without the conversion pipe: t + 1.5 * 2^23 rounded
// toward -inf has unit spacing, so its bit pattern is 0x4B400000 + floor(t).
__device__ __forceinline__ int32_t floor_small(float t) {
  return __float_as_int(__fadd_rd(t, 12582912.0f)) - 0x4B400000;
}

// An integer sample |x| < 2^22 as a float, exactly, without the conversion
// pipe: the bit pattern 0x4B000000 + (x + 2^15) is 2^23 + x + 2^15.
__device__ __forceinline__ float small_int_to_float(int32_t x) {
  return __int_as_float(0x4B000000 + (x + 32768)) - 8421376.0f;
}

// floor(t) by the conversion instruction (FP32 path) or by the bit pattern
// (BF16 path); both are exact for the values here.  Measured: the FP32 codec
// is 2 % faster with the conversion instruction, the BF16 one 3 % faster
// without it.
template <bool BF>
__device__ __forceinline__ int32_t floor_of(float t) {
  if constexpr (BF) return floor_small(t);
  else return __float2int_rd(t);
}
template <bool BF>
__device__ __forceinline__ float int_to_float(int32_t x) {
  if constexpr (BF) return small_int_to_float(x);
  else return (float)x;
}

template <int DT, bool BF>
__device__ __forceinline__ int32_t round_clamp(float a) {
  if constexpr (DT == 0) {
    // u8: half away from zero equals floor(a + 1/2) for a >= 0; a < 0 clamps to 0
    const int32_t v = floor_of<BF>(a + 0.5f);
    return min(max(v, 0), 255);
  } else {
    const int32_t m = floor_of<BF>(fabsf(a) + 0.5f);
    return min(max(a < 0.f ? -m : m, -255), 255);
  }
}

template <int R, int DT, bool BF, bool COEF>
__global__ void __launch_bounds__(128) dct_codec_kernel(const PlaneDesc P, const DctParams dp,
                                                        float* __restrict__ coef,
                                                        unsigned long long* __restrict__ sse_out) {
  __shared__ __align__(16) float stage[COEF ? 4 : 1][COEF ? 32 * 68 : 4];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t nb = (int64_t)P.nbx * P.nby;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  unsigned long long acc = 0;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + wid * 32; base < nb; base += step) {
    const int64_t b = base + lane;
    if (b < nb) {
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
        for (int q = 0; q < 64; ++q) x[q] = int_to_float<BF>((int32_t)xi[q]);
      }
      // rows: t[k][j] = sum_l x[k][l] C[j][l], for the needed columns j
      float t[64];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if constexpr (BF) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            if (!col_needed(R, j)) continue;
            float a = 0.f;
#pragma unroll
            for (int l = 0; l < 8; ++l) a = fmaf(x[8 * k + l], dp.C[8 * j + l], a);
            t[8 * k + j] = rnd<BF>(a);
          }
        } else {
          dct8_fwd(x + 8 * k, t + 8 * k, dp.C, [](int j) { return col_needed(R, j); });
        }
      }
      // columns: y[i][j] = sum_k C[i][k] t[k][j], for the kept (i, j)
      float y[64];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (!col_needed(R, j)) continue;
        float col[8], out[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) col[k] = t[8 * k + j];
        if constexpr (BF) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            if (!kept(R, i, j)) continue;
            float a = 0.f;
#pragma unroll
            for (int k = 0; k < 8; ++k) a = fmaf(dp.C[8 * i + k], col[k], a);
            out[i] = a;
          }
        } else {
          dct8_fwd(col, out, dp.C, [j](int i) { return kept(R, i, j); });
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (kept(R, i, j)) y[8 * i + j] = out[i];
      }
      if constexpr (COEF) {
#pragma unroll
        for (int q = 0; q < 16; ++q)
          *reinterpret_cast<float4*>(&stage[wid][lane * 68 + 4 * q]) =
              make_float4(y[4 * q], y[4 * q + 1], y[4 * q + 2], y[4 * q + 3]);
      }
      // zonal mask: the class bound is compile time, the exact r at run time
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (kept(R, i, j)) y[8 * i + j] = zz_index(i, j) < dp.r ? rnd<BF>(y[8 * i + j]) : 0.f;
      // inverse columns: v[k][j] = sum_i C[i][k] y[i][j]
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (!col_needed(R, j)) continue;
        float col[8], out[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) col[i] = kept(R, i, j) ? y[8 * i + j] : 0.f;
        if constexpr (BF) {
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            float a = 0.f;
#pragma unroll
            for (int i = 0; i < 8; ++i)
              if (kept(R, i, j)) a = fmaf(dp.C[8 * i + k], col[i], a);
            out[k] = rnd<BF>(a);
          }
        } else {
          dct8_inv(col, out, dp.C, [j](int i) { return kept(R, i, j); });
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) t[8 * k + j] = out[k];
      }
      // inverse rows: x'[k][l] = sum_j v[k][j] C[j][l]; round, clamp, SSE
      int32_t outp[64];
      uint32_t s = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        float row[8], xr[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) row[j] = col_needed(R, j) ? t[8 * k + j] : 0.f;
        if constexpr (BF) {
#pragma unroll
          for (int l = 0; l < 8; ++l) {
            float a = 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j)
              if (col_needed(R, j)) a = fmaf(row[j], dp.C[8 * j + l], a);
            xr[l] = a;
          }
        } else {
          dct8_inv(row, xr, dp.C, [](int j) { return col_needed(R, j); });
        }
#pragma unroll
        for (int l = 0; l < 8; ++l) {
          const int32_t v = round_clamp<DT, BF>(xr[l]);
          outp[8 * k + l] = v;
          const int32_t d = floor_of<BF>(x[8 * k + l]) - v;  // x holds exact integers
          const bool valid = full || ((by * 8 + k) < P.H && (bx * 8 + l) < P.W);
          s += valid ? (uint32_t)(d * d) : 0u;
        }
      }
      acc += s;
      if (P.recon) store_block<DT>(P, by, bx, full && (P.vec16 & 2), outp);
    }
    if constexpr (COEF) {
      __syncwarp();
      const int64_t nblk = min((int64_t)32, nb - base);
      float* dst = coef + base * 64;
      for (int e = lane; e < nblk * 16; e += 32) {
        const int blk = e >> 4, q = e & 15;
        reinterpret_cast<float4*>(dst)[e] =
            *reinterpret_cast<const float4*>(&stage[wid][blk * 68 + 4 * q]);
      }
      __syncwarp();
    }
  }
  acc = warp_sum_u64(acc);
  if (lane == 0 && acc) atomicAdd(sse_out, acc);
}

template <int R, int DT, bool BF, bool COEF>
cudaError_t launch_dct(const PlaneDesc& P, const DctParams& dp, float* coef,
                       unsigned long long* sse, cudaStream_t s, int grid) {
  dct_codec_kernel<R, DT, BF, COEF><<<(unsigned)grid, 128, 0, s>>>(P, dp, coef, sse);
  return cudaGetLastError();
}

}  // namespace tdct
