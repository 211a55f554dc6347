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

// ---- u8 FP32: two blocks per lane as FP32 pairs ------------------------------
//
// The lane's two horizontally adjacent blocks A and B go through every stage
// together as float2 pairs (A in .x, B in .y): each FP32x2 instruction (FADD2,
// FMUL2, FFMA2) does the work of two FP32 instructions, element for element
// the same FP32 arithmetic as one block at a time.  The 8-point transforms are
// the even/odd factorisation of the DCT (C[k][7-l] = (-1)^k C[k][l]):
//   even:  e = (s0 + s3, s1 + s2, s0 - s3, s1 - s2),
//          y0 = C00 (e0 + e1), y4 = C40 (e0 - e1),
//          y2 = c2 e2 + c6 e3, y6 = c6 e2 - c2 e3;
//   odd:   y_k = sum_m C[k][m] d_m with the 4x4 sign pattern of (c1, c3, c5, c7);
// (c_m = C[m][0] = cos(m pi / 16) / 2) and the transpose for the inverse,
// each pruned at compile time to the class's needed outputs or inputs.
// Samples enter as the FP32 bit pattern 2^23 + x (one byte permute each):
// d_m = X_m - X_l is exact as it stands, s_m = X_m + (X_l - 2^24) exactly.
// The rounding 1/2 rides the DC path of the last inverse, the floor is one
// FADD2 rounding down onto 1.5 * 2^23 (the integer in the low bits), pairs
// are clamped as s16x2 and packed to bytes, the SSE is a byte dot product of
// absolute differences.  Rows reach the warp through a ring of PF slots of
// 8 rows x 32 lanes x 16 bytes (row k of both blocks) filled by 16-byte
// cp.async copies; pairs that cross the plane's edge, or planes whose rows
// are not 16-byte aligned, are staged by the lane's own loads.  Each lane
// reads back only what it copied or stored, so the ring needs no barrier;
// the rows are read twice (forward, SSE) and the slot refilled after.
// Work: units of one block row x 64 blocks (32 pairs), contiguous ranges of
// units per warp; ring depth 3 (2 and 4 measured the same).
struct DctK {
  float2 c0, c4, c1, c2, c3, c5, c6, c7;
};

__device__ __forceinline__ float2 f2b(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
}
// acc + c y and acc - c y
__device__ __forceinline__ float2 fma2(float2 c, float2 y, float2 acc) { return __ffma2_rn(c, y, acc); }
__device__ __forceinline__ float2 fms2(float2 c, float2 y, float2 acc) {
  return __ffma2_rn(make_float2(-c.x, -c.y), y, acc);
}

// Forward from the first stage's sums s and differences d: outputs y[k] for want(k).
template <typename F>
__device__ __forceinline__ void fdct8_sd2(const float2 s[4], const float2 d[4], float2 y[8],
                                          const DctK& c, F want) {
  const float2 z = make_float2(0.f, 0.f);
  const float2 e0 = add2(s[0], s[3]), e1 = add2(s[1], s[2]);
  const float2 e2 = sub2(s[0], s[3]), e3 = sub2(s[1], s[2]);
  if (want(0)) y[0] = __fmul2_rn(c.c0, add2(e0, e1));
  if (want(4)) y[4] = __fmul2_rn(c.c4, sub2(e0, e1));
  if (want(2)) y[2] = fma2(c.c6, e3, __fmul2_rn(c.c2, e2));
  if (want(6)) y[6] = fms2(c.c2, e3, __fmul2_rn(c.c6, e2));
  if (want(1)) y[1] = fma2(c.c7, d[3], fma2(c.c5, d[2], fma2(c.c3, d[1], fma2(c.c1, d[0], z))));
  if (want(3)) y[3] = fms2(c.c5, d[3], fms2(c.c1, d[2], fms2(c.c7, d[1], fma2(c.c3, d[0], z))));
  if (want(5)) y[5] = fma2(c.c3, d[3], fma2(c.c7, d[2], fms2(c.c1, d[1], fma2(c.c5, d[0], z))));
  if (want(7)) y[7] = fms2(c.c1, d[3], fma2(c.c3, d[2], fms2(c.c5, d[1], fma2(c.c7, d[0], z))));
}

template <typename F>
__device__ __forceinline__ void fdct8_2(const float2 x[8], float2 y[8], const DctK& c, F want) {
  float2 s[4], d[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    s[m] = add2(x[m], x[7 - m]);
    d[m] = sub2(x[m], x[7 - m]);
  }
  fdct8_sd2(s, d, y, c, want);
}

// Inverse x_l = sum_k C[k][l] y_k + bias over the y_k with has(k).
template <typename F>
__device__ __forceinline__ void idct8_2(const float2 y[8], float2 x[8], const DctK& c, F has,
                                        float bias) {
  const float2 b = f2b(bias);
  float2 P = b, Q = b;
  if (has(0)) {
    P = fma2(c.c0, y[0], b);
    Q = P;
  }
  if (has(4)) {
    P = fma2(c.c4, y[4], P);
    Q = fms2(c.c4, y[4], Q);
  }
  float2 E0 = P, E3 = P, E1 = Q, E2 = Q;
  if (has(2)) {
    E0 = fma2(c.c2, y[2], E0);
    E3 = fms2(c.c2, y[2], E3);
    E1 = fma2(c.c6, y[2], E1);
    E2 = fms2(c.c6, y[2], E2);
  }
  if (has(6)) {
    E0 = fma2(c.c6, y[6], E0);
    E3 = fms2(c.c6, y[6], E3);
    E1 = fms2(c.c2, y[6], E1);
    E2 = fma2(c.c2, y[6], E2);
  }
  const bool odd = has(1) || has(3) || has(5) || has(7);
  if (!odd) {
    x[0] = E0, x[7] = E0, x[1] = E1, x[6] = E1, x[2] = E2, x[5] = E2, x[3] = E3, x[4] = E3;
    return;
  }
  const float2 z = make_float2(0.f, 0.f);
  float2 O0 = z, O1 = z, O2 = z, O3 = z;
  if (has(1)) {
    O0 = fma2(c.c1, y[1], O0), O1 = fma2(c.c3, y[1], O1);
    O2 = fma2(c.c5, y[1], O2), O3 = fma2(c.c7, y[1], O3);
  }
  if (has(3)) {
    O0 = fma2(c.c3, y[3], O0), O1 = fms2(c.c7, y[3], O1);
    O2 = fms2(c.c1, y[3], O2), O3 = fms2(c.c5, y[3], O3);
  }
  if (has(5)) {
    O0 = fma2(c.c5, y[5], O0), O1 = fms2(c.c1, y[5], O1);
    O2 = fma2(c.c7, y[5], O2), O3 = fma2(c.c3, y[5], O3);
  }
  if (has(7)) {
    O0 = fma2(c.c7, y[7], O0), O1 = fms2(c.c5, y[7], O1);
    O2 = fma2(c.c3, y[7], O2), O3 = fms2(c.c1, y[7], O3);
  }
  x[0] = add2(E0, O0), x[7] = sub2(E0, O0);
  x[1] = add2(E1, O1), x[6] = sub2(E1, O1);
  x[2] = add2(E2, O2), x[5] = sub2(E2, O2);
  x[3] = add2(E3, O3), x[4] = sub2(E3, O3);
}

// 2^23 + byte m of the row word pair (m < 4: w0), as an FP32 bit pattern.
__device__ __forceinline__ float biased_sample(uint32_t w0, uint32_t w1, int m) {
  return __uint_as_float(__byte_perm(m < 4 ? w0 : w1, 0x4B000000u, (uint32_t)((m & 3) + 0x7540)));
}

// Eight FP32 bit patterns 0x4B400000 + v (v = floor of a sample, |v| < 2^15)
// -> eight bytes clamp(v, 0, 255): low halves paired as s16x2, clamped,
// packed.
__device__ __forceinline__ uint2 pack_floor_bits_u8(const uint32_t f[8]) {
  const uint32_t c01 = min_relu_s16x2(__byte_perm(f[0], f[1], 0x5410u), 0x00ff00ffu);
  const uint32_t c23 = min_relu_s16x2(__byte_perm(f[2], f[3], 0x5410u), 0x00ff00ffu);
  const uint32_t c45 = min_relu_s16x2(__byte_perm(f[4], f[5], 0x5410u), 0x00ff00ffu);
  const uint32_t c67 = min_relu_s16x2(__byte_perm(f[6], f[7], 0x5410u), 0x00ff00ffu);
  return make_uint2(__byte_perm(c01, c23, 0x6420u), __byte_perm(c45, c67, 0x6420u));
}

#ifndef TDCT_DCT_PAIR_STAGES
#define TDCT_DCT_PAIR_STAGES 3
#endif
constexpr int kDctPairStages = TDCT_DCT_PAIR_STAGES;
constexpr int kDctPairSlotBytes = 8 * 32 * 16;  // 8 rows x 32 lanes x 16 bytes

// Resident CTAs per SM the pair kernel is compiled for: 4 (128 registers, no
// spills) up to class 16 (2 % faster than 3 at r = 16, bench workload), 3 for
// class 21 (it would spill at 128), 2 from class 28 (more coefficients live).
__host__ __device__ constexpr int dct_pair_min_ctas(int R) {
#ifdef TDCT_DCT_PAIR_MINB
  return R >= 28 ? 2 : TDCT_DCT_PAIR_MINB;
#else
  return R >= 28 ? 2 : R >= 21 ? 3 : 4;
#endif
}

template <int R>
__global__ void __launch_bounds__(128, dct_pair_min_ctas(R))
    dct_fp32_pair_kernel(const PlaneDesc P, const DctParams dp, unsigned long long* __restrict__ sse_out) {
  constexpr int PF = kDctPairStages;
  extern __shared__ __align__(16) uint4 dct_ring[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // row k of slot s, per lane: + (s 8 + k) 32
  uint4* const ring = dct_ring + (size_t)wid * PF * (kDctPairSlotBytes / 16) + lane;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t U = (int64_t)P.nby * P.chunks;
  const int64_t u_begin = (U * warp) / nwarps;
  const int n_units = (int)((U * (warp + 1)) / nwarps - u_begin);
  const bool al16 = ((reinterpret_cast<uintptr_t>(P.img) | (uintptr_t)P.pitch) & 15) == 0;
  const bool rec16 =
      P.recon && ((reinterpret_cast<uintptr_t>(P.recon) | (uintptr_t)P.recon_pitch) & 15) == 0;
  const bool rec8 = P.recon && (P.vec16 & 2);
  DctK c;
  c.c0 = f2b(dp.C[0]);
  c.c4 = f2b(dp.C[32]);
  c.c1 = f2b(dp.C[8]);
  c.c2 = f2b(dp.C[16]);
  c.c3 = f2b(dp.C[24]);
  c.c5 = f2b(dp.C[40]);
  c.c6 = f2b(dp.C[48]);
  c.c7 = f2b(dp.C[56]);
  const int rmask = dp.r < R ? dp.r : 64;  // zonal mask needed only below the class bound

  // The pair (bx0, bx0 + 1) of block row by from its ring slot: SSE of both.
  auto pair_codec = [&](const uint4* rows, int by, int bx0) -> uint32_t {
    // rows: t[k][j] for the needed columns j
    float2 t[64];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint4 rk = rows[k * 32];
      float2 sd_s[4], sd_d[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const float2 xm = make_float2(biased_sample(rk.x, rk.y, m), biased_sample(rk.z, rk.w, m));
        const float2 xl =
            make_float2(biased_sample(rk.x, rk.y, 7 - m), biased_sample(rk.z, rk.w, 7 - m));
        sd_d[m] = sub2(xm, xl);
        sd_s[m] = add2(xm, add2(xl, f2b(-16777216.0f)));
      }
      fdct8_sd2(sd_s, sd_d, t + 8 * k, c, [](int j) { return col_needed(R, j); });
    }
    // columns: y[i][j] for the kept (i, j); zonal mask at run time below the class bound
    float2 y[64];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (!col_needed(R, j)) continue;
      float2 col[8], out[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) col[k] = t[8 * k + j];
      fdct8_2(col, out, c, [j](int i) { return kept(R, i, j); });
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (kept(R, i, j)) y[8 * i + j] = out[i];
    }
    if (rmask < 64) {
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (kept(R, i, j) && zz_index(i, j) >= rmask) y[8 * i + j] = make_float2(0.f, 0.f);
    }
    // inverse columns: v[k][j] = sum_i C[i][k] y[i][j], into t
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (!col_needed(R, j)) continue;
      float2 col[8], out[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) col[i] = kept(R, i, j) ? y[8 * i + j] : make_float2(0.f, 0.f);
      idct8_2(col, out, c, [j](int i) { return kept(R, i, j); }, 0.0f);
#pragma unroll
      for (int k = 0; k < 8; ++k) t[8 * k + j] = out[k];
    }
    // inverse rows (+ 1/2 through the DC path), floor, clamp, SSE, store
    const bool has1 = bx0 + 1 < P.nbx;
    const int vr = min(8, P.H - by * 8);
    const int vcA = min(8, P.W - bx0 * 8), vcB = has1 ? min(8, P.W - (bx0 + 1) * 8) : 0;
    const bool fullA = vr == 8 && vcA == 8, fullB = vr == 8 && vcB == 8;
    const uint64_t mA = vcA >= 8 ? ~0ull : ((1ull << (8 * vcA)) - 1ull);
    const uint64_t mB = vcB >= 8 ? ~0ull : vcB <= 0 ? 0ull : ((1ull << (8 * vcB)) - 1ull);
    uint8_t* out0 =
        P.recon ? P.recon + (int64_t)(by * 8) * P.recon_pitch + (int64_t)bx0 * 8 : nullptr;
    uint32_t sse = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      float2 row[8], xr[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) row[j] = col_needed(R, j) ? t[8 * k + j] : make_float2(0.f, 0.f);
      idct8_2(row, xr, c, [](int j) { return col_needed(R, j); }, 0.5f);
      uint32_t fa[8], fb[8];
#pragma unroll
      for (int l = 0; l < 8; ++l) {
        const float2 f = __fadd2_rd(xr[l], f2b(12582912.0f));  // 0x4B400000 + floor(x' + 1/2)
        fa[l] = __float_as_uint(f.x);
        fb[l] = __float_as_uint(f.y);
      }
      uint2 ya = pack_floor_bits_u8(fa), yb = pack_floor_bits_u8(fb);
      const uint4 rk = rows[k * 32];
      const uint2 xa = make_uint2(rk.x, rk.y), xb = make_uint2(rk.z, rk.w);
      if (!(fullA && fullB)) {
        // outside the plane the samples were staged as 0: give the
        // reconstruction the same bytes there (no SSE contribution)
        const uint64_t ma = k < vr ? mA : 0ull, mb = k < vr ? mB : 0ull;
        ya.x = (ya.x & (uint32_t)ma) | (xa.x & ~(uint32_t)ma);
        ya.y = (ya.y & (uint32_t)(ma >> 32)) | (xa.y & ~(uint32_t)(ma >> 32));
        yb.x = (yb.x & (uint32_t)mb) | (xb.x & ~(uint32_t)mb);
        yb.y = (yb.y & (uint32_t)(mb >> 32)) | (xb.y & ~(uint32_t)(mb >> 32));
      }
      const uint32_t d0 = __vabsdiffu4(xa.x, ya.x), d1 = __vabsdiffu4(xa.y, ya.y);
      const uint32_t d2 = __vabsdiffu4(xb.x, yb.x), d3 = __vabsdiffu4(xb.y, yb.y);
      sse = __dp4a(d0, d0, __dp4a(d1, d1, __dp4a(d2, d2, __dp4a(d3, d3, sse))));
      if (out0 && k < vr) {
        uint8_t* orow = out0 + (int64_t)k * P.recon_pitch;
        if (fullA && fullB && rec16) {
          *reinterpret_cast<uint4*>(orow) = make_uint4(ya.x, ya.y, yb.x, yb.y);
        } else {
          if (vcA == 8 && rec8) {
            *reinterpret_cast<uint2*>(orow) = ya;
          } else {
#pragma unroll
            for (int l = 0; l < 8; ++l)
              if (l < vcA) orow[l] = (uint8_t)(((l < 4 ? ya.x : ya.y) >> (8 * (l & 3))) & 0xffu);
          }
          if (vcB == 8 && rec8) {
            *reinterpret_cast<uint2*>(orow + 8) = yb;
          } else {
#pragma unroll
            for (int l = 0; l < 8; ++l)
              if (l < vcB) orow[8 + l] = (uint8_t)(((l < 4 ? yb.x : yb.y) >> (8 * (l & 3))) & 0xffu);
          }
        }
      }
    }
    return sse;
  };

  // producer: unit (by, chunk) of the next fetch
  int f_by = 0, f_chunk = 0;
  if (n_units > 0) {
    f_by = (int)(u_begin / P.chunks);
    f_chunk = (int)(u_begin - (int64_t)f_by * P.chunks);
  }
  int c_by = f_by, c_chunk = f_chunk;  // consumer
  auto fetch = [&](int slot) {
    uint4* dst = ring + slot * 8 * 32;
    const int bx0 = f_chunk * 64 + 2 * lane;
    const uint8_t* src = P.img + (int64_t)(f_by * 8) * P.pitch + (int64_t)bx0 * 8;
    const bool full = f_by * 8 + 8 <= P.H && bx0 * 8 + 16 <= P.W;
    if (full && al16) {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(dst + k * 32)),
                     "l"(src + (int64_t)k * P.pitch)
                     : "memory");
    } else {
      const int vr = min(8, P.H - f_by * 8), vc = min(16, P.W - bx0 * 8);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        if (k < vr)
#pragma unroll
          for (int l = 0; l < 16; ++l)
            if (l < vc) w[l >> 2] |= (uint32_t)src[(int64_t)k * P.pitch + l] << (8 * (l & 3));
        dst[k * 32] = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    if (++f_chunk == P.chunks) {
      f_chunk = 0;
      ++f_by;
    }
  };
#pragma unroll
  for (int sl = 0; sl < PF; ++sl) {
    if (sl < n_units) fetch(sl);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  unsigned long long acc = 0;
  int slot = 0;
  for (int i = 0; i < n_units; ++i) {
    asm volatile("cp.async.wait_group %0;" ::"n"(PF - 1) : "memory");
    const int by = c_by, bx0 = c_chunk * 64 + 2 * lane;
    if (++c_chunk == P.chunks) {
      c_chunk = 0;
      ++c_by;
    }
    if (bx0 < P.nbx) acc += pair_codec(ring + slot * 8 * 32, by, bx0);
    if (i + PF < n_units) fetch(slot);  // refill the slot just used
    asm volatile("cp.async.commit_group;" ::: "memory");
    slot = slot + 1 == PF ? 0 : slot + 1;
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  acc = warp_sum_u64(acc);
  if (lane == 0 && acc) atomicAdd(sse_out, acc);
}

template <int R>
cudaError_t launch_dct_pair(const PlaneDesc& P, const DctParams& dp, unsigned long long* sse,
                            cudaStream_t s) {
  constexpr int kThreads = 128;
  constexpr size_t kSmem = (size_t)(kThreads / 32) * kDctPairStages * kDctPairSlotBytes;
  static int resident = 0, sms = 0;
  if (resident == 0) {
    cudaError_t e = cudaFuncSetAttribute(dct_fp32_pair_kernel<R>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, dct_fp32_pair_kernel<R>, kThreads,
                                                      kSmem);
    if (e != cudaSuccess) return e;
    if (resident < 1) resident = 1;
    sms = device_sms();
  }
  const int64_t units = (int64_t)P.nby * P.chunks;
  int64_t grid = (int64_t)resident * sms;
  const int64_t by_work = (units + kThreads / 32 - 1) / (kThreads / 32);
  if (by_work < grid) grid = by_work;
  if (grid < 1) grid = 1;
  dct_fp32_pair_kernel<R><<<(unsigned)grid, kThreads, kSmem, s>>>(P, dp, sse);
  return cudaGetLastError();
}

template <int R, int DT, bool BF, bool COEF>
cudaError_t launch_dct(const PlaneDesc& P, const DctParams& dp, float* coef,
                       unsigned long long* sse, cudaStream_t s, int grid) {
  // u8 FP32 without coefficients: two blocks per lane as FP32 pairs
  if constexpr (DT == 0 && !BF && !COEF) return launch_dct_pair<R>(P, dp, sse, s);
  dct_codec_kernel<R, DT, BF, COEF><<<(unsigned)grid, 128, 0, s>>>(P, dp, coef, sse);
  return cudaGetLastError();
}

}  // namespace tdct
