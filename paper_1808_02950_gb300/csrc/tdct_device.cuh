// tdct_device.cuh -- device building blocks of the T1 block codec.
//
// T1 (§4.1) and its fast algorithm (§5.1): 24 additions and 6 doublings per
// 8-point transform.  The paper factors T1 = D A4 A3 A2 A1; the butterflies
// below use the same even/odd split (first stage = A1) and the same counts,
// but group the remaining additions so that every output is one or two
// integer adds (IADD3 / LEA on sm_103a) instead of the D.A4 stage with
// halves.  All linear arithmetic is done in uint32 (two's complement wrap):
// additions, subtractions and doublings are exact modulo 2^32, so any
// intermediate may wrap as long as the final value fits int32, which holds
// for every output here.
#pragma once
#include <cstdint>

namespace tdct {

// ---- zig-zag scan (JPEG / Pao convention), by rule ------------------------
// Anti-diagonals s = i + j in order; odd s run from (0, s) with i
// increasing, even s from (s, 0) with i decreasing.  Returns the scan index
// of position (i, j) (i = vertical frequency, j = horizontal frequency).
__host__ __device__ constexpr int zz_index(int i, int j) {
  const int s = i + j;
  const int before = s <= 7 ? s * (s + 1) / 2 : 64 - (15 - s) * (16 - s) / 2;
  int pos = 0;
  if (s <= 7) {
    pos = (s & 1) ? i : (s - i);
  } else {
    pos = (s & 1) ? (i - (s - 7)) : (7 - i);
  }
  return before + pos;
}

// Retention mask M_r of §6.1: position (i, j) kept iff its scan index < r.
__host__ __device__ constexpr bool kept(int r, int i, int j) { return zz_index(i, j) < r; }

// Rows (vertical frequencies i) and columns (horizontal frequencies j) that
// hold a kept position: 1 + the largest such index.  A separable pass along
// one direction only has to form the outputs inside the other's extent, so
// the cheaper pass order follows from these.
__host__ __device__ constexpr int kept_rows(int r) {
  int e = 0;
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j)
      if (kept(r, i, j) && i + 1 > e) e = i + 1;
  return e;
}
__host__ __device__ constexpr int kept_cols(int r) {
  int e = 0;
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j)
      if (kept(r, i, j) && j + 1 > e) e = j + 1;
  return e;
}

// ---- T1 constants ---------------------------------------------------------
// q = L / n with n = diag(T1 T1^T) = (8,18,20,18,8,18,20,18), L = lcm(n) = 360.
__host__ __device__ constexpr int q_of(int i) {
  return (i == 0 || i == 4) ? 45 : ((i == 2 || i == 6) ? 18 : 20);
}
constexpr uint32_t kL2 = 129600u;        // L^2
constexpr uint32_t kHalfL2 = 64800u;     // L^2 / 2
// floor(a / 129600) == (a * kDivMagic) >> 47 for 0 <= a < 1.27e9, and the
// result is negative for every negative a (signed high product).
constexpr int32_t kDivMagic = 1085937411;

__device__ __forceinline__ int32_t div_L2_floor(int32_t a) {
  return __mulhi(a, kDivMagic) >> 15;
}

// ---- 8-point forward butterfly: y_i = sum_l T1[i][l] x_l ---------------------
// Even/odd split s_m = x_m + x_{7-m}, d_m = x_m - x_{7-m} (the A1 stage);
// even rows (t1, t3, t5, t7 of the paper, indices 0,2,4,6 here) act on s,
// odd rows on d.  Unused outputs are removed by the compiler.
template <typename V>
__device__ __forceinline__ void fwd8(const V x[8], V y[8]) {
  const V s0 = x[0] + x[7], s1 = x[1] + x[6], s2 = x[2] + x[5], s3 = x[3] + x[4];
  const V d0 = x[0] - x[7], d1 = x[1] - x[6], d2 = x[2] - x[5], d3 = x[3] - x[4];
  const V e0 = s0 + s3, e1 = s1 + s2, e2 = s0 - s3, e3 = s1 - s2;
  y[0] = e0 + e1;
  y[4] = e0 - e1;
  y[2] = e2 + e2 + e3;
  y[6] = e2 - e3 - e3;
  const V a = d0 + d1, b = d0 - d1, c = d2 + d3, e = d2 - d3;
  y[1] = a + a + d2;
  y[3] = d0 - c - c;
  y[5] = b + b + d3;
  y[7] = e + e - d1;
}

// ---- 8-point inverse butterfly: x_l = sum_i T1[i][l] y_i (transpose) ------
template <typename V>
__device__ __forceinline__ void inv8(const V y[8], V x[8]) {
  const V E0 = y[0] + y[4], E1 = y[0] - y[4];
  const V F0 = y[2] + y[2] + y[6], F1 = y[2] - y[6] - y[6];
  const V S0 = E0 + F0, S3 = E0 - F0, S1 = E1 + F1, S2 = E1 - F1;
  const V g = y[1] + y[5], h = y[1] - y[5], u = y[3] - y[7], w = y[3] + y[7];
  const V D0 = g + g + y[3];
  const V D1 = h + h - y[7];
  const V D2 = y[1] - u - u;
  const V D3 = y[5] - w - w;
  x[0] = S0 + D0;
  x[7] = S0 - D0;
  x[1] = S1 + D1;
  x[6] = S1 - D1;
  x[2] = S2 + D2;
  x[5] = S2 - D2;
  x[3] = S3 + D3;
  x[4] = S3 - D3;
}

// ---- 2-D forward of one block: Z = T1 X T1^T --------------------------------
// X[k][l] row-major in x[64]; Z[i][j] row-major in z[64].  Rows first
// (horizontal frequencies), then columns.
template <typename V>
__device__ __forceinline__ void fwd2d(const V x[64], V z[64]) {
  V t[64];
#pragma unroll
  for (int k = 0; k < 8; ++k) fwd8<V>(x + 8 * k, t + 8 * k);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    V col[8], out[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) col[k] = t[8 * k + j];
    fwd8<V>(col, out);
#pragma unroll
    for (int i = 0; i < 8; ++i) z[8 * i + j] = out[i];
  }
}

// ---- 2-D inverse of one block: N = T1^T W T1 --------------------------------
template <typename V>
__device__ __forceinline__ void inv2d(const V w[64], V n[64]) {
  V t[64];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    V col[8], out[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) col[i] = w[8 * i + j];
    inv8<V>(col, out);
#pragma unroll
    for (int k = 0; k < 8; ++k) t[8 * k + j] = out[k];
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) inv8<V>(t + 8 * k, n + 8 * k);
}

}  // namespace tdct
