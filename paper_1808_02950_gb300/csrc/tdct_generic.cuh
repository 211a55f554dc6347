// tdct_generic.cuh -- the block codec for any orthogonal integer T (§2, Eq. (1)-(2)).
//
// The fused kernels of tdct_kernels.cuh implement T1 with its fast algorithm
// (§5.1).  The approximations of Table 2 (and any other orthogonal integer
// T with T T^T = diag(n)) run here: T enters at run time through the kernel
// parameter bank, the 8-point transforms are direct integer products
// (integer multiply-adds with the entries of T), and the zonal mask is
// applied with the same compile-time r-classes as the T1 kernels.  With
// L = lcm(n), q = L / n, the reconstruction is N / L^2 with the integer
// N = T^T (M o Z o q q^T) T; it is rounded half away from zero as
// floor((2|N| + L^2) / (2 L^2)) with a multiply-high division whose constant
// the host computes and checks for every T (GenericParams).
#pragma once
#include <cuda_runtime.h>

#include "tdct_kernels.cuh"

namespace tdct {

struct GenericParams {
  int32_t T[64];      // row-major, row k = t_k^T
  int32_t cmul2[64];  // 2 q_i q_j if (i, j) is among the first r zig-zag positions, else 0
  int32_t L2;         // L^2
  int32_t magic;      // floor(a / (2 L^2)) == (a * magic) >> (32 + shift) for 0 <= a < bound
  int32_t shift;
  int32_t flags;      // kGenSym | kGenPackU8 | kGenDcU16 (set by the host for T)
};

// T's even rows are symmetric and its odd rows antisymmetric (t_k[7-l] =
// (-1)^k t_k[l]), like the DCT and every approximation of the paper: the
// 8-point transforms then split into sums and differences of mirrored
// samples, 4 multiply-adds per output instead of 8.
constexpr int32_t kGenSym = 1;
// For u8 samples every coefficient but Z_00 lies in [-32768, 32767] (bound
// 255 * max(sum of positive, sum of negative entries of t_i kron t_j),
// checked by the host): the forward runs on two blocks per register.
constexpr int32_t kGenPackU8 = 2;
// ... and Z_00 in [0, 65535] (t_0 >= 0, too large for a signed lane): its
// lanes are read as unsigned.
constexpr int32_t kGenDcU16 = 4;

// Columns j holding a kept coefficient of class R.
__host__ __device__ constexpr bool gen_col_needed(int R, int j) {
  for (int i = 0; i < 8; ++i)
    if (kept(R, i, j)) return true;
  return false;
}

// Codec of one block with a run-time T: returns the rounded reconstruction.
template <int R, int DT>
__device__ __forceinline__ void codec_block_generic(const uint32_t x[64], int32_t out[64],
                                                    const GenericParams& gp) {
  // rows: t[k][j] = sum_l x[k][l] T[j][l] for the needed columns j
  uint32_t t[64];
#pragma unroll
  for (int k = 0; k < 8; ++k)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (!gen_col_needed(R, j)) continue;
      uint32_t a = 0;
#pragma unroll
      for (int l = 0; l < 8; ++l) a += x[8 * k + l] * (uint32_t)gp.T[8 * j + l];
      t[8 * k + j] = a;
    }
  // columns: z[i][j] = sum_k T[i][k] t[k][j] for the kept (i, j), scaled and masked
  uint32_t w[64];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (!kept(R, i, j)) continue;
      uint32_t a = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) a += (uint32_t)gp.T[8 * i + k] * t[8 * k + j];
      w[8 * i + j] = a * (uint32_t)gp.cmul2[8 * i + j];
    }
  // inverse columns: v[k][j] = sum_i T[i][k] w[i][j]
  uint32_t v[64];
#pragma unroll
  for (int k = 0; k < 8; ++k)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (!gen_col_needed(R, j)) continue;
      uint32_t a = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (kept(R, i, j)) a += (uint32_t)gp.T[8 * i + k] * w[8 * i + j];
      v[8 * k + j] = a;
    }
  // inverse rows: 2N[k][l] = sum_j v[k][j] T[j][l]; round half away from zero
#pragma unroll
  for (int k = 0; k < 8; ++k)
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      uint32_t a = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (gen_col_needed(R, j)) a += v[8 * k + j] * (uint32_t)gp.T[8 * j + l];
      const int32_t n2 = (int32_t)a;  // 2 N (the multipliers are doubled)
      if (DT == 0) {
        // u8: n2 + L^2 >= 0 rounds half up; a negative value clamps to 0
        const int32_t m = __mulhi(n2 + gp.L2, gp.magic) >> gp.shift;
        out[8 * k + l] = min(max(m, 0), 255);
      } else {
        const int32_t mag = n2 < 0 ? -n2 : n2;
        const int32_t m = __mulhi(mag + gp.L2, gp.magic) >> gp.shift;
        out[8 * k + l] = min(max(n2 < 0 ? -m : m, -255), 255);
      }
    }
}

// ---- symmetric T: even/odd split --------------------------------------------

// y_j = sum_l T[j][l] x_l for the wanted j: s_m = x_m + x_{7-m} (even j),
// d_m = x_m - x_{7-m} (odd j), then 4 multiply-adds.  V = uint32_t: one
// block, or two blocks packed as a + 65536 b (exact modulo 2^32).
template <typename F>
__device__ __forceinline__ void gen_fwd8_sym(const uint32_t x[8], uint32_t y[8],
                                             const GenericParams& gp, F want) {
  uint32_t s[4], d[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    s[m] = x[m] + x[7 - m];
    d[m] = x[m] - x[7 - m];
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (!want(j)) continue;
    const uint32_t* v = (j & 1) ? d : s;
    uint32_t a = v[0] * (uint32_t)gp.T[8 * j];
#pragma unroll
    for (int m = 1; m < 4; ++m) a += v[m] * (uint32_t)gp.T[8 * j + m];
    y[j] = a;
  }
}

// x_l = sum_j T[j][l] y_j over the j with has(j): E_m over even j, O_m over
// odd j (m < 4), x_m = E_m + O_m, x_{7-m} = E_m - O_m.
template <typename F>
__device__ __forceinline__ void gen_inv8_sym(const uint32_t y[8], uint32_t x[8],
                                             const GenericParams& gp, F has) {
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    uint32_t e = 0, o = 0;
#pragma unroll
    for (int j = 0; j < 8; j += 2)
      if (has(j)) e += y[j] * (uint32_t)gp.T[8 * j + m];
#pragma unroll
    for (int j = 1; j < 8; j += 2)
      if (has(j)) o += y[j] * (uint32_t)gp.T[8 * j + m];
    x[m] = e + o;
    x[7 - m] = e - o;
  }
}

// Inverse of one block from its kept, scaled coefficients w (doubled),
// columns then rows, each 2N row rounded as the u8 codec does (half up for
// u8: floor((2N + L^2) / (2 L^2)), negative values clamp to 0) and packed
// two samples per word for the clamp, four per word for the store and the
// byte SSE against the sample row words xr (u8).  Returns the block's SSE.
template <int R>
__device__ __forceinline__ uint32_t gen_inverse_u8_sym(const uint32_t w[64], const uint2 xr[8],
                                                       const GenericParams& gp, uint2 yr[8],
                                                       bool full, int valid_rows, int valid_cols) {
  const uint64_t colmask = valid_cols >= 8 ? ~0ull : ((1ull << (8 * valid_cols)) - 1ull);
  uint32_t v[64];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (!gen_col_needed(R, j)) continue;
    uint32_t col[8], o[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) col[i] = w[8 * i + j];
    gen_inv8_sym(col, o, gp, [j](int i) { return kept(R, i, j); });
#pragma unroll
    for (int k = 0; k < 8; ++k) v[8 * k + j] = o[k];
  }
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    uint32_t n2[8];
    gen_inv8_sym(v + 8 * k, n2, gp, [](int j) { return gen_col_needed(R, j); });
    uint32_t m[8];
#pragma unroll
    for (int l = 0; l < 8; ++l)
      m[l] = (uint32_t)(__mulhi((int32_t)n2[l] + gp.L2, gp.magic) >> gp.shift);
    const uint32_t c01 = min_relu_s16x2(__byte_perm(m[0], m[1], 0x5410u), 0x00ff00ffu);
    const uint32_t c23 = min_relu_s16x2(__byte_perm(m[2], m[3], 0x5410u), 0x00ff00ffu);
    const uint32_t c45 = min_relu_s16x2(__byte_perm(m[4], m[5], 0x5410u), 0x00ff00ffu);
    const uint32_t c67 = min_relu_s16x2(__byte_perm(m[6], m[7], 0x5410u), 0x00ff00ffu);
    yr[k] = make_uint2(__byte_perm(c01, c23, 0x6420u), __byte_perm(c45, c67, 0x6420u));
    uint2 yk = yr[k];
    if (!full) {  // samples outside the plane (zero in xr) leave the SSE
      const uint64_t msk = k < valid_rows ? colmask : 0ull;
      yk.x &= (uint32_t)msk;
      yk.y &= (uint32_t)(msk >> 32);
    }
    const uint32_t d0 = __vabsdiffu4(xr[k].x, yk.x), d1 = __vabsdiffu4(xr[k].y, yk.y);
    acc = __dp4a(d0, d0, __dp4a(d1, d1, acc));
  }
  return acc;
}

// One block (u8 or int16 samples in x) with the even/odd split, rounded as
// codec_block_generic.
template <int R, int DT>
__device__ __forceinline__ void codec_block_generic_sym(const uint32_t x[64], int32_t out[64],
                                                        const GenericParams& gp) {
  uint32_t t[64];
#pragma unroll
  for (int k = 0; k < 8; ++k)
    gen_fwd8_sym(x + 8 * k, t + 8 * k, gp, [](int j) { return gen_col_needed(R, j); });
  uint32_t w[64];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (!gen_col_needed(R, j)) continue;
    uint32_t col[8], o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) col[k] = t[8 * k + j];
    gen_fwd8_sym(col, o, gp, [j](int i) { return kept(R, i, j); });
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (kept(R, i, j)) w[8 * i + j] = o[i] * (uint32_t)gp.cmul2[8 * i + j];
  }
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (!kept(R, i, j)) w[8 * i + j] = 0u;
  uint32_t v[64];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (!gen_col_needed(R, j)) continue;
    uint32_t col[8], o[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) col[i] = w[8 * i + j];
    gen_inv8_sym(col, o, gp, [j](int i) { return kept(R, i, j); });
#pragma unroll
    for (int k = 0; k < 8; ++k) v[8 * k + j] = o[k];
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    uint32_t n2[8];
    gen_inv8_sym(v + 8 * k, n2, gp, [](int j) { return gen_col_needed(R, j); });
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      const int32_t a = (int32_t)n2[l];  // 2 N
      if (DT == 0) {
        const int32_t m = __mulhi(a + gp.L2, gp.magic) >> gp.shift;
        out[8 * k + l] = min(max(m, 0), 255);
      } else {
        const int32_t mag = a < 0 ? -a : a;
        const int32_t m = __mulhi(mag + gp.L2, gp.magic) >> gp.shift;
        out[8 * k + l] = min(max(a < 0 ? -m : m, -255), 255);
      }
    }
  }
}

template <int R, int DT>
cudaError_t launch_codec_generic(const PlaneTable& tab, const GenericParams& gp,
                                 unsigned long long* sse, cudaStream_t s);
cudaError_t launch_forward_generic(const PlaneDesc& P, const GenericParams& gp, int32_t* coef,
                                   cudaStream_t s, int grid);
cudaError_t launch_inverse_generic(const int32_t* coef, const PlaneDesc& P,
                                   const GenericParams& gp, cudaStream_t s, int grid);

}  // namespace tdct
