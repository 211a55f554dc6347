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
  int32_t pad_;
};

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

template <int R, int DT>
cudaError_t launch_codec_generic(const PlaneTable& tab, const GenericParams& gp,
                                 unsigned long long* sse, cudaStream_t s);
cudaError_t launch_forward_generic(const PlaneDesc& P, const GenericParams& gp, int32_t* coef,
                                   cudaStream_t s, int grid);
cudaError_t launch_inverse_generic(const int32_t* coef, const PlaneDesc& P,
                                   const GenericParams& gp, cudaStream_t s, int grid);

}  // namespace tdct
