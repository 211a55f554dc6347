// Instantiations of the generic-T codec for r-classes group A (tdct_generic_impl.cuh).
#include "tdct_generic_impl.cuh"

namespace tdct {
#define TDCT_GEN_INST(R)                                                                      \
  template cudaError_t launch_codec_generic<R, 0>(const PlaneTable&, const GenericParams&,    \
                                                  unsigned long long*, cudaStream_t);         \
  template cudaError_t launch_codec_generic<R, 1>(const PlaneTable&, const GenericParams&,    \
                                                  unsigned long long*, cudaStream_t);
TDCT_FOR_EACH_CLASS_A(TDCT_GEN_INST)
#undef TDCT_GEN_INST

// Forward only / inverse only with a run-time T (tdct_forward, tdct_zonal_inverse).
namespace gen_detail {
template <int DT>
__global__ void __launch_bounds__(128) forward_generic_kernel(const PlaneDesc P, const GenericParams gp,
                                                              int32_t* __restrict__ coef) {
  const int64_t nb = (int64_t)P.nbx * P.nby;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int by = (int)(b / P.nbx), bx = (int)(b - (int64_t)by * P.nbx);
    const bool interior = (by * 8 + 8 <= P.H) && ((bx + 1) * 8 <= P.W) && (P.vec16 & 1);
    RowWords<DT> rw;
    load_block<DT>(P, by, bx, interior, rw);
    uint32_t x[64], t[64];
#pragma unroll
    for (int k = 0; k < 8; ++k) unpack_row<DT>(rw, k, x + 8 * k);
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint32_t a = 0;
#pragma unroll
        for (int l = 0; l < 8; ++l) a += x[8 * k + l] * (uint32_t)gp.T[8 * j + l];
        t[8 * k + j] = a;
      }
    int32_t* dst = coef + b * 64;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint32_t a = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) a += (uint32_t)gp.T[8 * i + k] * t[8 * k + j];
        dst[8 * i + j] = (int32_t)a;
      }
  }
}

template <int DT>
__global__ void __launch_bounds__(128) inverse_generic_kernel(const int32_t* __restrict__ coef,
                                                              const PlaneDesc P,
                                                              const GenericParams gp) {
  const int64_t nb = (int64_t)P.nbx * P.nby;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int by = (int)(b / P.nbx), bx = (int)(b - (int64_t)by * P.nbx);
    const int32_t* src = coef + b * 64;
    uint32_t w[64], v[64];
#pragma unroll
    for (int q = 0; q < 64; ++q) w[q] = (uint32_t)__ldg(src + q) * (uint32_t)gp.cmul2[q];
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint32_t a = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) a += (uint32_t)gp.T[8 * i + k] * w[8 * i + j];
        v[8 * k + j] = a;
      }
    int32_t out[64];
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int l = 0; l < 8; ++l) {
        uint32_t a = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) a += v[8 * k + j] * (uint32_t)gp.T[8 * j + l];
        const int32_t n2 = (int32_t)a;
        if (DT == 0) {
          const int32_t m = __mulhi(n2 + gp.L2, gp.magic) >> gp.shift;
          out[8 * k + l] = min(max(m, 0), 255);
        } else {
          const int32_t mag = n2 < 0 ? -n2 : n2;
          const int32_t m = __mulhi(mag + gp.L2, gp.magic) >> gp.shift;
          out[8 * k + l] = min(max(n2 < 0 ? -m : m, -255), 255);
        }
      }
    const bool fast = (by * 8 + 8 <= P.H) && ((bx + 1) * 8 <= P.W) && (P.vec16 & 2);
    store_block<DT>(P, by, bx, fast, out);
  }
}
}  // namespace gen_detail

cudaError_t launch_forward_generic(const PlaneDesc& P, const GenericParams& gp, int32_t* coef,
                                   cudaStream_t s, int grid) {
  if (P.dtype == 0) gen_detail::forward_generic_kernel<0><<<grid, 128, 0, s>>>(P, gp, coef);
  else gen_detail::forward_generic_kernel<1><<<grid, 128, 0, s>>>(P, gp, coef);
  return cudaGetLastError();
}

cudaError_t launch_inverse_generic(const int32_t* coef, const PlaneDesc& P,
                                   const GenericParams& gp, cudaStream_t s, int grid) {
  if (P.dtype == 0) gen_detail::inverse_generic_kernel<0><<<grid, 128, 0, s>>>(coef, P, gp);
  else gen_detail::inverse_generic_kernel<1><<<grid, 128, 0, s>>>(coef, P, gp);
  return cudaGetLastError();
}

}  // namespace tdct
