// tdct_generic_impl.cuh -- kernels of the block codec for any orthogonal
// integer T (see tdct_generic.cuh); included by the instantiation units
// tdct_gen_*.cu only.  Same work decomposition as the T1 kernels: persistent
// warps over the units of a block-offset table, each lane owning two
// horizontally adjacent blocks.
#pragma once
#include "tdct_classes.h"
#include "tdct_generic.cuh"

namespace tdct {

namespace gen_detail {

template <int R, int DT>
__device__ __forceinline__ uint32_t generic_lane(const PlaneDesc& P, int by, int bx0,
                                                 const GenericParams& gp) {
  constexpr int SB = DT == 0 ? 1 : 2;
  uint32_t sse = 0;
#pragma unroll 1
  for (int b = 0; b < 2; ++b) {
    const int bx = bx0 + b;
    if (bx >= P.nbx) break;
    const bool full = (by * 8 + 8 <= P.H) && ((bx + 1) * 8 <= P.W);
    RowWords<DT> rw;
    load_block<DT>(P, by, bx, full && (P.vec16 & 1), rw);
    uint32_t x[64];
#pragma unroll
    for (int k = 0; k < 8; ++k) unpack_row<DT>(rw, k, x + 8 * k);
    int32_t out[64];
    codec_block_generic<R, DT>(x, out, gp);
#pragma unroll
    for (int p = 0; p < 64; ++p) {
      const int32_t d = (int32_t)x[p] - out[p];
      const bool valid = full || ((by * 8 + p / 8) < P.H && (bx * 8 + p % 8) < P.W);
      sse += valid ? (uint32_t)(d * d) : 0u;
    }
    if (P.recon) store_block<DT>(P, by, bx, full && (P.vec16 & 2), out);
    (void)SB;
  }
  return sse;
}

template <int R, int DT>
__global__ void __launch_bounds__(256) codec_generic_kernel(const PlaneTable tab,
                                                            const GenericParams gp,
                                                            unsigned long long* __restrict__ sse_out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t U = tab.total_units;
  const int64_t u_begin = (U * warp) / nwarps;
  const int64_t u_end = (U * (warp + 1)) / nwarps;
  int p = -1;
  int64_t p_end = -1;
  PlaneDesc P;
  unsigned long long acc = 0;
  for (int64_t u = u_begin; u < u_end; ++u) {
    if (u >= p_end) {
      if (p >= 0) {
        acc = warp_sum_u64(acc);
        if (lane == 0 && acc) atomicAdd(sse_out + P.slot, acc);
        acc = 0;
      }
      p = find_plane(tab, u);
      P = tab.d ? tab.d[p] : tab.one;
      p_end = (p + 1 < tab.n) ? tab.d[p + 1].unit_begin : U;
    }
    const int64_t local = u - P.unit_begin;
    const int by = (int)(local / P.chunks);
    const int chunk = (int)(local - (int64_t)by * P.chunks);
    acc += generic_lane<R, DT>(P, by, chunk * 64 + 2 * lane, gp);
  }
  if (p >= 0) {
    acc = warp_sum_u64(acc);
    if (lane == 0 && acc) atomicAdd(sse_out + P.slot, acc);
  }
}

}  // namespace gen_detail

template <int R, int DT>
cudaError_t launch_codec_generic(const PlaneTable& tab, const GenericParams& gp,
                                 unsigned long long* sse, cudaStream_t s) {
  constexpr int kThreads = 256;
  static int resident = 0, sms = 0;
  if (resident == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &resident, gen_detail::codec_generic_kernel<R, DT>, kThreads, 0);
    if (e != cudaSuccess) return e;
    if (resident < 1) resident = 1;
    sms = device_sms();
  }
  int64_t grid = (int64_t)resident * sms;
  const int64_t by_work = (tab.total_units + kThreads / 32 - 1) / (kThreads / 32);
  if (by_work < grid) grid = by_work;
  if (grid < 1) grid = 1;
  gen_detail::codec_generic_kernel<R, DT><<<(unsigned)grid, kThreads, 0, s>>>(tab, gp, sse);
  return cudaGetLastError();
}

}  // namespace tdct
