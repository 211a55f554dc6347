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

// Symmetric T, one block at a time (int16 samples, or u8 when the packed
// forward's bound does not hold).
template <int R, int DT>
__device__ __forceinline__ uint32_t generic_lane_sym(const PlaneDesc& P, int by, int bx0,
                                                     const GenericParams& gp) {
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
    codec_block_generic_sym<R, DT>(x, out, gp);
#pragma unroll
    for (int p = 0; p < 64; ++p) {
      const int32_t d = (int32_t)x[p] - out[p];
      const bool valid = full || ((by * 8 + p / 8) < P.H && (bx * 8 + p % 8) < P.W);
      sse += valid ? (uint32_t)(d * d) : 0u;
    }
    if (P.recon) store_block<DT>(P, by, bx, full && (P.vec16 & 2), out);
  }
  return sse;
}

// Symmetric T on u8 samples: the lane's two blocks through the packed
// even/odd forward (two blocks per register, exact by the host's bound),
// then each block's inverse, rounding, byte SSE and store.
template <int R>
__device__ __forceinline__ uint32_t generic_pair_u8_sym(const PlaneDesc& P, int by, int bx0,
                                                        const GenericParams& gp) {
  if (bx0 >= P.nbx) return 0u;
  const bool has1 = bx0 + 1 < P.nbx;
  const int vr = min(8, P.H - by * 8);
  const int vc[2] = {min(8, P.W - bx0 * 8), has1 ? min(8, P.W - (bx0 + 1) * 8) : 0};
  const bool full[2] = {vr == 8 && vc[0] == 8, has1 && vr == 8 && vc[1] == 8};
  RowWords<0> rw[2];
  load_block<0>(P, by, bx0, full[0] && (P.vec16 & 1), rw[0]);
  if (has1) {
    load_block<0>(P, by, bx0 + 1, full[1] && (P.vec16 & 1), rw[1]);
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) rw[1].w[k] = make_uint2(0u, 0u);
  }
  // packed forward: rows (the needed columns), then the kept positions
  uint32_t z[64];
  {
    uint32_t pk[64], t[64];
#pragma unroll
    for (int k = 0; k < 8; ++k) pair_row(rw[0].w[k], rw[1].w[k], pk + 8 * k);
#pragma unroll
    for (int k = 0; k < 8; ++k)
      gen_fwd8_sym(pk + 8 * k, t + 8 * k, gp, [](int j) { return gen_col_needed(R, j); });
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (!gen_col_needed(R, j)) continue;
      uint32_t col[8], o[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) col[k] = t[8 * k + j];
      gen_fwd8_sym(col, o, gp, [j](int i) { return kept(R, i, j); });
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (kept(R, i, j)) z[8 * i + j] = o[i];
    }
  }
  const bool dc_u16 = (gp.flags & kGenDcU16) != 0;
  uint32_t sse = 0;
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    if (b == 1 && !has1) break;
    uint32_t w[64];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int p = 8 * i + j;
        if (!kept(R, i, j)) {
          w[p] = 0u;
          continue;
        }
        const uint32_t v = z[p];
        int32_t c;
        if (p == 0 && dc_u16) c = b == 0 ? (int32_t)(v & 0xffffu) : (int32_t)((v - (v & 0xffffu)) >> 16);
        else c = b == 0 ? lane_lo(v) : lane_hi(v);
        w[p] = (uint32_t)c * (uint32_t)gp.cmul2[p];
      }
    uint2 yr[8];
    sse += gen_inverse_u8_sym<R>(w, rw[b].w, gp, yr, full[b], vr, vc[b]);
    if (P.recon) {
      uint8_t* base = P.recon + (int64_t)(by * 8) * P.recon_pitch + (int64_t)(bx0 + b) * 8;
      if (full[b] && (P.vec16 & 2)) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
          *reinterpret_cast<uint2*>(base + (int64_t)k * P.recon_pitch) = yr[k];
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (k < vr)
#pragma unroll
            for (int l = 0; l < 8; ++l)
              if (l < vc[b])
                base[(int64_t)k * P.recon_pitch + l] =
                    (uint8_t)(((l < 4 ? yr[k].x : yr[k].y) >> (8 * (l & 3))) & 0xffu);
      }
    }
  }
  return sse;
}

// MODE 0: direct products (any orthogonal T); 1: symmetric T, one block at
// a time; 2: symmetric T, u8, packed two-block forward.
template <int R, int DT, int MODE>
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
    if constexpr (MODE == 2)
      acc += generic_pair_u8_sym<R>(P, by, chunk * 64 + 2 * lane, gp);
    else if constexpr (MODE == 1)
      acc += generic_lane_sym<R, DT>(P, by, chunk * 64 + 2 * lane, gp);
    else
      acc += generic_lane<R, DT>(P, by, chunk * 64 + 2 * lane, gp);
  }
  if (p >= 0) {
    acc = warp_sum_u64(acc);
    if (lane == 0 && acc) atomicAdd(sse_out + P.slot, acc);
  }
}

}  // namespace gen_detail

template <int R, int DT, int MODE>
cudaError_t launch_codec_generic_mode(const PlaneTable& tab, const GenericParams& gp,
                                      unsigned long long* sse, cudaStream_t s) {
  constexpr int kThreads = 256;
  static int resident = 0, sms = 0;
  if (resident == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &resident, gen_detail::codec_generic_kernel<R, DT, MODE>, kThreads, 0);
    if (e != cudaSuccess) return e;
    if (resident < 1) resident = 1;
    sms = device_sms();
  }
  int64_t grid = (int64_t)resident * sms;
  const int64_t by_work = (tab.total_units + kThreads / 32 - 1) / (kThreads / 32);
  if (by_work < grid) grid = by_work;
  if (grid < 1) grid = 1;
  gen_detail::codec_generic_kernel<R, DT, MODE><<<(unsigned)grid, kThreads, 0, s>>>(tab, gp, sse);
  return cudaGetLastError();
}

template <int R, int DT>
cudaError_t launch_codec_generic(const PlaneTable& tab, const GenericParams& gp,
                                 unsigned long long* sse, cudaStream_t s) {
  if (!(gp.flags & kGenSym)) return launch_codec_generic_mode<R, DT, 0>(tab, gp, sse, s);
  if constexpr (DT == 0)
    if (gp.flags & kGenPackU8) return launch_codec_generic_mode<R, 0, 2>(tab, gp, sse, s);
  return launch_codec_generic_mode<R, DT, 1>(tab, gp, sse, s);
}

}  // namespace tdct
