// tdct_kernels.cuh -- the fused T1 block codec and its helpers (sm_103a).
//
// Work decomposition (all planes of a launch share it):
//   unit  = one warp's work: 64 consecutive 8x8 blocks of one block-row of
//           one plane (lane L owns blocks 2L and 2L+1 of the unit), i.e. a
//           warp covers 8 rows x 512 samples.  A block-row of a plane with
//           nbx blocks holds ceil(nbx / 64) units; the last may be ragged.
//   table = per-plane descriptors with the exclusive prefix sum of units
//           (the block-offset table); a warp finds its plane by binary search.
//   grid  = persistent: one CTA per resident slot, each warp takes one
//           contiguous range of units, so it stays inside one plane for long
//           stretches and flushes its SSE with one atomic per plane visited.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "tdct_device.cuh"

namespace tdct {

struct PlaneDesc {
  const uint8_t* img;
  uint8_t* recon;
  int64_t pitch;
  int64_t recon_pitch;
  int64_t unit_begin;  // exclusive prefix of units over planes
  int32_t H, W;
  int32_t nbx, nby;
  int32_t chunks;      // units per block-row = ceil(nbx / 64)
  int32_t dtype;       // 0 = u8, 1 = i16
  int32_t r;
  int32_t vec16;       // bit 0: img rows 8-byte aligned; bit 1: recon rows
  int32_t slot;        // output index for SSE / PSNR
  int32_t pad_;
};

struct PlaneTable {
  const PlaneDesc* d;  // device array, or nullptr to use `one`
  int32_t n;
  int32_t pad_;
  int64_t total_units;
  PlaneDesc one;
};

__device__ __forceinline__ const PlaneDesc& plane_at(const PlaneTable& t, int i) {
  return t.d ? t.d[i] : t.one;
}

// Largest plane index p with unit_begin(p) <= u.
__device__ __forceinline__ int find_plane(const PlaneTable& t, int64_t u) {
  if (!t.d) return 0;
  int lo = 0, hi = t.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&t.d[mid].unit_begin) <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---- sample I/O -------------------------------------------------------------

// Load the 8 rows of one block (u8) into x[64] as int32; zero outside the plane.
__device__ __forceinline__ void load_block_u8_edge(const PlaneDesc& P, int by, int bx,
                                                   uint32_t x[64]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int y = by * 8 + k;
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      const int xx = bx * 8 + l;
      x[8 * k + l] = (y < P.H && xx < P.W) ? (uint32_t)__ldg(P.img + (int64_t)y * P.pitch + xx) : 0u;
    }
  }
}

__device__ __forceinline__ void load_block_i16_edge(const PlaneDesc& P, int by, int bx,
                                                    uint32_t x[64]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int y = by * 8 + k;
    const int16_t* row = reinterpret_cast<const int16_t*>(P.img + (int64_t)y * P.pitch);
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      const int xx = bx * 8 + l;
      x[8 * k + l] = (y < P.H && xx < P.W) ? (uint32_t)(int32_t)__ldg(row + xx) : 0u;
    }
  }
}

__device__ __forceinline__ void unpack_u8x8(uint2 w, uint32_t* x) {
  x[0] = w.x & 0xffu;
  x[1] = (w.x >> 8) & 0xffu;
  x[2] = (w.x >> 16) & 0xffu;
  x[3] = w.x >> 24;
  x[4] = w.y & 0xffu;
  x[5] = (w.y >> 8) & 0xffu;
  x[6] = (w.y >> 16) & 0xffu;
  x[7] = w.y >> 24;
}

__device__ __forceinline__ void unpack_i16x8(uint4 w, uint32_t* x) {
  x[0] = (uint32_t)(int32_t)(int16_t)(w.x & 0xffffu);
  x[1] = (uint32_t)((int32_t)w.x >> 16);
  x[2] = (uint32_t)(int32_t)(int16_t)(w.y & 0xffffu);
  x[3] = (uint32_t)((int32_t)w.y >> 16);
  x[4] = (uint32_t)(int32_t)(int16_t)(w.z & 0xffffu);
  x[5] = (uint32_t)((int32_t)w.z >> 16);
  x[6] = (uint32_t)(int32_t)(int16_t)(w.w & 0xffffu);
  x[7] = (uint32_t)((int32_t)w.w >> 16);
}

// ---- the per-block codec ------------------------------------------------------

// Inverse and rounding of one block from its scaled coefficients
// W = M_r o Z o q q^T: N = T1^T W T1 (exact in int32), then
// x' = round_half_away(N / L^2) clamped to [0,255] (u8) or [-255,255] (i16).
template <int DT>
__device__ __forceinline__ void reconstruct(uint32_t w[64], int32_t out[64]) {
  if (DT == 0) w[0] += kHalfL2;  // row t_1 = 1: adds L^2/2 to every N (rounding bias)
  uint32_t nn[64];
  inv2d<uint32_t>(w, nn);
#pragma unroll
  for (int p = 0; p < 64; ++p) {
    const int32_t N = (int32_t)nn[p];
    int32_t v;
    if (DT == 0) {
      // u8: N >= 0 rounds half up (= half away from zero); N < 0 gives a
      // value <= 0, which the clamp maps to 0 as the exact rule would.
      v = div_L2_floor(N);
      v = min(max(v, 0), 255);
    } else {
      const int32_t a = N < 0 ? -N : N;
      const int32_t m = div_L2_floor(a + (int32_t)kHalfL2);
      v = N < 0 ? -m : m;
      v = min(max(v, -255), 255);
    }
    out[p] = v;
  }
}

// Per-launch constants: cmul[8 i + j] = q_i q_j if position (i, j) is among
// the first r zig-zag positions, else 0 (the zonal mask M_r with S^2 folded
// in, §6.1).  Lives in the kernel parameter (constant) bank.
struct CodecParams {
  int32_t cmul[64];
};

// Forward, zonal mask, scale by q_i q_j, inverse, round and clamp one block.
// R is the launch's r-class: positions with scan index >= R are known to be
// zero at compile time, so the work they would need is never emitted; the
// exact r <= R is applied through cmul.  Returns the reconstruction in out[64].
template <int R, int DT>
__device__ __forceinline__ void codec_block(const uint32_t x[64], int32_t out[64],
                                            const CodecParams& cp) {
  uint32_t z[64];
  fwd2d<uint32_t>(x, z);
  uint32_t w[64];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j)
      w[8 * i + j] = kept(R, i, j) ? z[8 * i + j] * (uint32_t)cp.cmul[8 * i + j] : 0u;
  reconstruct<DT>(w, out);
}

__device__ __forceinline__ uint2 pack_u8x8(const int32_t* v) {
  uint2 w;
  w.x = (uint32_t)v[0] | ((uint32_t)v[1] << 8) | ((uint32_t)v[2] << 16) | ((uint32_t)v[3] << 24);
  w.y = (uint32_t)v[4] | ((uint32_t)v[5] << 8) | ((uint32_t)v[6] << 16) | ((uint32_t)v[7] << 24);
  return w;
}

__device__ __forceinline__ uint4 pack_i16x8(const int32_t* v) {
  uint4 w;
  w.x = ((uint32_t)v[0] & 0xffffu) | ((uint32_t)v[1] << 16);
  w.y = ((uint32_t)v[2] & 0xffffu) | ((uint32_t)v[3] << 16);
  w.z = ((uint32_t)v[4] & 0xffffu) | ((uint32_t)v[5] << 16);
  w.w = ((uint32_t)v[6] & 0xffffu) | ((uint32_t)v[7] << 16);
  return w;
}

// Store one reconstructed block; `fast` = whole block inside the plane and
// recon rows 8-byte aligned.
template <int DT>
__device__ __forceinline__ void store_block(const PlaneDesc& P, int by, int bx, bool fast,
                                            const int32_t out[64]) {
  constexpr int SB = DT == 0 ? 1 : 2;
  if (fast) {
    uint8_t* rbase = P.recon + (int64_t)(by * 8) * P.recon_pitch + (int64_t)bx * 8 * SB;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      uint8_t* row = rbase + (int64_t)k * P.recon_pitch;
      if constexpr (DT == 0) {
        *reinterpret_cast<uint2*>(row) = pack_u8x8(out + 8 * k);
      } else {
        const uint4 v = pack_i16x8(out + 8 * k);
        reinterpret_cast<uint2*>(row)[0] = make_uint2(v.x, v.y);
        reinterpret_cast<uint2*>(row)[1] = make_uint2(v.z, v.w);
      }
    }
  } else {
#pragma unroll
    for (int p = 0; p < 64; ++p) {
      const int y = by * 8 + p / 8, xx = bx * 8 + p % 8;
      if (y < P.H && xx < P.W) {
        uint8_t* row = P.recon + (int64_t)y * P.recon_pitch;
        if constexpr (DT == 0) row[xx] = (uint8_t)out[p];
        else reinterpret_cast<int16_t*>(row)[xx] = (int16_t)out[p];
      }
    }
  }
}

// Raw row words of one block: u8 = 8 samples in a uint2, i16 = 8 in a uint4.
template <int DT>
struct RowWords;
template <>
struct RowWords<0> { uint2 w[8]; };
template <>
struct RowWords<1> { uint4 w[8]; };

template <int DT>
__device__ __forceinline__ void unpack_row(const RowWords<DT>& rw, int k, uint32_t* x) {
  if constexpr (DT == 0) unpack_u8x8(rw.w[k], x);
  else unpack_i16x8(rw.w[k], x);
}

// Load one block's rows; `interior` means the whole 8x8 block lies inside the
// plane and `align` (0, 8 or 16) is the guaranteed alignment of its rows.
template <int DT>
__device__ __forceinline__ void load_block(const PlaneDesc& P, int by, int bx, bool interior,
                                           RowWords<DT>& rw) {
  constexpr int SB = DT == 0 ? 1 : 2;
  if (interior) {
    const uint8_t* base = P.img + (int64_t)(by * 8) * P.pitch + (int64_t)bx * 8 * SB;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint8_t* row = base + (int64_t)k * P.pitch;
      if constexpr (DT == 0) {
        rw.w[k] = __ldg(reinterpret_cast<const uint2*>(row));
      } else {
        const uint2 a = __ldg(reinterpret_cast<const uint2*>(row));
        const uint2 b = __ldg(reinterpret_cast<const uint2*>(row) + 1);
        rw.w[k] = make_uint4(a.x, a.y, b.x, b.y);
      }
    }
  } else {
    uint32_t x[64];
    if constexpr (DT == 0) load_block_u8_edge(P, by, bx, x);
    else load_block_i16_edge(P, by, bx, x);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if constexpr (DT == 0) {
        rw.w[k].x = x[8 * k] | (x[8 * k + 1] << 8) | (x[8 * k + 2] << 16) | (x[8 * k + 3] << 24);
        rw.w[k].y = x[8 * k + 4] | (x[8 * k + 5] << 8) | (x[8 * k + 6] << 16) | (x[8 * k + 7] << 24);
      } else {
        rw.w[k].x = (x[8 * k] & 0xffffu) | (x[8 * k + 1] << 16);
        rw.w[k].y = (x[8 * k + 2] & 0xffffu) | (x[8 * k + 3] << 16);
        rw.w[k].z = (x[8 * k + 4] & 0xffffu) | (x[8 * k + 5] << 16);
        rw.w[k].w = (x[8 * k + 6] & 0xffffu) | (x[8 * k + 7] << 16);
      }
    }
  }
}

// Codec of one block held as raw row words; returns its SSE over valid samples.
template <int R, int DT>
__device__ __forceinline__ uint32_t codec_one(const PlaneDesc& P, int by, int bx,
                                              const RowWords<DT>& rw, const CodecParams& cp) {
  constexpr int SB = DT == 0 ? 1 : 2;
  int32_t out[64];
  {
    uint32_t x[64];
#pragma unroll
    for (int k = 0; k < 8; ++k) unpack_row<DT>(rw, k, x + 8 * k);
    codec_block<R, DT>(x, out, cp);
  }
  const bool full = (by * 8 + 8 <= P.H) && ((bx + 1) * 8 <= P.W);
  uint32_t sse = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    uint32_t x[8];
    unpack_row<DT>(rw, k, x);
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      const int32_t d = (int32_t)x[l] - out[8 * k + l];
      const bool valid = full || ((by * 8 + k) < P.H && (bx * 8 + l) < P.W);
      sse += valid ? (uint32_t)(d * d) : 0u;
    }
  }
  if (P.recon) store_block<DT>(P, by, bx, full && (P.vec16 & 2), out);
  return sse;
}

// Process the two blocks (bx0, bx0 + 1) of block-row `by` owned by a lane.
// Both blocks are loaded before either is computed.  Returns the lane's SSE.
// Interior rows need 8-byte alignment of img / recon rows (checked on the
// host: P.vec16 & 1 for img, & 2 for recon); other blocks use sample loads.
template <int R, int DT>
__device__ __forceinline__ uint32_t codec_lane(const PlaneDesc& P, int by, int bx0,
                                               const CodecParams& cp) {
  const bool has0 = bx0 < P.nbx, has1 = bx0 + 1 < P.nbx;
  if (!has0) return 0u;
  const bool rows_in = by * 8 + 8 <= P.H;
  const bool in0 = rows_in && (bx0 + 1) * 8 <= P.W && (P.vec16 & 1);
  const bool in1 = rows_in && (bx0 + 2) * 8 <= P.W && (P.vec16 & 1);
  RowWords<DT> ra, rb;
  load_block<DT>(P, by, bx0, in0, ra);
  if (has1) load_block<DT>(P, by, bx0 + 1, in1, rb);
  uint32_t sse = codec_one<R, DT>(P, by, bx0, ra, cp);
  if (has1) sse += codec_one<R, DT>(P, by, bx0 + 1, rb, cp);
  return sse;
}

// Persistent fused codec: every warp takes a contiguous range of units.
template <int R, int DT>
__global__ void __launch_bounds__(256) codec_kernel(const PlaneTable tab, const CodecParams cp,
                                                    unsigned long long* __restrict__ sse_out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t U = tab.total_units;
  const int64_t u_begin = (U * warp) / nwarps;
  const int64_t u_end = (U * (warp + 1)) / nwarps;
  int p = -1;
  int64_t p_end = -1;
  PlaneDesc P;  // current plane, held in registers
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
    if (P.dtype != DT) continue;  // never true for tables the host builds
    const int64_t local = u - P.unit_begin;
    const int by = (int)(local / P.chunks);
    const int chunk = (int)(local - (int64_t)by * P.chunks);
    acc += codec_lane<R, DT>(P, by, chunk * 64 + 2 * lane, cp);
  }
  if (p >= 0) {
    acc = warp_sum_u64(acc);
    if (lane == 0 && acc) atomicAdd(sse_out + P.slot, acc);
  }
}

// Host-side launcher of one instantiation (defined where instantiated).
template <int R, int DT>
cudaError_t launch_codec(const PlaneTable& tab, const CodecParams& cp, unsigned long long* sse,
                         int max_ctas, cudaStream_t s) {
  constexpr int kThreads = 256;
  static int resident = 0;  // CTAs per SM, computed once per instantiation
  static int sms = 0;
  if (resident == 0) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, codec_kernel<R, DT>, kThreads, 0);
    if (e != cudaSuccess) return e;
    if (resident < 1) resident = 1;
  }
  const int64_t warps_needed = tab.total_units;
  int64_t grid = (int64_t)resident * sms;
  const int64_t by_work = (warps_needed + kThreads / 32 - 1) / (kThreads / 32);
  if (by_work < grid) grid = by_work;
  if (max_ctas > 0 && grid > max_ctas) grid = max_ctas;
  if (grid < 1) grid = 1;
  codec_kernel<R, DT><<<(unsigned)grid, kThreads, 0, s>>>(tab, cp, sse);
  return cudaGetLastError();
}

}  // namespace tdct
