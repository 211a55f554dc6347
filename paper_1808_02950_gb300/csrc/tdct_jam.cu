// tdct_jam.cu -- the codec of §6.1 with 16x16 and 32x32 blocks and the
// 16- and 32-point transforms that §6.2 derives from T1 with the JAM
// recursion: T_(N) = M_per [T_(N/2) 0; 0 T_(N/2)] M_add (the 1/sqrt(2) merged
// into the scaling), down to T1 and its fast algorithm (§5.1).
//
// The recursion is also the fast algorithm: M_add is N/2 sums and N/2
// differences (x_m +- x_(N-1-m)), the two half-size transforms follow, and
// M_per interleaves their outputs (even rows from the sums, odd rows from the
// differences): 64 additions and 12 doublings for N = 16, 160 and 24 for
// N = 32 (Table 9).  The inverse is the transpose: de-interleave, two
// half-size inverses, then x_m = u_m + w_m, x_(N-1-m) = u_m - w_m.
//
// Exactness: Z = T X T^T is formed in 32-bit integers (|Z| < 2^20); the
// inverse N = T^T (M o Z o q q^T) T in 64-bit integers (|N| < 2^43 at
// N = 32), with q = L / n, L = lcm(n); the factor 2 q_i and the bias L^2 make
// the last stage yield 2N + L^2, and x' = floor((2N + L^2) / (2 L^2)) once
// the value is inside the clamp window (a 32-bit multiply-high with a
// host-checked constant).
//
// Work: a lane owns one row of a block (two 16x16 blocks or one 32x32 block
// per warp); rows are transformed in registers, columns after a transpose
// through a padded shared-memory tile, and back.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "tdct_jam.h"
#include "tdct_kernels.cuh"

namespace tdct {

namespace {

template <int B, typename V>
__device__ __forceinline__ void jam_fwd(const V* x, V* y) {
  if constexpr (B == 8) {
    fwd8<V>(x, y);
  } else {
    constexpr int H = B / 2;
    V s[H], d[H], a[H], b[H];
#pragma unroll
    for (int m = 0; m < H; ++m) {
      s[m] = x[m] + x[B - 1 - m];
      d[m] = x[m] - x[B - 1 - m];
    }
    jam_fwd<H, V>(s, a);
    jam_fwd<H, V>(d, b);
#pragma unroll
    for (int i = 0; i < H; ++i) {
      y[2 * i] = a[i];
      y[2 * i + 1] = b[i];
    }
  }
}

template <int B, typename V>
__device__ __forceinline__ void jam_inv(const V* y, V* x) {
  if constexpr (B == 8) {
    inv8<V>(y, x);
  } else {
    constexpr int H = B / 2;
    V a[H], b[H], u[H], w[H];
#pragma unroll
    for (int i = 0; i < H; ++i) {
      a[i] = y[2 * i];
      b[i] = y[2 * i + 1];
    }
    jam_inv<H, V>(a, u);
    jam_inv<H, V>(b, w);
#pragma unroll
    for (int m = 0; m < H; ++m) {
      x[m] = u[m] + w[m];
      x[B - 1 - m] = u[m] - w[m];
    }
  }
}

// Scan index of (i, j) in the B x B zig-zag (anti-diagonals; odd ones start
// at (0, s) with i increasing, even ones at (s, 0) with i decreasing).
__device__ __forceinline__ int zz_b(int B, int i, int j) {
  const int s = i + j;
  if (s < B) return s * (s + 1) / 2 + ((s & 1) ? i : s - i);
  const int before = B * B - (2 * B - 1 - s) * (2 * B - s) / 2;
  return before + ((s & 1) ? i - (s - (B - 1)) : (B - 1) - i);
}

template <int DT>
__device__ __forceinline__ int32_t load_px(const PlaneDesc& P, int y, int x) {
  if (y >= P.H || x >= P.W) return 0;
  const uint8_t* row = P.img + (int64_t)y * P.pitch;
  if constexpr (DT == 0) return row[x];
  else return reinterpret_cast<const int16_t*>(row)[x];
}

// Height of column c of the kept set: a prefix of the zig-zag scan keeps, in
// every column, the positions i < h (whole anti-diagonals, plus at most one
// position of the partial one).
__device__ __forceinline__ int kept_height(int B, int r, int c) {
  int h = 0;
  for (int i = 0; i < B; ++i)
    if (zz_b(B, i, c) < r) h = i + 1;
  return h;
}

// A row of one block as raw 16-byte words (u8: B bytes, int16: 2B bytes).
template <int B, int DT>
struct RowRaw {
  static constexpr int kWords = B * (DT == 0 ? 1 : 2) / 16;
  uint4 w[kWords];
  __device__ __forceinline__ int32_t at(int l) const {
    const uint32_t* u = reinterpret_cast<const uint32_t*>(w);
    if constexpr (DT == 0) return (int32_t)((u[l >> 2] >> (8 * (l & 3))) & 0xffu);
    else return (int32_t)(int16_t)(u[l >> 1] >> (16 * (l & 1)));
  }
};

// The column inverse V' = T^T (2 q o Z) of a column is exact in 32 bits
// when |V'| < 2^31: at B = 16, |Z| <= 146880 and |V'| <= 16 * 2 * 90 * |Z|
// < 4.3e8 for both sample types; at B = 32, u8 gives |Z| <= 293760 and
// |V'| <= 32 * 2 * 90 * |Z| < 1.7e9, int16 residuals do not fit.  There the
// stage and both transposes run in 32 bits, elsewhere in 64.
template <int B, int DT>
using StageA = std::conditional_t<(B == 16 || DT == 0), uint32_t, long long>;

template <int B, int DT>
__global__ void __launch_bounds__(128) jam_codec_kernel(const PlaneDesc P, const JamParams jp,
                                                        unsigned long long* __restrict__ sse_out) {
  constexpr int BPW = 32 / B;  // blocks per warp
  constexpr int SB = DT == 0 ? 1 : 2;
  using VA = StageA<B, DT>;
  using TileT = std::conditional_t<std::is_same_v<VA, uint32_t>, int32_t, long long>;
  __shared__ TileT tile[4][BPW][B][B + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int bsub = lane / B, k = lane % B;
  const int64_t nbx = (P.W + B - 1) / B, nby = (P.H + B - 1) / B, nb = nbx * nby;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  TileT (*tl)[B + 1] = tile[wid][bsub];
  const int hk = kept_height(B, jp.r, k);  // the lane's column in the column stage
  unsigned long long acc = 0;
  for (int64_t base = warp * BPW; base < nb; base += nwarps * BPW) {
    const int64_t blk = base + bsub;
    const bool valid = blk < nb;
    const int by = valid ? (int)(blk / nbx) : 0, bx = valid ? (int)(blk - (int64_t)by * nbx) : 0;
    const int y = by * B + k;
    const bool full = valid && (by + 1) * B <= P.H && (bx + 1) * B <= P.W;
    // rows: t = T x for row k of the block; the raw row stays for the error
    RowRaw<B, DT> raw;
    {
      if (full && (jp.aligned & 1)) {
        const uint4* src =
            reinterpret_cast<const uint4*>(P.img + (int64_t)y * P.pitch + (int64_t)bx * B * SB);
#pragma unroll
        for (int q = 0; q < RowRaw<B, DT>::kWords; ++q) raw.w[q] = __ldg(src + q);
      } else {
        uint32_t* u = reinterpret_cast<uint32_t*>(raw.w);
#pragma unroll
        for (int q = 0; q < 4 * RowRaw<B, DT>::kWords; ++q) u[q] = 0u;
        if (valid) {
#pragma unroll
          for (int l = 0; l < B; ++l) {
            const uint32_t v = (uint32_t)load_px<DT>(P, y, bx * B + l);
            if (DT == 0) u[l >> 2] |= (v & 0xffu) << (8 * (l & 3));
            else u[l >> 1] |= (v & 0xffffu) << (16 * (l & 1));
          }
        }
      }
      uint32_t x[B], t[B];
#pragma unroll
      for (int l = 0; l < B; ++l) x[l] = (uint32_t)raw.at(l);
      jam_fwd<B, uint32_t>(x, t);
#pragma unroll
      for (int j = 0; j < B; ++j) tl[k][j] = (TileT)(int32_t)t[j];
    }
    __syncwarp();
    // column c = k: Z[i][c], zonal mask with 2 q_i, inverse along the column
    {
      uint32_t col[B], z[B];
#pragma unroll
      for (int i = 0; i < B; ++i) col[i] = (uint32_t)tl[i][k];
      jam_fwd<B, uint32_t>(col, z);
      VA w[B], u[B];
#pragma unroll
      for (int i = 0; i < B; ++i)
        w[i] = i < hk ? (VA)((long long)(int32_t)z[i] * (2 * jp.q[i])) : (VA)0;
      jam_inv<B, VA>(w, u);
      __syncwarp();
#pragma unroll
      for (int i = 0; i < B; ++i) tl[i][k] = (TileT)u[i];
    }
    __syncwarp();
    // row k: 2N[k][l] = sum_j q_j V'[k][j] T[j][l]; round, clamp, error, store
    {
      long long v[B], n2[B];
#pragma unroll
      for (int j = 0; j < B; ++j) v[j] = (long long)tl[k][j] * jp.q[j];
      jam_inv<B, long long>(v, n2);
      RowRaw<B, DT> out;
      uint32_t* ou = reinterpret_cast<uint32_t*>(out.w);
#pragma unroll
      for (int q = 0; q < 4 * RowRaw<B, DT>::kWords; ++q) ou[q] = 0u;
      uint32_t sse = 0;
      const bool row_in = valid && y < P.H;
#pragma unroll
      for (int l = 0; l < B; ++l) {
        int32_t xr;
        if (DT == 0) {
          const long long a = n2[l] + jp.L2;
          xr = a < 0 ? 0 : (a >= jp.limit ? 255 : (int32_t)(__umulhi((uint32_t)a, jp.magic) >> jp.shift));
          xr = min(xr, 255);
          ou[l >> 2] |= (uint32_t)xr << (8 * (l & 3));
        } else {
          const long long a = (n2[l] < 0 ? -n2[l] : n2[l]) + jp.L2;
          int32_t m = a >= jp.limit ? 255 : (int32_t)(__umulhi((uint32_t)a, jp.magic) >> jp.shift);
          m = min(m, 255);
          xr = n2[l] < 0 ? -m : m;
          ou[l >> 1] |= ((uint32_t)xr & 0xffffu) << (16 * (l & 1));
        }
        const bool in = full || (row_in && bx * B + l < P.W);
        const int32_t d = raw.at(l) - xr;
        sse += in ? (uint32_t)(d * d) : 0u;
      }
      acc += sse;
      if (P.recon && row_in) {
        uint8_t* rrow = P.recon + (int64_t)y * P.recon_pitch + (int64_t)bx * B * SB;
        if (full && (jp.aligned & 2)) {
#pragma unroll
          for (int q = 0; q < RowRaw<B, DT>::kWords; ++q) reinterpret_cast<uint4*>(rrow)[q] = out.w[q];
        } else {
#pragma unroll
          for (int l = 0; l < B; ++l) {
            if (bx * B + l < P.W) {
              if constexpr (DT == 0) rrow[l] = (uint8_t)out.at(l);
              else reinterpret_cast<int16_t*>(rrow)[l] = (int16_t)out.at(l);
            }
          }
        }
      }
    }
    __syncwarp();
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0 && acc) atomicAdd(sse_out, acc);
}

template <int B, int DT>
cudaError_t launch_b(const PlaneDesc& P, const JamParams& jp, unsigned long long* sse,
                     cudaStream_t s) {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t nb = (int64_t)((P.W + B - 1) / B) * ((P.H + B - 1) / B);
  const int64_t warps = (nb + (32 / B) - 1) / (32 / B);
  int64_t grid = (warps + 3) / 4;
  if (grid > (int64_t)sms * 8) grid = (int64_t)sms * 8;
  if (grid < 1) grid = 1;
  jam_codec_kernel<B, DT><<<(unsigned)grid, 128, 0, s>>>(P, jp, sse);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_jam_codec(int B, const PlaneDesc& P, const JamParams& jp,
                             unsigned long long* sse, cudaStream_t s) {
  if (B == 16) return P.dtype == 0 ? launch_b<16, 0>(P, jp, sse, s) : launch_b<16, 1>(P, jp, sse, s);
  if (B == 32) return P.dtype == 0 ? launch_b<32, 0>(P, jp, sse, s) : launch_b<32, 1>(P, jp, sse, s);
  return cudaErrorInvalidValue;
}

}  // namespace tdct
