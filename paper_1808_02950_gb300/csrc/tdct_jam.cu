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
// inverse N = T^T (M o Z o q q^T) T with q = L / n, L = lcm(n); the factor
// 2 q_i and the bias L^2 make the last stage yield 2N + L^2, and
// x' = floor((2N + L^2) / (2 L^2)) once the value is inside the clamp window
// (a 32-bit multiply-high with a host-checked constant).  u8 samples enter
// centred (x - 128; the reconstruction is shifted back by the rounding
// bias): the kept-coefficient reconstruction is an orthogonal projection,
// so |x'_exact - 128| <= ||X - 128||_F <= 128 B and |2N| <= 256 B L^2.  For
// 16x16 u8 blocks that is below 2.13e9 < 2^31 and the second inverse stage
// runs in 32-bit integers (wrapping intermediates, exact result); for 32x32
// blocks and int16 residuals it runs in 64-bit integers.
//
// Work: a lane owns one row of a block (two 16x16 blocks or one 32x32 block
// per warp); rows are transformed in registers, columns after a transpose
// through a padded shared-memory tile, and back.  Kernels are compiled per
// kept-extent class KE (every kept position (i, j) has i, j < KE): the row
// forward forms KE outputs, only the KE leading columns are transformed, and
// the row inverse has KE inputs; the exact r is applied at run time.
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
__host__ __device__ __forceinline__ int zz_b(int B, int i, int j) {
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
// The row inverse (second stage) in 32 bits: 16x16 u8 blocks (see above).
template <int B, int DT>
constexpr bool kStageB32 = (B == 16 && DT == 0);

template <int B, int DT, int KE>
__global__ void __launch_bounds__(128) jam_codec_kernel(const PlaneDesc P, const JamParams jp,
                                                        unsigned long long* __restrict__ sse_out) {
  constexpr int BPW = 32 / B;  // blocks per warp
  constexpr int SB = DT == 0 ? 1 : 2;
  using VA = StageA<B, DT>;
  using VB = std::conditional_t<kStageB32<B, DT>, uint32_t, long long>;
  using TileT = std::conditional_t<std::is_same_v<VA, uint32_t>, int32_t, long long>;
  __shared__ TileT tile[4][BPW][B][B + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int bsub = lane / B, k = lane % B;
  const int64_t nbx = (P.W + B - 1) / B, nby = (P.H + B - 1) / B, nb = nbx * nby;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  TileT (*tl)[B + 1] = tile[wid][bsub];
  // the column stage: two lanes per column when the kept extent allows (16x16
  // blocks; at 32x32 the extra registers cost a resident CTA and the split
  // measured 2 % slower)
  constexpr bool kSplit = B == 16 && 2 * KE <= B;
  constexpr uint32_t kBlockMask = (2 * KE >= 32) ? 0xffffffffu : ((1u << (2 * KE)) - 1u);
  constexpr uint32_t kSplitMask = B == 16 ? (kBlockMask | (kBlockMask << 16)) : kBlockMask;
  // kept rows of the lane's column in the column stage
  const int hk = kept_height(B, jp.r, kSplit ? (k >> 1) : k);
  // rounding bias folded into the DC input of the row inverse (T's first row
  // is all ones, so it reaches every output): L^2, plus the centring shift
  // 128 * 2 L^2 where the stage is 64-bit
  const VB bias = DT == 0 ? (VB)(kStageB32<B, DT> ? jp.L2 : jp.L2 + jp.hiw) : (VB)0;
  unsigned long long acc = 0;
  // Block geometry of the lane at warp position b (one division; 32-bit when
  // the plane's block count allows).
  struct Geo {
    bool valid, full;
    int by, bx;
  };
  const bool small = nb < ((int64_t)1 << 31);
  auto geo_of = [&](int64_t b) {
    Geo g;
    const int64_t blk = b + bsub;
    g.valid = blk < nb;
    if (small) {
      const int q = (int)blk / (int)nbx;
      g.by = g.valid ? q : 0;
      g.bx = g.valid ? (int)blk - q * (int)nbx : 0;
    } else {
      g.by = g.valid ? (int)(blk / nbx) : 0;
      g.bx = g.valid ? (int)(blk - (int64_t)g.by * nbx) : 0;
    }
    g.full = g.valid && (g.by + 1) * B <= P.H && (g.bx + 1) * B <= P.W;
    return g;
  };
  // The lane's row k of the block at g (zero outside the plane).
  auto fetch_row = [&](const Geo& g, RowRaw<B, DT>& rr) {
    const int fy = g.by * B + k;
    if (g.full && (jp.aligned & 1)) {
      const uint4* src =
          reinterpret_cast<const uint4*>(P.img + (int64_t)fy * P.pitch + (int64_t)g.bx * B * SB);
#pragma unroll
      for (int q = 0; q < RowRaw<B, DT>::kWords; ++q) rr.w[q] = __ldg(src + q);
    } else {
      uint32_t* u = reinterpret_cast<uint32_t*>(rr.w);
#pragma unroll
      for (int q = 0; q < 4 * RowRaw<B, DT>::kWords; ++q) u[q] = 0u;
      if (g.valid) {
#pragma unroll
        for (int l = 0; l < B; ++l) {
          const uint32_t v = (uint32_t)load_px<DT>(P, fy, g.bx * B + l);
          if (DT == 0) u[l >> 2] |= (v & 0xffu) << (8 * (l & 3));
          else u[l >> 1] |= (v & 0xffffu) << (16 * (l & 1));
        }
      }
    }
  };
  // rows are fetched one iteration ahead: the loads of the next blocks are
  // in flight while the current ones are transformed (measured 8 % faster at
  // B = 16, 5 % at B = 32)
  RowRaw<B, DT> raw_next;
  Geo g_next{};
  if (warp * BPW < nb) {
    g_next = geo_of(warp * BPW);
    fetch_row(g_next, raw_next);
  }
  for (int64_t base = warp * BPW; base < nb; base += nwarps * BPW) {
    const Geo g = g_next;
    const RowRaw<B, DT> raw = raw_next;  // the raw row stays for the error
    if (base + nwarps * BPW < nb) {
      g_next = geo_of(base + nwarps * BPW);
      fetch_row(g_next, raw_next);
    }
    const bool valid = g.valid, full = g.full;
    const int by = g.by, bx = g.bx;
    const int y = by * B + k;
    // rows: t = T x for row k of the block (KE leading outputs)
    {
      uint32_t x[B], t[B];
#pragma unroll
      for (int l = 0; l < B; ++l) x[l] = (uint32_t)(raw.at(l) - (DT == 0 ? 128 : 0));
      jam_fwd<B, uint32_t>(x, t);
#pragma unroll
      for (int j = 0; j < KE; ++j) tl[k][j] = (TileT)(int32_t)t[j];
    }
    __syncwarp();
    // columns c < KE: Z[i][c] (i < KE), zonal mask with 2 q_i, inverse along
    // the column.  With 2 KE <= B = 16 two lanes share a column: lane half h takes
    // the sums (h = 0: even rows of Z) or the differences (h = 1: odd rows)
    // of the first JAM stage, the half-size forward and inverse, and the
    // pair combines u +- w by one exchange; otherwise one lane per column.
    // Lanes write only the column they read.
    if constexpr (kSplit) {
      if (k < 2 * KE) {
        const int c = k >> 1;
        const uint32_t hm = (k & 1) ? 0xffffffffu : 0u;  // all ones for h = 1
        uint32_t col[B], v[B / 2], zh[B / 2];
#pragma unroll
        for (int i = 0; i < B; ++i) col[i] = (uint32_t)tl[i][c];
#pragma unroll
        for (int m = 0; m < B / 2; ++m) v[m] = col[m] + (col[B - 1 - m] ^ hm) - hm;
        jam_fwd<B / 2, uint32_t>(v, zh);  // zh[i] = Z[2 i + h][c]
        VA w[B / 2], rh[B / 2];
#pragma unroll
        for (int i = 0; i < B / 2; ++i) {
          const int ifull = 2 * i + (int)(hm & 1u);
          const int32_t qm = hm ? jp.q[2 * i + 1] : jp.q[2 * i];
          w[i] = (2 * i < KE && ifull < KE && ifull < hk)
                     ? (VA)((long long)(int32_t)zh[i] * (2 * qm)) : (VA)0;
        }
        jam_inv<B / 2, VA>(w, rh);  // h = 0: u, h = 1: w
        const int rx = hm ? B - 1 : 0;
#pragma unroll
        for (int m = 0; m < B / 2; ++m) {
          const VA pm = __shfl_xor_sync(kSplitMask, rh[m], 1);
          // h = 0: row m = u + w; h = 1: row B - 1 - m = u - w
          const VA val = hm ? pm - rh[m] : rh[m] + pm;
          tl[m ^ rx][c] = (TileT)val;
        }
      }
    } else if (k < KE) {
      uint32_t col[B], z[B];
#pragma unroll
      for (int i = 0; i < B; ++i) col[i] = (uint32_t)tl[i][k];
      jam_fwd<B, uint32_t>(col, z);
      VA w[B], u[B];
#pragma unroll
      for (int i = 0; i < B; ++i)
        w[i] = (i < KE && i < hk) ? (VA)((long long)(int32_t)z[i] * (2 * jp.q[i])) : (VA)0;
      jam_inv<B, VA>(w, u);
#pragma unroll
      for (int i = 0; i < B; ++i) tl[i][k] = (TileT)u[i];
    }
    __syncwarp();
    // row k: 2N[k][l] + bias = sum_j q_j V'[k][j] T[j][l] (j < KE); round,
    // clamp, error, store
    {
      VB v[B], n2[B];
#pragma unroll
      for (int j = 0; j < B; ++j)
        v[j] = j < KE ? (VB)tl[k][j] * (VB)jp.q[j] : (VB)0;
      v[0] += bias;
      jam_inv<B, VB>(v, n2);
      RowRaw<B, DT> out;
      uint32_t* ou = reinterpret_cast<uint32_t*>(out.w);
#pragma unroll
      for (int q = 0; q < 4 * RowRaw<B, DT>::kWords; ++q) ou[q] = 0u;
      uint32_t sse = 0;
      const bool row_in = valid && y < P.H;
      if constexpr (kStageB32<B, DT>) {
        // n2 = 2N + L^2 exactly; capped at 128 * 2 L^2 and shifted by it (no
        // wrap), the signed high product with magic16 carries
        // floor(a / (2 L^2)) = x' in its upper 16 bits (negative below the
        // window); pairs are clamped to [0, 255] as s16x2 and packed to bytes
        uint32_t h[B];
#pragma unroll
        for (int l = 0; l < B; ++l) {
          const int32_t a = min((int32_t)n2[l], jp.hiw) + jp.hiw;
          h[l] = (uint32_t)__mulhi(a, jp.magic16);
        }
#pragma unroll
        for (int q = 0; q < B / 4; ++q) {
          const uint32_t c01 = min_relu_s16x2(__byte_perm(h[4 * q], h[4 * q + 1], 0x7632u), 0x00ff00ffu);
          const uint32_t c23 =
              min_relu_s16x2(__byte_perm(h[4 * q + 2], h[4 * q + 3], 0x7632u), 0x00ff00ffu);
          ou[q] = __byte_perm(c01, c23, 0x6420u);
        }
        const uint32_t* ru = reinterpret_cast<const uint32_t*>(raw.w);
        if (full) {
#pragma unroll
          for (int q = 0; q < B / 4; ++q) {
            const uint32_t dq = __vabsdiffu4(ru[q], ou[q]);
            sse = __dp4a(dq, dq, sse);
          }
        } else {
#pragma unroll
          for (int l = 0; l < B; ++l) {
            const bool in = row_in && bx * B + l < P.W;
            const int32_t d = raw.at(l) - out.at(l);
            sse += in ? (uint32_t)(d * d) : 0u;
          }
        }
      } else if constexpr (DT == 0) {
        // 64-bit stage: n2 = 2N + L^2 + 128 * 2 L^2; clamped to [0, limit]
        // before the 32-bit division (limit itself gives 256 -> 255)
        uint32_t qv[B];
#pragma unroll
        for (int l = 0; l < B; ++l) {
          const long long a = (long long)n2[l];
          const uint32_t ac = a < 0 ? 0u : (a > jp.limit ? (uint32_t)jp.limit : (uint32_t)a);
          qv[l] = min(__umulhi(ac, jp.magic) >> jp.shift, 255u);
        }
#pragma unroll
        for (int q = 0; q < B / 4; ++q)
          ou[q] = __byte_perm(__byte_perm(qv[4 * q], qv[4 * q + 1], 0x0040u),
                              __byte_perm(qv[4 * q + 2], qv[4 * q + 3], 0x0040u), 0x5410u);
        const uint32_t* ru = reinterpret_cast<const uint32_t*>(raw.w);
        if (full) {
#pragma unroll
          for (int q = 0; q < B / 4; ++q) {
            const uint32_t dq = __vabsdiffu4(ru[q], ou[q]);
            sse = __dp4a(dq, dq, sse);
          }
        } else {
#pragma unroll
          for (int l = 0; l < B; ++l) {
            const bool in = row_in && bx * B + l < P.W;
            const int32_t d = raw.at(l) - out.at(l);
            sse += in ? (uint32_t)(d * d) : 0u;
          }
        }
      } else {
        // int16 residuals: |x'| rounded half away from zero, clamped to 255
#pragma unroll
        for (int l = 0; l < B; ++l) {
          const long long nn = (long long)n2[l];
          const long long a = (nn < 0 ? -nn : nn) + jp.L2;
          int32_t m = a >= jp.limit ? 255 : (int32_t)(__umulhi((uint32_t)a, jp.magic) >> jp.shift);
          m = min(m, 255);
          const int32_t xr = nn < 0 ? -m : m;
          ou[l >> 1] |= ((uint32_t)xr & 0xffffu) << (16 * (l & 1));
          const bool in = full || (row_in && bx * B + l < P.W);
          const int32_t d = raw.at(l) - xr;
          sse += in ? (uint32_t)(d * d) : 0u;
        }
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

// Kept-extent classes: the smallest class at least the extent of the first
// r zig-zag positions of a B x B block.
__host__ __device__ constexpr int jam_extent_class(int ext) {
  return ext <= 2 ? 2 : ext <= 4 ? 4 : ext <= 6 ? 6 : ext <= 8 ? 8 : ext <= 12 ? 12
       : ext <= 16 ? 16 : ext <= 24 ? 24 : 32;
}

template <int B, int DT, int KE>
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
  jam_codec_kernel<B, DT, KE><<<(unsigned)grid, 128, 0, s>>>(P, jp, sse);
  return cudaGetLastError();
}

template <int B, int DT>
cudaError_t launch_ke(int ke, const PlaneDesc& P, const JamParams& jp, unsigned long long* sse,
                      cudaStream_t s) {
  switch (ke) {
    case 2: return launch_b<B, DT, 2>(P, jp, sse, s);
    case 4: return launch_b<B, DT, 4>(P, jp, sse, s);
    case 6: return launch_b<B, DT, 6>(P, jp, sse, s);
    case 8: return launch_b<B, DT, 8>(P, jp, sse, s);
    case 12: return launch_b<B, DT, 12>(P, jp, sse, s);
    case 16: return launch_b<B, DT, 16>(P, jp, sse, s);
    default:
      if constexpr (B == 32) {
        if (ke == 24) return launch_b<B, DT, 24>(P, jp, sse, s);
        if (ke == 32) return launch_b<B, DT, 32>(P, jp, sse, s);
      }
      return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_jam_codec(int B, const PlaneDesc& P, const JamParams& jp,
                             unsigned long long* sse, cudaStream_t s) {
  // extent of the first r scan positions: 1 + the largest row or column index
  int ext = 0;
  for (int i = 0; i < B; ++i)
    for (int j = 0; j < B; ++j)
      if (zz_b(B, i, j) < jp.r) ext = max(ext, max(i, j) + 1);
  const int ke = min(jam_extent_class(ext), B);
  if (B == 16)
    return P.dtype == 0 ? launch_ke<16, 0>(ke, P, jp, sse, s) : launch_ke<16, 1>(ke, P, jp, sse, s);
  if (B == 32)
    return P.dtype == 0 ? launch_ke<32, 0>(ke, P, jp, sse, s) : launch_ke<32, 1>(ke, P, jp, sse, s);
  return cudaErrorInvalidValue;
}

}  // namespace tdct
