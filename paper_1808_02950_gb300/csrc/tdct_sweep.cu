// tdct_sweep.cu -- the zonal sweep of §6.1 from one read of each plane.
//
// §6.1 codes every image with r = 1, 2, ..., 64 retained coefficients and
// reports the error for each r.  The reconstruction from the first r + 1
// zig-zag coefficients differs from the one from the first r by one basis
// image, so the sweep reads each block once, forms its transform once, and
// adds the basis images one r at a time, rounding, clamping and summing the
// squared error after each:
//
//   T1 (integer, exact):  A_r[k][l] = L^2 + sum_{s < r} 2 q_i q_j Z_ij t_i[k] t_j[l]
//                         ((i, j) the zig-zag position s; q = L / n, L = 360):
//                         the doubled and biased inverse 2N + L^2 of the
//                         fused codec, so the reconstruction of every r is
//                         bit for bit the codec's (the multiply-high division
//                         and the clamp are the same);
//   exact DCT (FP32):     x_r[k][l] = 1/2 + sum_{s < r} Y_ij C_i[k] C_j[l],
//                         floored and clamped (round half away from zero for
//                         the u8 range).
//
// Work split: a unit is 32 consecutive blocks of one block-row (8 rows x 256
// samples) of one plane.  A warp stages its unit in shared memory, forms the
// coefficients of the 32 blocks (T1: the packed two-block butterfly of the
// fused codec on lanes 0-15; DCT: one block per lane) and stores them by
// zig-zag position; then the half-warps sweep two blocks at a time.  Lane
// (k, l), k, l in 0..3, of a half-warp owns the samples (k, l), (k, 7-l),
// (7-k, l) and (7-k, 7-l): even rows of T1 and of the DCT are symmetric and
// odd rows antisymmetric, so one product per r serves all four, with the
// signs (-1)^j, (-1)^i and (-1)^(i+j).  The four rounded samples are packed
// into one word, and the SSE of the four takes one byte absolute difference
// and one byte dot product.  The 64 per-r partial sums stay in registers
// (32-bit) and are flushed with a reduce-scatter across the warp and 64
// atomics when the warp leaves a plane, or every 256 units (before a partial
// sum could reach 2^32).
#include <cstring>
#include <utility>

#include "tdct_dct.cuh"
#include "tdct_sweep.h"

namespace tdct {
namespace {

constexpr int kSwThreads = 128;
constexpr int kSwWarps = kSwThreads / 32;
constexpr int kSwRowBytes = 8 * kSweepUnitBlocks;  // 256 samples per unit row
constexpr int kSwFlushUnits = 256;  // 256 x 32 blocks x 4 samples x 255^2 < 2^32

// (i, j) of zig-zag position s.
__host__ __device__ constexpr int zz_i(int s) {
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j)
      if (zz_index(i, j) == s) return i;
  return 0;
}
__host__ __device__ constexpr int zz_j(int s) {
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j)
      if (zz_index(i, j) == s) return j;
  return 0;
}

// Row i of T1 (§4.1) at column k, for k = 0..3 given at run time (k is a
// lane's position, the rows are compile-time constants).
template <int I>
__device__ __forceinline__ int t1_row(int k) {
  constexpr int8_t kT[8][4] = {{1, 1, 1, 1},  {2, 2, 1, 0},   {2, 1, -1, -2}, {1, 0, -2, -2},
                               {1, -1, -1, 1}, {2, -2, 0, 1}, {1, -2, 2, -1}, {0, -1, 2, -2}};
  return k == 0 ? kT[I][0] : k == 1 ? kT[I][1] : k == 2 ? kT[I][2] : kT[I][3];
}

struct SweepParams {
  float C[64];  // orthonormal DCT-II, row-major (exact-DCT sweep)
};

// The per-lane state of one block sweep.
struct SweepLane {
  uint32_t x4;    // the four samples, bytes (k,l), (k,7-l), (7-k,l), (7-k,7-l)
  uint32_t keep;  // bytes 0xff where the sample lies inside the plane
};

// Byte B of w, sign-extended: PTX prmt with the sign-replicate bit set in
// the selectors of the upper three bytes (the __byte_perm intrinsic keeps only
// the low three bits of each selector, so it cannot do this).
template <int B>
__device__ __forceinline__ int32_t byte_sext(uint32_t w) {
  constexpr uint32_t sel = B | ((B | 8) << 4) | ((B | 8) << 8) | ((B | 8) << 12);
  uint32_t d;
  asm("prmt.b32 %0, %1, 0, %2;" : "=r"(d) : "r"(w), "n"(sel));
  return (int32_t)d;
}

// One r of the T1 sweep.  cpk: the lane's products t_i[k] t_j[l] as int8,
// byte s % 4 of word s / 4.
template <int S, bool MASK>
__device__ __forceinline__ void t1_step(const uint32_t* __restrict__ wtab, int b,
                                        const uint32_t (&cpk)[16], int32_t (&N)[4],
                                        const SweepLane& sl, uint32_t (&acc)[64]) {
  constexpr int i = zz_i(S), j = zz_j(S);
  const int32_t c = byte_sext<S & 3>(cpk[S >> 2]);
  const int32_t p = (int32_t)wtab[S * kSweepUnitBlocks + b] * c;
  N[0] += p;
  N[1] += (j & 1) ? -p : p;
  N[2] += (i & 1) ? -p : p;
  N[3] += ((i ^ j) & 1) ? -p : p;
  const uint32_t h0 = (uint32_t)__mulhi(N[0], kDivMagic), h1 = (uint32_t)__mulhi(N[1], kDivMagic);
  const uint32_t h2 = (uint32_t)__mulhi(N[2], kDivMagic), h3 = (uint32_t)__mulhi(N[3], kDivMagic);
  const uint32_t c01 = min_relu_s16x2(__byte_perm(h0, h1, 0x7632u), 0x00ff00ffu);
  const uint32_t c23 = min_relu_s16x2(__byte_perm(h2, h3, 0x7632u), 0x00ff00ffu);
  uint32_t y = __byte_perm(c01, c23, 0x6420u);
  if constexpr (MASK) y = (y & sl.keep) | (sl.x4 & ~sl.keep);
  const uint32_t d = __vabsdiffu4(sl.x4, y);
  acc[S] = __dp4a(d, d, acc[S]);
}

// One r of the exact-DCT sweep (FP32).  ci, cj: C_i[k] and C_j[l] of the lane.
template <int S, bool MASK>
__device__ __forceinline__ void dct_step(const uint32_t* __restrict__ wtab, int b,
                                         const float (&ck)[8], const float (&cl)[8],
                                         float (&N)[4], const SweepLane& sl, uint32_t (&acc)[64]) {
  constexpr int i = zz_i(S), j = zz_j(S);
  const float p = __int_as_float((int)wtab[S * kSweepUnitBlocks + b]) * ck[i] * cl[j];
  N[0] += p;
  N[1] += (j & 1) ? -p : p;
  N[2] += (i & 1) ? -p : p;
  N[3] += ((i ^ j) & 1) ? -p : p;
  // floor(N) by the bit pattern of N + 1.5 * 2^23 rounded toward -inf (unit
  // spacing there); its low 16 bits are floor(N) as int16 (|N| < 2^15)
  const uint32_t f0 = (uint32_t)__float_as_int(__fadd_rd(N[0], 12582912.0f));
  const uint32_t f1 = (uint32_t)__float_as_int(__fadd_rd(N[1], 12582912.0f));
  const uint32_t f2 = (uint32_t)__float_as_int(__fadd_rd(N[2], 12582912.0f));
  const uint32_t f3 = (uint32_t)__float_as_int(__fadd_rd(N[3], 12582912.0f));
  const uint32_t c01 = min_relu_s16x2(__byte_perm(f0, f1, 0x5410u), 0x00ff00ffu);
  const uint32_t c23 = min_relu_s16x2(__byte_perm(f2, f3, 0x5410u), 0x00ff00ffu);
  uint32_t y = __byte_perm(c01, c23, 0x6420u);
  if constexpr (MASK) y = (y & sl.keep) | (sl.x4 & ~sl.keep);
  const uint32_t d = __vabsdiffu4(sl.x4, y);
  acc[S] = __dp4a(d, d, acc[S]);
}

template <bool MASK, int... S>
__device__ __forceinline__ void t1_sweep(const uint32_t* wtab, int b, const uint32_t (&cpk)[16],
                                         const SweepLane& sl, uint32_t (&acc)[64],
                                         std::integer_sequence<int, S...>) {
  int32_t N[4] = {(int32_t)kL2, (int32_t)kL2, (int32_t)kL2, (int32_t)kL2};
  (t1_step<S, MASK>(wtab, b, cpk, N, sl, acc), ...);
}

template <bool MASK, int... S>
__device__ __forceinline__ void dct_sweep(const uint32_t* wtab, int b, const float (&ck)[8],
                                          const float (&cl)[8], const SweepLane& sl,
                                          uint32_t (&acc)[64], std::integer_sequence<int, S...>) {
  float N[4] = {0.5f, 0.5f, 0.5f, 0.5f};
  (dct_step<S, MASK>(wtab, b, ck, cl, N, sl, acc), ...);
}

// Coefficients of the two blocks of lane L (< 16) by zig-zag position:
// wtab[s][2L], wtab[s][2L + 1] = 2 q_i q_j Z_ij of blocks 2L and 2L + 1.
template <int S>
__device__ __forceinline__ void t1_store_one(const uint32_t (&z)[64], uint32_t* wtab, int lane) {
  constexpr int i = zz_i(S), j = zz_j(S);
  constexpr int32_t m = 2 * q_of(i) * q_of(j);
  const uint32_t v = z[8 * i + j];
  *reinterpret_cast<uint2*>(wtab + S * kSweepUnitBlocks + 2 * lane) =
      make_uint2((uint32_t)(lane_lo(v) * m), (uint32_t)(lane_hi(v) * m));
}
template <int... S>
__device__ __forceinline__ void t1_store(const uint32_t (&z)[64], uint32_t* wtab, int lane,
                                         std::integer_sequence<int, S...>) {
  (t1_store_one<S>(z, wtab, lane), ...);
}

template <int... S>
__device__ __forceinline__ void dct_store(const float (&y)[64], uint32_t* wtab, int lane,
                                          std::integer_sequence<int, S...>) {
  ((wtab[S * kSweepUnitBlocks + lane] = (uint32_t)__float_as_int(y[8 * zz_i(S) + zz_j(S)])), ...);
}

// The lane's products t_i[k] t_j[l] (int8, in {0, +-1, +-2, +-4}) packed
// four per word in zig-zag order.
template <int S>
__device__ __forceinline__ void cpk_one(uint32_t (&cpk)[16], int k, int l) {
  const int c = t1_row<zz_i(S)>(k) * t1_row<zz_j(S)>(l);
  cpk[S >> 2] |= ((uint32_t)c & 0xffu) << (8 * (S & 3));
}
template <int... S>
__device__ __forceinline__ void make_cpk(uint32_t (&cpk)[16], int k, int l,
                                         std::integer_sequence<int, S...>) {
  (cpk_one<S>(cpk, k, l), ...);
}

// Reduce-scatter of the 64 per-lane partial sums across the warp, 32 at a
// time; after the five halving steps each lane holds the total of one
// r-index of the 32 (the steps keep the lower or upper half by the lane's
// bits), which it adds to out[] with one atomic.
__device__ __forceinline__ void flush_sweep(uint32_t (&acc)[64], unsigned long long* out,
                                            int lane) {
#pragma unroll
  for (int part = 0; part < 2; ++part) {
    unsigned long long v[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      v[t] = acc[32 * part + t];
      acc[32 * part + t] = 0u;
    }
    int base = 32 * part;
#pragma unroll
    for (int half = 16; half >= 1; half >>= 1) {
      const bool upper = (lane & half) != 0;
#pragma unroll
      for (int t = 0; t < half; ++t) {
        const unsigned long long send = upper ? v[t] : v[t + half];
        const unsigned long long keep = upper ? v[t + half] : v[t];
        v[t] = keep + __shfl_xor_sync(0xffffffffu, send, half);
      }
      if (upper) base += half;
    }
    if (v[0]) atomicAdd(out + base, v[0]);
  }
}

template <bool DCT>
__global__ void __launch_bounds__(kSwThreads, 3)
    sweep_u8_kernel(const PlaneTable tab, const SweepParams sp,
                    unsigned long long* __restrict__ sse) {
  __shared__ __align__(16) uint8_t tiles[kSwWarps][8 * kSwRowBytes];
  __shared__ __align__(16) uint32_t wtabs[kSwWarps][64 * kSweepUnitBlocks];
  // the per-r partial sums wait here while the coefficients are formed (the
  // transform needs the registers)
  __shared__ uint32_t parked[kSwWarps][64][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint8_t* tile = tiles[wid];
  uint32_t* wtab = wtabs[wid];
  const int h = lane >> 4, q = lane & 15, k = q >> 2, l = q & 3;

  // per-lane products of the basis images at (k, l)
  uint32_t cpk[16];
  float ck[8], cl[8];
  if constexpr (DCT) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      ck[i] = sp.C[8 * i + k];
      cl[i] = sp.C[8 * i + l];
    }
  } else {
#pragma unroll
    for (int w = 0; w < 16; ++w) cpk[w] = 0u;
    make_cpk(cpk, k, l, std::make_integer_sequence<int, 64>{});
  }

  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t U = tab.total_units;
  const int64_t u_begin = (U * warp) / nwarps;
  const int n_units = (int)((U * (warp + 1)) / nwarps - u_begin);

  uint32_t acc[64];
#pragma unroll
  for (int s = 0; s < 64; ++s) acc[s] = 0u;
  int p = -1, p_end = -1, by = 0, chunk = 0, since_flush = 0;
  PlaneDesc P;
  for (int it = 0; it < n_units; ++it) {
    if (it >= p_end) {
      if (p >= 0) flush_sweep(acc, sse + 64 * (int64_t)P.slot, lane);
      since_flush = 0;
      const int64_t u = u_begin + it;
      p = find_plane(tab, u);
      P = tab.d ? tab.d[p] : tab.one;
      const int64_t e = ((p + 1 < tab.n) ? tab.d[p + 1].unit_begin : U) - u_begin;
      p_end = (int)(e < n_units ? e : n_units);
      const int64_t local = u - P.unit_begin;
      by = (int)(local / P.chunks);
      chunk = (int)(local - (int64_t)by * P.chunks);
    }
    const int bx0 = chunk * kSweepUnitBlocks;
    const int nb = min(kSweepUnitBlocks, P.nbx - bx0);
    const int x0 = bx0 * 8, rows = min(8, P.H - by * 8), cols = min(kSwRowBytes, P.W - x0);

    // stage the unit: 8 rows x 256 bytes, zero outside the plane
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int e = lane + 32 * m, row = e >> 4, c16 = (e & 15) * 16;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (row < rows) {
        const uint8_t* src = P.img + (int64_t)(by * 8 + row) * P.pitch + x0 + c16;
        if (c16 + 16 <= cols && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
          v = __ldg(reinterpret_cast<const uint4*>(src));
        } else {
          uint8_t bytes[16];
#pragma unroll
          for (int t = 0; t < 16; ++t) bytes[t] = (c16 + t < cols) ? __ldg(src + t) : (uint8_t)0;
          v = *reinterpret_cast<const uint4*>(bytes);
        }
      }
      *reinterpret_cast<uint4*>(tile + row * kSwRowBytes + c16) = v;
    }
    __syncwarp();

    // coefficients of the unit's blocks, by zig-zag position
    volatile uint32_t* park = &parked[wid][0][lane];  // volatile: really leave the registers
#pragma unroll
    for (int t = 0; t < 64; ++t) park[32 * t] = acc[t];
    if constexpr (DCT) {
      if (lane < nb) {
        float x[64];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const uint2 w = *reinterpret_cast<const uint2*>(tile + r * kSwRowBytes + 8 * lane);
          uint32_t xi[8];
          unpack_u8x8(w, xi);
#pragma unroll
          for (int c = 0; c < 8; ++c) x[8 * r + c] = (float)xi[c];
        }
        float t[64], y[64];
#pragma unroll
        for (int r = 0; r < 8; ++r) dct8_fwd(x + 8 * r, t + 8 * r, sp.C, [](int) { return true; });
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          float col[8], o[8];
#pragma unroll
          for (int r = 0; r < 8; ++r) col[r] = t[8 * r + c];
          dct8_fwd(col, o, sp.C, [](int) { return true; });
#pragma unroll
          for (int r = 0; r < 8; ++r) y[8 * r + c] = o[r];
        }
        dct_store(y, wtab, lane, std::make_integer_sequence<int, 64>{});
      }
    } else {
      if (lane < 16 && 2 * lane < nb) {
        uint32_t pk[64], z[64];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const uint4 w = *reinterpret_cast<const uint4*>(tile + r * kSwRowBytes + 16 * lane);
          pair_row(make_uint2(w.x, w.y), make_uint2(w.z, w.w), pk + 8 * r);
        }
        fwd2d<uint32_t>(pk, z);
        t1_store(z, wtab, lane, std::make_integer_sequence<int, 64>{});
      }
    }
#pragma unroll
    for (int t = 0; t < 64; ++t) acc[t] = park[32 * t];
    __syncwarp();

    // the sweep, two blocks at a time (one per half-warp)
    for (int bp = 0; bp < kSweepUnitBlocks / 2; ++bp) {
      const int b = 2 * bp + h;
      if (b >= nb) continue;
      const uint8_t* blk = tile + 8 * b;
      SweepLane sl;
      sl.x4 = (uint32_t)blk[k * kSwRowBytes + l] | ((uint32_t)blk[k * kSwRowBytes + 7 - l] << 8) |
              ((uint32_t)blk[(7 - k) * kSwRowBytes + l] << 16) |
              ((uint32_t)blk[(7 - k) * kSwRowBytes + 7 - l] << 24);
      const int vr = rows, vc = cols - 8 * b;  // valid rows / columns of this block
      if (vr >= 8 && vc >= 8) {
        sl.keep = 0xffffffffu;
        if constexpr (DCT)
          dct_sweep<false>(wtab, b, ck, cl, sl, acc, std::make_integer_sequence<int, 64>{});
        else
          t1_sweep<false>(wtab, b, cpk, sl, acc, std::make_integer_sequence<int, 64>{});
      } else {
        sl.keep = ((k < vr && l < vc) ? 0xffu : 0u) | ((k < vr && 7 - l < vc) ? 0xff00u : 0u) |
                  ((7 - k < vr && l < vc) ? 0xff0000u : 0u) |
                  ((7 - k < vr && 7 - l < vc) ? 0xff000000u : 0u);
        if constexpr (DCT)
          dct_sweep<true>(wtab, b, ck, cl, sl, acc, std::make_integer_sequence<int, 64>{});
        else
          t1_sweep<true>(wtab, b, cpk, sl, acc, std::make_integer_sequence<int, 64>{});
      }
    }

    if (++chunk == P.chunks) {
      chunk = 0;
      ++by;
    }
    if (++since_flush == kSwFlushUnits) {
      flush_sweep(acc, sse + 64 * (int64_t)P.slot, lane);
      since_flush = 0;
    }
  }
  if (p >= 0) flush_sweep(acc, sse + 64 * (int64_t)P.slot, lane);
}

}  // namespace

cudaError_t launch_sweep(const PlaneTable& tab, bool dct, const float C[64],
                         unsigned long long* d_sse, cudaStream_t s) {
  SweepParams sp;
  std::memcpy(sp.C, C, sizeof sp.C);
  static int resident[2] = {0, 0};
  static int sms = 0;
  int& res = resident[dct ? 1 : 0];
  if (res == 0) {
    sms = device_sms();
    const cudaError_t e = dct ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                    &res, sweep_u8_kernel<true>, kSwThreads, 0)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                    &res, sweep_u8_kernel<false>, kSwThreads, 0);
    if (e != cudaSuccess) return e;
    if (res < 1) res = 1;
  }
  int64_t grid = (int64_t)res * sms;
  const int64_t by_work = (tab.total_units + kSwWarps - 1) / kSwWarps;
  if (by_work < grid) grid = by_work;
  if (grid < 1) grid = 1;
  if (dct)
    sweep_u8_kernel<true><<<(unsigned)grid, kSwThreads, 0, s>>>(tab, sp, d_sse);
  else
    sweep_u8_kernel<false><<<(unsigned)grid, kSwThreads, 0, s>>>(tab, sp, d_sse);
  return cudaGetLastError();
}

}  // namespace tdct
