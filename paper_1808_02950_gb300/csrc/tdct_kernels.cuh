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
  int32_t vec16;       // bit 0: img rows 8-byte aligned; bit 1: recon rows;
                       // bit 2: u8 plane eligible for the bulk-copy ring;
                       // bit 3: plane eligible for a staged-copy ring (u8 or int16);
                       // bit 4: bulk-copy plane whose odd rows start 8 mod 16;
                       // bit 5: bulk-copy plane with units across block rows
  int32_t slot;        // output index for SSE / PSNR
  int32_t pad_;
};

struct PlaneTable {
  const PlaneDesc* d;  // device array, or nullptr to use `one`
  int32_t n;
  int32_t any_bulk;    // some plane takes the bulk-copy path (vec16 bit 2)
  int64_t total_units;
  PlaneDesc one;
  int32_t staged;      // the planes take a staged-copy ring (vec16 bit 3)
  int32_t shifted;     // bulk-copy planes with rows 8 mod 16 (vec16 bit 4)
  int32_t wrap;        // bulk-copy planes whose units run on across block rows (vec16 bit 5)
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
// in, §6.1); cmul2 = 2 cmul (the doubled multipliers of the u8 paths).  Lives
// in the kernel parameter (constant) bank.
struct CodecParams {
  int32_t cmul[64];
  int32_t cmul2[64];
  int32_t cmul2h[64];    // cmul2 * 2^16 (< 2^31): block B's scaled coefficient in one multiply-high
  int* status;           // device status word (TDCT_ETIMEOUT on a bounded wait giving up)
  long long wait_limit;  // clock cycles a bulk-copy wait may take before giving up
  int32_t test_hook;     // 1: the first copy of warp 0 is never issued (timeout test)
  int32_t ctas_per_sm;   // > 0: cap on resident CTAs per SM (launch tuning)
  int32_t tc_variant;    // tensor engine: 0 one tile at a time, 1 software-pipelined
  int32_t pad_;
  // Per-plane closing of the u8 bulk-copy ring kernel (plans): with fin_cnt
  // set, the kernel's SSE pointer is an accumulator and fin_cnt a count of
  // finished units per plane slot, both zero at launch; the warp that
  // finishes a plane's last units moves its SSE to fin_sse, writes its PSNR
  // to fin_psnr (if set) and leaves both at zero for the next launch.
  unsigned long long* fin_sse;
  double* fin_psnr;
  unsigned int* fin_cnt;
};

// Forward, zonal mask, scale by q_i q_j, inverse, round and clamp one block.
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

// min(a, b) then max(., 0) on each signed 16-bit lane.
__device__ __forceinline__ uint32_t min_relu_s16x2(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("min.relu.s16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

// Lanes of a packed word a + 2^16 b (a, b in [-2^15, 2^15)).
__device__ __forceinline__ int32_t lane_lo(uint32_t v) { return (int32_t)(int16_t)(v & 0xffffu); }
__device__ __forceinline__ int32_t lane_hi(uint32_t v) {
  return (int32_t)(v - (uint32_t)lane_lo(v)) >> 16;
}

// ---- int16 residual path: one block at a time, epilogue streamed by rows ------
//
// Residuals reach |Z| = 36720 (> int16), so the forward is per block in int32.
// The inverse uses the doubled multipliers (2N) and is streamed row by row
// into rounding, SSE and the store, which keeps no 64-sample output array
// live.  Rounding half away from zero for both signs:
//   x' = floor((2N + L^2 - [N < 0]) / (2 L^2)),
// evaluated as q = floor((2N + L^2 - [N < 0] + 255 * 2 L^2) / (2 L^2)) = x' + 255
// by the multiply-high (exact for dividends in [0, 2.5e9); |2N| <= 2 * 255 *
// 8 * L^2 by the orthogonal-projection bound, so the dividend is below 6e8,
// and a negative dividend gives a negative q, which the clamp takes to 0).
// Two q share a word (high halves of the products, one byte permute), one
// min.relu.s16x2 clamps both to [0, 510], one vsub2 gives the two int16
// samples x' = q - 255, and one vabsdiffs2 against the raw sample word gives
// both |x - x'| for the SSE.
constexpr int32_t kI16BiasQ = (int32_t)(511u * kL2);

// Where the int16 codec reads a block's row k (8 samples in a uint4): the row
// words in registers, or a staged-copy slot in shared memory (row stride
// 1024 B), re-read for the SSE instead of being held across the inverse.
struct I16RowsInRegs {
  const uint4* w;
  __device__ __forceinline__ uint4 row(int k) const { return w[k]; }
};
struct I16RowsInSmem {
  const uint8_t* p;
  __device__ __forceinline__ uint4 row(int k) const {
    return *reinterpret_cast<const uint4*>(p + k * 1024);
  }
};

// Inverse, rounding, SSE and store of one int16 block from its kept, scaled
// coefficients w (doubled multipliers; samples re-read through rw).
template <int R, typename RS>
__device__ __forceinline__ uint32_t inverse_epilogue_i16(const uint32_t w[64], const PlaneDesc& P,
                                                         int by, int bx, RS rw, int valid_rows,
                                                         int valid_cols) {
  const bool full = valid_rows == 8 && valid_cols == 8;
  // columns first: v[k][j] = sum_i t_i[k] w[i][j]
  uint32_t v[64];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    uint32_t col[8], o[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) col[i] = w[8 * i + j];
    inv8<uint32_t>(col, o);
#pragma unroll
    for (int k = 0; k < 8; ++k) v[8 * k + j] = o[k];
  }
  const bool store = P.recon != nullptr;
  const bool fast_store = store && full && (P.vec16 & 2);
  // the valid samples of a row as 16-bit lane masks of its four words
  uint32_t colmask[4];
#pragma unroll
  for (int m = 0; m < 4; ++m)
    colmask[m] = (2 * m < valid_cols ? 0xffffu : 0u) | (2 * m + 1 < valid_cols ? 0xffff0000u : 0u);
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    uint32_t n2[8];
    inv8<uint32_t>(v + 8 * k, n2);
    uint32_t h[8];
#pragma unroll
    for (int l = 0; l < 8; ++l)
      h[l] = (uint32_t)__mulhi((int32_t)n2[l] + ((int32_t)n2[l] >> 31) + kI16BiasQ, kDivMagic);
    const uint4 xw = rw.row(k);
    const uint32_t xs[4] = {xw.x, xw.y, xw.z, xw.w};
    uint32_t o[4];
    const bool row_in = k < valid_rows;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const uint32_t q = min_relu_s16x2(__byte_perm(h[2 * m], h[2 * m + 1], 0x7632u), 0x01fe01feu);
      o[m] = __vsub2(q, 0x00ff00ffu);  // x' = q - 255 in each int16 lane
      uint32_t d = __vabsdiffs2(xs[m], o[m]);
      if (!full) d &= row_in ? colmask[m] : 0u;
      acc += (d & 0xffffu) * (d & 0xffffu) + (d >> 16) * (d >> 16);
    }
    if (store && row_in) {
      uint8_t* row = P.recon + (int64_t)(by * 8 + k) * P.recon_pitch + (int64_t)bx * 16;
      if (fast_store) {
        reinterpret_cast<uint2*>(row)[0] = make_uint2(o[0], o[1]);
        reinterpret_cast<uint2*>(row)[1] = make_uint2(o[2], o[3]);
      } else {
#pragma unroll
        for (int l = 0; l < 8; ++l)
          if (l < valid_cols)
            reinterpret_cast<int16_t*>(row)[l] = (int16_t)(o[l >> 1] >> (16 * (l & 1)));
      }
    }
  }
  return acc;
}

template <int R, typename RS>
__device__ __forceinline__ uint32_t codec_block_i16(const PlaneDesc& P, int by, int bx, RS rw,
                                                    const CodecParams& cp, int valid_rows,
                                                    int valid_cols) {
  uint32_t w[64];
  {
    uint32_t x[64], z[64];
#pragma unroll
    for (int k = 0; k < 8; ++k) unpack_i16x8(rw.row(k), x + 8 * k);
    fwd2d<uint32_t>(x, z);
#pragma unroll
    for (int p = 0; p < 64; ++p)
      w[p] = kept(R, p / 8, p % 8) ? z[p] * (uint32_t)cp.cmul2[p] : 0u;
  }
  return inverse_epilogue_i16<R>(w, P, by, bx, rw, valid_rows, valid_cols);
}

// Classes whose kept coefficients all fit 16-bit lanes for int16 residuals
// (|x| <= 255) except possibly Z_22: with the row sums of |T1| (8, 10, 12, 10,
// 8, 10, 12, 10), |Z_ij| <= 255 * 120 < 2^15 unless both i and j are 2 or 6
// (36720); up to class 36 only (2, 2) is kept among those, and it is formed
// separately in 32 bits.  Used up to class 32 (class 36 would spill).
template <int R>
__host__ __device__ constexpr bool i16_packed_forward() {
#ifdef TDCT_I16_PACKED
  return TDCT_I16_PACKED && R <= 32;
#else
  return R <= 32;
#endif
}

// The lane's two int16 blocks (A at slot, B at slot + 16; rows 1024 bytes
// apart) through one packed forward (a + 2^16 b per word), then each block's
// inverse.  Samples enter biased by 2^15 (x ^ 0x8000 per lane: unsigned 16-bit
// lanes, packed by one byte permute), which only moves Z_00, by 64 * 2^15 per
// lane (2^21 in the packed word, mod 2^32); Z_22 of classes that keep it is
// evaluated per block from the first pass's column (or row) 2.
template <int R>
__device__ __forceinline__ uint32_t codec_pair_i16(const PlaneDesc& P, int by, int bx0,
                                                   const uint8_t* slot, const CodecParams& cp,
                                                   int valid_rows, bool has1) {
  uint32_t z[64];
  int32_t z22[2] = {0, 0};
  {
    uint32_t pk[64], t[64];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint4 a = *reinterpret_cast<const uint4*>(slot + k * 1024);
      const uint4 b = *reinterpret_cast<const uint4*>(slot + 16 + k * 1024);
      const uint32_t aw[4] = {a.x ^ 0x80008000u, a.y ^ 0x80008000u, a.z ^ 0x80008000u,
                              a.w ^ 0x80008000u};
      const uint32_t bw[4] = {b.x ^ 0x80008000u, b.y ^ 0x80008000u, b.z ^ 0x80008000u,
                              b.w ^ 0x80008000u};
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        pk[8 * k + 2 * m] = __byte_perm(aw[m], bw[m], 0x5410u);
        pk[8 * k + 2 * m + 1] = __byte_perm(aw[m], bw[m], 0x7632u);
      }
    }
    constexpr bool kFix = kept(R, 2, 2);
    if constexpr (kept_cols(R) <= kept_rows(R)) {
      // rows first: t[k][j], then the kept positions of each column
#pragma unroll
      for (int k = 0; k < 8; ++k) fwd8<uint32_t>(pk + 8 * k, t + 8 * k);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint32_t col[8], o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) col[k] = t[8 * k + j];
        fwd8<uint32_t>(col, o);
#pragma unroll
        for (int i = 0; i < 8; ++i) z[8 * i + j] = o[i];
      }
      if constexpr (kFix) {
        // Z_22 = sum_k T1[2][k] t[k][2] per block (|t| <= 12 * 255: exact lanes)
        uint32_t ca[8], cb[8], oa[8], ob[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          ca[k] = (uint32_t)lane_lo(t[8 * k + 2]);
          cb[k] = (uint32_t)lane_hi(t[8 * k + 2]);
        }
        fwd8<uint32_t>(ca, oa);
        fwd8<uint32_t>(cb, ob);
        z22[0] = (int32_t)oa[2];
        z22[1] = (int32_t)ob[2];
      }
    } else {
#pragma unroll
      for (int l = 0; l < 8; ++l) {
        uint32_t col[8], o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) col[k] = pk[8 * k + l];
        fwd8<uint32_t>(col, o);
#pragma unroll
        for (int i = 0; i < 8; ++i) t[8 * i + l] = o[i];
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) fwd8<uint32_t>(t + 8 * i, z + 8 * i);
      if constexpr (kFix) {
        uint32_t ra[8], rb[8], oa[8], ob[8];
#pragma unroll
        for (int l = 0; l < 8; ++l) {
          ra[l] = (uint32_t)lane_lo(t[16 + l]);
          rb[l] = (uint32_t)lane_hi(t[16 + l]);
        }
        fwd8<uint32_t>(ra, oa);
        fwd8<uint32_t>(rb, ob);
        z22[0] = (int32_t)oa[2];
        z22[1] = (int32_t)ob[2];
      }
    }
    z[0] -= 2097152u;  // the 2^15 bias of both lanes: 64 * 2^15 (1 + 2^16) mod 2^32
  }
  uint32_t sse = 0;
#pragma unroll 1
  for (int b = 0; b < 2; ++b) {
    if (b == 1 && !has1) break;
    uint32_t w[64];
#pragma unroll
    for (int p = 0; p < 64; ++p) {
      const int i = p / 8, j = p % 8;
      if (!kept(R, i, j)) {
        w[p] = 0u;
        continue;
      }
      int32_t zz = b == 0 ? lane_lo(z[p]) : lane_hi(z[p]);
      if (i == 2 && j == 2) zz = z22[b];
      w[p] = (uint32_t)zz * (uint32_t)cp.cmul2[p];
    }
    sse += inverse_epilogue_i16<R>(w, P, by, bx0 + b, I16RowsInSmem{slot + 16 * b}, valid_rows, 8);
  }
  return sse;
}

// The lane's two int16 blocks (bx0, bx0 + 1) of block-row `by`, one after the
// other (the second is loaded after the first is done: fewer live registers,
// more resident warps).
template <int R>
__device__ __forceinline__ uint32_t codec_lane_i16(const PlaneDesc& P, int by, int bx0,
                                                   const CodecParams& cp) {
  const bool has0 = bx0 < P.nbx, has1 = bx0 + 1 < P.nbx;
  if (!has0) return 0u;
  const int valid_rows = min(8, P.H - by * 8);
  uint32_t sse = 0;
#pragma unroll 1
  for (int b = 0; b < 2; ++b) {
    if (b == 1 && !has1) break;
    const int bx = bx0 + b;
    const int valid_cols = min(8, P.W - bx * 8);
    const bool interior = valid_rows == 8 && valid_cols == 8 && (P.vec16 & 1);
    RowWords<1> rw;
    load_block<1>(P, by, bx, interior, rw);
    sse += codec_block_i16<R>(P, by, bx, I16RowsInRegs{rw.w}, cp, valid_rows, valid_cols);
  }
  return sse;
}

// ---- u8 fast path: two blocks per 32-bit register ------------------------------
//
// The forward transform of the two blocks of a lane runs on packed registers
// v = a + 65536 b (mod 2^32), a from block A, b from block B.  Additions,
// subtractions and doublings act on both lanes at once and are exact modulo
// 2^32; each lane is recovered exactly as long as its final value lies in
// [-32768, 32767].  For u8 samples |Z_ij| <= 144 * 127.5 for (i, j) != (0, 0)
// and 0 <= Z_00 <= 16320, so every coefficient fits (intermediates may wrap).
//
// The inverse is per block in int32 and is streamed row by row into the
// epilogue.  With doubled multipliers the inverse yields 2N + L^2, and
// mulhi(2N + L^2, kDivMagic) carries x' = floor((N + L^2/2) / L^2) in its high
// 16 bits; one prmt packs two of them as s16x2, one min.relu.s16x2 clamps
// both to [0, 255], one prmt packs four bytes.  SSE per block is
// sum x^2 + sum x'^2 - 2 sum x x' from byte dot products (dp4a), exact in
// uint32 arithmetic since the true value is below 2^32.


// Lanes (block A, block B) of the 8 samples of one row pair: p[l] = a_l +
// 65536 b_l.  a02 = [a0, 0, a2, 0] supplies both a sample and a zero byte, so
// each p[l] is one more byte permute with the row word of block B
// (12 permutes per row pair).
__device__ __forceinline__ void pair_row(uint2 a, uint2 b, uint32_t p[8]) {
  const uint32_t a02 = __byte_perm(a.x, 0u, 0x4240u), a13 = __byte_perm(a.x, 0u, 0x4341u);
  const uint32_t a46 = __byte_perm(a.y, 0u, 0x4240u), a57 = __byte_perm(a.y, 0u, 0x4341u);
  // selectors: bytes 0-3 from the a-word, 4-7 from the b-word
  p[0] = __byte_perm(a02, b.x, 0x1410u);
  p[2] = __byte_perm(a02, b.x, 0x1612u);
  p[1] = __byte_perm(a13, b.x, 0x1510u);
  p[3] = __byte_perm(a13, b.x, 0x1712u);
  p[4] = __byte_perm(a46, b.y, 0x1410u);
  p[6] = __byte_perm(a46, b.y, 0x1612u);
  p[5] = __byte_perm(a57, b.y, 0x1510u);
  p[7] = __byte_perm(a57, b.y, 0x1712u);
}


// Round, clamp and pack one row of 8 doubled-and-biased inverse values.
__device__ __forceinline__ uint2 round_pack_row_u8(const uint32_t n2[8]) {
  uint32_t h[8];
#pragma unroll
  for (int l = 0; l < 8; ++l) h[l] = (uint32_t)__mulhi((int32_t)n2[l], kDivMagic);
  const uint32_t c01 = min_relu_s16x2(__byte_perm(h[0], h[1], 0x7632u), 0x00ff00ffu);
  const uint32_t c23 = min_relu_s16x2(__byte_perm(h[2], h[3], 0x7632u), 0x00ff00ffu);
  const uint32_t c45 = min_relu_s16x2(__byte_perm(h[4], h[5], 0x7632u), 0x00ff00ffu);
  const uint32_t c67 = min_relu_s16x2(__byte_perm(h[6], h[7], 0x7632u), 0x00ff00ffu);
  return make_uint2(__byte_perm(c01, c23, 0x6420u), __byte_perm(c45, c67, 0x6420u));
}

// Where the codec reads a block's samples (row k as 8 bytes): row words held
// in registers, or re-read from a shared-memory ring slot (row stride 512 B),
// which keeps 16 registers per block free between the forward and the
// epilogue.
struct RowsInRegs {
  static constexpr bool kInSmem = false;
  const uint2* x;
  __device__ __forceinline__ uint2 row(int k) const { return x[k]; }
};
struct RowsInSmem {
  static constexpr bool kInSmem = true;
  const uint8_t* p;
  __device__ __forceinline__ uint2 row(int k) const {
    return *reinterpret_cast<const uint2*>(p + k * 512);
  }
};

// SSE per row of 8 samples.  1: per-byte absolute differences |x - x'|
// (vabsdiff4), squared and summed by one byte dot product per 4 samples;
// 0: sum x^2 + sum x'^2 - 2 sum x x' from three byte dot products per 4
// samples (sum x^2 formed once per block).
#ifndef TDCT_SSE_ABSDIFF
#define TDCT_SSE_ABSDIFF 1
#endif

__device__ __forceinline__ uint32_t row_sse_terms(uint2 xk, uint2 y, uint32_t acc) {
#if TDCT_SSE_ABSDIFF
  const uint32_t d0 = __vabsdiffu4(xk.x, y.x), d1 = __vabsdiffu4(xk.y, y.y);
  return __dp4a(d0, d0, __dp4a(d1, d1, acc));
#else
  acc = __dp4a(y.x, y.x, acc);
  acc = __dp4a(y.y, y.y, acc);
  return acc - 2u * __dp4a(xk.x, y.x, __dp4a(xk.y, y.y, 0u));
#endif
}

// 1: accumulate each row's SSE terms into one running sum (a dependency
// chain across rows); 0: form each row's terms independently.
#ifndef TDCT_SSE_CHAIN
#define TDCT_SSE_CHAIN 1
#endif

// Inverse of one block from its kept, scaled coefficients w (doubled and
// biased), streamed by rows into rounding, SSE terms and the store.
// `valid_cols` = samples of each row inside the plane (8 when full),
// `valid_rows` = rows inside the plane.  Returns sum x^2 + x'^2 - 2 x x'.
template <int R, typename XS>
__device__ __forceinline__ uint32_t inverse_epilogue_u8(const uint32_t w[64], XS x,
                                                        uint2* __restrict__ out_row0,
                                                        int64_t out_pitch, bool store,
                                                        bool full, int valid_rows,
                                                        int valid_cols) {
  // columns first: v[k][j] = sum_i t_i[k] w[i][j] (only columns with kept entries)
  uint32_t v[64];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    uint32_t col[8], o[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) col[i] = w[8 * i + j];
    inv8<uint32_t>(col, o);
#pragma unroll
    for (int k = 0; k < 8; ++k) v[8 * k + j] = o[k];
  }
  uint32_t acc = 0;
  const uint64_t colmask =
      valid_cols >= 8 ? ~0ull : ((1ull << (8 * valid_cols)) - 1ull);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    uint32_t n2[8];
    inv8<uint32_t>(v + 8 * k, n2);
    uint2 y = round_pack_row_u8(n2);
    if (!full) {
      const uint64_t m = k < valid_rows ? colmask : 0ull;
      y.x &= (uint32_t)m;
      y.y &= (uint32_t)(m >> 32);
    }
    const uint2 xk = x.row(k);
#if TDCT_SSE_CHAIN || TDCT_SSE_ABSDIFF
    acc = row_sse_terms(xk, y, acc);
#else
    // per-row partials are independent; only the final add joins them
    const uint32_t yy = __dp4a(y.x, y.x, __dp4a(y.y, y.y, 0u));
    const uint32_t xy = __dp4a(xk.x, y.x, __dp4a(xk.y, y.y, 0u));
    acc += yy - 2u * xy;
#endif
    if (store && full) out_row0[(int64_t)k * (out_pitch >> 3)] = y;
    if (store && !full && k < valid_rows) {
      uint8_t* row = reinterpret_cast<uint8_t*>(out_row0) + (int64_t)k * out_pitch;
#pragma unroll
      for (int l = 0; l < 8; ++l)
        if (l < valid_cols) row[l] = (uint8_t)((l < 4 ? y.x >> (8 * l) : y.y >> (8 * (l - 4))) & 0xffu);
    }
  }
  return acc;
}

// The inverse with rows first: r[i][l] = sum_j w[i][j] t_j[l] for the kept
// rows only, then each column l: 2N[k][l] + L^2 = sum_i t_i[k] r[i][l] over
// the kept rows.  The dense second pass then has kept_rows(R) inputs instead
// of kept_cols(R); it yields columns, so the rounded samples are packed per
// column pair and the row bytes assembled after columns 0-3 and 4-7.  It
// holds more values live than the row-streaming order.  Policy 4 (default)
// is the per-class choice measured on GB300 for the bulk-copy ring kernel
// (samples re-read from shared memory; bench workload): rows first for
// r-classes 6, 15, 16, 28 and 32 (1-3 % faster there), columns first for the
// others (up to 1 % slower rows first).  Kernels that keep the samples in
// registers use policy 1 (more values live would spill).  Policy 0: never;
// 1: kept set spanning all 8 columns but not all 8 rows; 2: kept_rows(R) <
// kept_cols(R); 3: kept_rows(R) <= kept_cols(R).
#ifndef TDCT_INV_ROWS_FIRST
#define TDCT_INV_ROWS_FIRST 4
#endif

template <int R, int POLICY>
__host__ __device__ constexpr bool inverse_rows_first_policy() {
  return POLICY == 4   ? (R == 6 || R == 15 || R == 16 || R == 28 || R == 32)
         : POLICY == 3 ? kept_rows(R) <= kept_cols(R)
         : POLICY == 2 ? kept_rows(R) < kept_cols(R)
         : POLICY == 1 ? (kept_cols(R) == 8 && kept_rows(R) < 8)
                       : false;
}

template <int R, typename XS>
__host__ __device__ constexpr bool inverse_rows_first() {
  return inverse_rows_first_policy<R, (TDCT_INV_ROWS_FIRST == 4 && !XS::kInSmem)
                                          ? 1 : TDCT_INV_ROWS_FIRST>();
}

template <int R, typename XS>
__device__ __forceinline__ uint32_t inverse_epilogue_u8_rows(const uint32_t w[64], XS x,
                                                             uint2* __restrict__ out_row0,
                                                             int64_t out_pitch, bool store,
                                                             bool full, int valid_rows,
                                                             int valid_cols) {
  uint32_t rr[64];
#pragma unroll
  for (int i = 0; i < 8; ++i) inv8<uint32_t>(w + 8 * i, rr + 8 * i);
  uint32_t yw[2][8];  // packed row bytes: yw[0][k] = samples 0-3 of row k, yw[1][k] = 4-7
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    uint32_t c[2][8];  // clamped s16x2 pairs of columns (4 half + 2 m, +1) per row
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      const int l = 4 * half + 2 * m;
      uint32_t ca[8], cb[8], na[8], nb[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        ca[i] = rr[8 * i + l];
        cb[i] = rr[8 * i + l + 1];
      }
      inv8<uint32_t>(ca, na);
      inv8<uint32_t>(cb, nb);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint32_t ha = (uint32_t)__mulhi((int32_t)na[k], kDivMagic);
        const uint32_t hb = (uint32_t)__mulhi((int32_t)nb[k], kDivMagic);
        c[m][k] = min_relu_s16x2(__byte_perm(ha, hb, 0x7632u), 0x00ff00ffu);
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) yw[half][k] = __byte_perm(c[0][k], c[1][k], 0x6420u);
  }
  uint32_t acc = 0;
  const uint64_t colmask = valid_cols >= 8 ? ~0ull : ((1ull << (8 * valid_cols)) - 1ull);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    uint2 y = make_uint2(yw[0][k], yw[1][k]);
    if (!full) {
      const uint64_t m = k < valid_rows ? colmask : 0ull;
      y.x &= (uint32_t)m;
      y.y &= (uint32_t)(m >> 32);
    }
    const uint2 xk = x.row(k);
    acc = row_sse_terms(xk, y, acc);
    if (store && full) out_row0[(int64_t)k * (out_pitch >> 3)] = y;
    if (store && !full && k < valid_rows) {
      uint8_t* row = reinterpret_cast<uint8_t*>(out_row0) + (int64_t)k * out_pitch;
#pragma unroll
      for (int l = 0; l < 8; ++l)
        if (l < valid_cols) row[l] = (uint8_t)((l < 4 ? y.x >> (8 * l) : y.y >> (8 * (l - 4))) & 0xffu);
    }
  }
  return acc;
}

// Inverse pass order for class R and sample source XS (inverse_rows_first).
template <int R, typename XS>
__device__ __forceinline__ uint32_t inverse_epilogue_u8_any(const uint32_t w[64], XS x,
                                                            uint2* __restrict__ out_row0,
                                                            int64_t out_pitch, bool store,
                                                            bool full, int valid_rows,
                                                            int valid_cols) {
  if constexpr (inverse_rows_first<R, XS>())
    return inverse_epilogue_u8_rows<R, XS>(w, x, out_row0, out_pitch, store, full, valid_rows,
                                       valid_cols);
  else
    return inverse_epilogue_u8<R, XS>(w, x, out_row0, out_pitch, store, full, valid_rows,
                                      valid_cols);
}

// Forward pass order when the kept set is as wide as tall: 1 rows first,
// 0 columns first.
#ifndef TDCT_FWD_ROWS_FIRST_ON_TIE
#define TDCT_FWD_ROWS_FIRST_ON_TIE 1
#endif

// Classes whose bulk-copy ring kernel (rows 16-byte aligned, units within a
// block row) runs 4 CTAs per SM at 128 registers (16 warps, 4 per
// scheduler) instead of 3 at 168: the kernel is bound by dependency latency
// there, and forming both blocks' scaled coefficients right after the
// forward (block B's by one multiply-high each) is what fits it in 128
// registers without spills.  Measured on GB300 (512 or 1024 images
// 1024x1024): 3-4 % faster at classes 15-21; slower at class 8, equal at 32
// (those keep 3 CTAs).
#ifndef TDCT_RING_FOUR_CTAS
#define TDCT_RING_FOUR_CTAS 1
#endif
template <int R>
__host__ __device__ constexpr bool ring_four_ctas() {
  return TDCT_RING_FOUR_CTAS && (R == 15 || R == 16 || R == 21 || R == 28);
}

// Both blocks of a lane (samples already in registers, zero outside the
// plane) through the packed forward and the per-block inverse.
// FULL: the caller guarantees both blocks exist, lie inside the plane and
// that recon (if any) has 8-byte aligned rows (the bulk-copy planes).
// PAIR_OPT (with FULL): the second block may lie past the plane's right
// edge (planes with an odd number of block columns); it is then skipped.
template <int R, bool FULL = false, typename XS = RowsInRegs, bool PAIR_OPT = false>
__device__ __forceinline__ uint32_t codec_pair_u8(const PlaneDesc& P, int by, int bx0, XS xa,
                                                  XS xb, const CodecParams& cp) {
  const bool has0 = FULL || bx0 < P.nbx;
  const bool has1 = FULL ? (!PAIR_OPT || bx0 + 1 < P.nbx) : bx0 + 1 < P.nbx;
  if (!has0) return 0u;
  const int valid_rows = FULL ? 8 : min(8, P.H - by * 8);
  const int vc0 = FULL ? 8 : min(8, P.W - bx0 * 8), vc1 = FULL ? 8 : min(8, P.W - (bx0 + 1) * 8);
  const bool full0 = FULL || (valid_rows == 8 && vc0 == 8);
  const bool full1 = FULL ? has1 : (has1 && valid_rows == 8 && vc1 == 8);
  uint32_t sse = 0;
#if !TDCT_SSE_ABSDIFF
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint2 a = xa.row(k), b = xb.row(k);
    sse = __dp4a(a.x, a.x, sse);
    sse = __dp4a(a.y, a.y, sse);
    sse = __dp4a(b.x, b.x, sse);
    sse = __dp4a(b.y, b.y, sse);
  }
#endif
  // packed forward.  The first pass forms, for each of the 8 rows (or
  // columns), only the outputs inside the kept columns (rows); the second
  // only the kept positions.  Rows first when the kept set is no wider than
  // tall, columns first otherwise (fewer first-pass outputs).
  uint32_t z[64];
  {
    uint32_t pk[64];
#pragma unroll
    for (int k = 0; k < 8; ++k) pair_row(xa.row(k), xb.row(k), pk + 8 * k);
    uint32_t t[64];
    if constexpr (TDCT_FWD_ROWS_FIRST_ON_TIE ? kept_cols(R) <= kept_rows(R) : kept_cols(R) < kept_rows(R)) {
#pragma unroll
      for (int k = 0; k < 8; ++k) fwd8<uint32_t>(pk + 8 * k, t + 8 * k);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint32_t col[8], o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) col[k] = t[8 * k + j];
        fwd8<uint32_t>(col, o);
#pragma unroll
        for (int i = 0; i < 8; ++i) z[8 * i + j] = o[i];
      }
    } else {
#pragma unroll
      for (int l = 0; l < 8; ++l) {
        uint32_t col[8], o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) col[k] = pk[8 * k + l];
        fwd8<uint32_t>(col, o);
#pragma unroll
        for (int i = 0; i < 8; ++i) t[8 * i + l] = o[i];
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) fwd8<uint32_t>(t + 8 * i, z + 8 * i);
    }
  }
  const bool store = P.recon != nullptr;
  const int64_t rp = P.recon_pitch;
  uint2* out0 = store ? reinterpret_cast<uint2*>(P.recon + (int64_t)(by * 8) * rp + (int64_t)bx0 * 8)
                      : nullptr;
  // 4-CTA classes: both blocks' scaled coefficients before either inverse:
  // block A's lane a times c in place of the packed word, block B's from
  // v - a = 2^16 b (exact), as mulhi(2^16 b, 2^16 c) = b c; the packed words
  // die here, which keeps the inverse within 128 registers
  uint32_t w1[64];
  if constexpr (ring_four_ctas<R>()) {
#pragma unroll
    for (int p = 0; p < 64; ++p) {
      if (kept(R, p >> 3, p & 7)) {
        const int32_t lo = lane_lo(z[p]);
        w1[p] = (uint32_t)__mulhi((int32_t)(z[p] - (uint32_t)lo), cp.cmul2h[p]);
        z[p] = (uint32_t)lo * (uint32_t)cp.cmul2[p];
      }
    }
  }
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    if (b == 1 && !has1) break;
    uint32_t w[64];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int p = 8 * i + j;
        if (kept(R, i, j)) {
          if constexpr (ring_four_ctas<R>()) {
            w[p] = b == 0 ? z[p] : w1[p];
          } else {
            const int32_t zz = b == 0 ? lane_lo(z[p]) : lane_hi(z[p]);
            w[p] = (uint32_t)zz * (uint32_t)cp.cmul2[p];
          }
        } else {
          w[p] = 0u;
        }
      }
    w[0] += kL2;  // doubled bias: 2 (N + L^2/2)
    const bool full = b == 0 ? full0 : full1;
    const bool fast_store = store && full && (FULL || (P.vec16 & 2));
    uint2* o = store ? (b == 0 ? out0 : out0 + 1) : nullptr;
    if (!FULL && store && !fast_store) {
      // unaligned recon or edge block: byte stores of valid samples
      sse += inverse_epilogue_u8_any<R, XS>(w, b == 0 ? xa : xb, o, rp, true, false, valid_rows,
                                        b == 0 ? vc0 : vc1);
    } else {
      sse += inverse_epilogue_u8_any<R, XS>(w, b == 0 ? xa : xb, o, rp, store, full, valid_rows,
                                        b == 0 ? vc0 : vc1);
    }
  }
  return sse;
}

// Load both blocks of a lane with plain global loads, then run the codec.
template <int R>
__device__ __forceinline__ uint32_t codec_lane_u8(const PlaneDesc& P, int by, int bx0,
                                                  const CodecParams& cp) {
  const bool has0 = bx0 < P.nbx, has1 = bx0 + 1 < P.nbx;
  if (!has0) return 0u;
  const bool rows_in = by * 8 + 8 <= P.H;
  const bool full0 = rows_in && (bx0 + 1) * 8 <= P.W, full1 = has1 && rows_in && (bx0 + 2) * 8 <= P.W;
  RowWords<0> ra, rb;
  load_block<0>(P, by, bx0, full0 && (P.vec16 & 1), ra);
  if (has1) load_block<0>(P, by, bx0 + 1, full1 && (P.vec16 & 1), rb);
  else {
#pragma unroll
    for (int k = 0; k < 8; ++k) rb.w[k] = make_uint2(0u, 0u);
  }
  return codec_pair_u8<R>(P, by, bx0, RowsInRegs{ra.w}, RowsInRegs{rb.w}, cp);
}

// Persistent fused codec: every warp takes a contiguous range of units.
// Resident CTAs per SM the kernels are compiled for (registers <= 65536 /
// (256 * MINB)).
#ifndef TDCT_U8_MINB
#define TDCT_U8_MINB 2
#endif
#ifndef TDCT_I16_MINB
#define TDCT_I16_MINB 2
#endif

template <int R, int DT>
__global__ void __launch_bounds__(256, DT == 0 ? TDCT_U8_MINB : TDCT_I16_MINB) codec_kernel(const PlaneTable tab, const CodecParams cp,
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
  int next_by = 0, next_chunk = 0;  // unit cursor inside the plane
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
      const int64_t local = u - P.unit_begin;
      next_by = (int)(local / P.chunks);
      next_chunk = (int)(local - (int64_t)next_by * P.chunks);
    }
    const int by = next_by, chunk = next_chunk;
    if (++next_chunk == P.chunks) {
      next_chunk = 0;
      ++next_by;
    }
    if (P.dtype != DT) continue;  // never true for tables the host builds
    if constexpr (DT == 0) acc += codec_lane_u8<R>(P, by, chunk * 64 + 2 * lane, cp);
    else acc += codec_lane_i16<R>(P, by, chunk * 64 + 2 * lane, cp);
  }
  if (p >= 0) {
    acc = warp_sum_u64(acc);
    if (lane == 0 && acc) atomicAdd(sse_out + P.slot, acc);
  }
}

// ---- u8 path with a bulk-copy ring in shared memory -------------------------
//
// Each warp owns STAGES slots of 8 rows x 512 bytes (one unit) in shared
// memory and one mbarrier per slot.  While it computes unit u, the copies of
// its next STAGES - 1 units are in flight: lane k < 8 issues the 1-D bulk
// copy (cp.async.bulk, the TMA engine) of row k of the unit, lane 0 arms the
// slot's mbarrier with the byte count.  The waits are bounded: a wait that
// gives up records TDCT_ETIMEOUT in the status word, drains the warp's other
// copies (again bounded) and ends the warp, so a stuck copy never hangs the
// GPU.  Planes whose rows are not 16-byte aligned, whose width is not a
// multiple of 16 or whose height is not a multiple of 8 take the plain-load
// path (codec_kernel); the host never puts them in a ring launch.  Ring
// planes have H % 8 == 0 and W % 16 == 0, so every existing block is full
// and both blocks of a lane exist together.
constexpr int kUnitBytes = 8 * 512;
// Slot rows of the bulk-copy ring: 512 samples plus the 16 bytes a copy of
// a row that starts 8 bytes past a 16-byte boundary needs (it starts 8 bytes
// early and rounds its length up to a multiple of 16).
constexpr int kRingRowBytes = 528;
constexpr int kRingUnitBytes = 8 * kRingRowBytes;

// A lane's block rows in a bulk-copy ring slot: odd rows of planes whose
// pitch is 8 mod 16 sit 8 bytes further into their slot row.
struct RowsInRing {
  static constexpr bool kInSmem = true;
  const uint8_t* p;      // row 0 of the block in the slot
  const uint8_t* p_odd;  // p + the odd rows' shift (0 or 8)
  __device__ __forceinline__ uint2 row(int k) const {
    return *reinterpret_cast<const uint2*>((k & 1 ? p_odd : p) + k * kRingRowBytes);
  }
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile(
      "{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(bar),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                              uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Suspend-time hint (ns) of the ring kernels' copy waits: 0 = the hardware's
// default time limit per try (tuning knob; measured on GB300).
#ifndef TDCT_RING_WAIT_HINT_NS
#define TDCT_RING_WAIT_HINT_NS 0
#endif

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
#if TDCT_RING_WAIT_HINT_NS > 0
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "n"(TDCT_RING_WAIT_HINT_NS)
      : "memory");
#else
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
#endif
  return ok != 0;
}

// Wait for phase `parity` of `bar`; false if `limit` cycles pass first.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

// Threads per CTA of the bulk-copy ring kernel and the resident CTAs per SM
// it is compiled for (registers <= 65536 / (threads * CTAs)).
// 4 warps x 3 CTAs per SM leave 168 registers per thread, enough for the
// unrolled two-block codec of the classes up to 32 (measured faster than
// 8 warps x 2 CTAs at 128 registers); the classes from 36 up need more live
// values and run faster at 2 CTAs (255 registers) than spilling at 3.
#ifndef TDCT_RING_THREADS
#define TDCT_RING_THREADS 128
#endif

// Resident CTAs per SM the bulk-copy ring kernel is compiled for; the
// shifted-row and row-wrapping variants keep 3 (their 16-warp builds measured
// 2-4 % slower on the ragged batch).
template <int R, bool SHIFT = false, bool WRAP = false>
__host__ __device__ constexpr int ring_min_blocks() {
#ifdef TDCT_RING_MINB
  return TDCT_RING_MINB;
#else
  return R >= 36 ? 2 : (ring_four_ctas<R>() && !SHIFT && !WRAP) ? 4 : 3;
#endif
}

// SHIFT: the launch's planes have a pitch of 8 mod 16 and W % 16 == 8 (odd
// rows start 8 bytes past a 16-byte boundary; the last pair of a block row
// has one block): slot rows of 528 bytes, per-row copy offsets and lengths.
// Otherwise rows are 16-byte aligned with W % 16 == 0: 512-byte slot rows,
// every pair complete.
template <bool SHIFT>
__host__ __device__ constexpr int ring_unit_bytes() {
  return SHIFT ? kRingUnitBytes : kUnitBytes;
}

// Per-plane closing (cp.fin_cnt set), run by one lane for a warp that has
// finished `units` of the `total` units of the plane in `slot`, with SSE
// partial sum v: add v, then (after a fence) the units; the call that brings
// the count to `total` has every other warp's sum in the accumulator, moves
// it to fin_sse with PSNR = 10 log10(255^2 npix / SSE) (+inf for SSE = 0,
// §6.1) and leaves accumulator and count at zero.  No warp waits for another.
// Not inlined: it keeps the main loop's register allocation.
static __device__ __noinline__ void close_plane_units(int slot, int64_t npix,
                                                      unsigned long long v, unsigned int units,
                                                      unsigned int total,
                                                      unsigned long long* acc,
                                                      const CodecParams& cp) {
  if (v) atomicAdd(acc + slot, v);
  __threadfence();
  if (atomicAdd(cp.fin_cnt + slot, units) + units != total) return;
  __threadfence();
  const unsigned long long sse = atomicExch(acc + slot, 0ull);
  atomicExch(cp.fin_cnt + slot, 0u);
  cp.fin_sse[slot] = sse;
  if (cp.fin_psnr)
    cp.fin_psnr[slot] =
        sse == 0ull ? (double)INFINITY : 10.0 * log10(65025.0 * (double)npix / (double)sse);
}

// WRAP: the launch's planes have units that run on across block rows (64
// consecutive blocks in raster order; vec16 bit 5): at most two row segments
// per unit, because such planes are at least 64 blocks wide.  The ring row k
// of a slot holds row k of segment 0 followed by row k of segment 1 (lanes
// 0-7 copy the first, lanes 8-15 the second); the segments hold even block
// counts (the width is a multiple of 16), so the second starts 16-byte
// aligned in the slot and every pair lies in one block row.  A block row
// whose width is not a multiple of 64 blocks then leaves no nearly empty unit
// behind, which at the compute-bound r cost a warp nearly a full unit.
template <int R, int STAGES, bool SHIFT = false, bool WRAP = false>
__global__ void __launch_bounds__(TDCT_RING_THREADS, ring_min_blocks<R, SHIFT, WRAP>())
    codec_u8_tma_kernel(const PlaneTable tab, const CodecParams cp,
                        unsigned long long* __restrict__ sse_out) {
  constexpr int UB = ring_unit_bytes<SHIFT>();
  constexpr int RB = SHIFT ? kRingRowBytes : 512;
  extern __shared__ __align__(128) uint8_t smem[];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  uint8_t* ring = smem + (size_t)wid * STAGES * UB;
  const uint32_t bars = smem_addr(smem + (size_t)(blockDim.x >> 5) * STAGES * UB) +
                        (uint32_t)(wid * STAGES * 8);
  if (lane == 0) {
#pragma unroll
    for (int s = 0; s < STAGES; ++s) mbar_init(bars + 8 * s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();

  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t U = tab.total_units;
  const int64_t u_begin = (U * warp) / nwarps;
  // The warp's units are counted from u_begin in 32 bits (fewer live
  // registers across the loop): a unit holds at least 8 rows x 16 bytes of
  // a ring plane, so even a full device gives under 2^31 units per warp.
  const int n_units = (int)((U * (warp + 1)) / nwarps - u_begin);
  const bool hook = cp.test_hook == 1 && warp == 0;

  // producer cursor: the plane of the next unit to prefetch and the unit's
  // (block-row, chunk) within it, advanced incrementally (a division only
  // when the cursor enters a plane)
  int64_t pp_pitch = 0;
  const uint8_t* pp_img = nullptr;
  int pp_end = -1, pp_W = 0, pp_chunks = 1, pp_by = 0, pp_chunk = 0, pp_s = 0;
  int64_t pp_rem = 0;  // WRAP: blocks from the unit's first to the plane's end
  int pp_nbx = 0;      // WRAP: the plane's block columns (pp_chunk is the unit's first one)
  uint32_t issued = 0;  // bit s: slot s holds a copy in flight
  uint32_t phase = 0;   // bit s: parity of slot s's next completion
  int pf = 0;           // next unit to prefetch (from u_begin)

  auto issue_next = [&]() {
    const int i = pf++;
    const int s = pp_s;
    pp_s = pp_s + 1 == STAGES ? 0 : pp_s + 1;
    if (i >= pp_end) {
      const int64_t u = u_begin + i;
      const int q = find_plane(tab, u);
      const PlaneDesc& Q = tab.d ? tab.d[q] : tab.one;
      pp_img = Q.img;
      pp_pitch = Q.pitch;
      pp_W = Q.W;
      pp_chunks = Q.chunks;
      const int64_t e = ((q + 1 < tab.n) ? tab.d[q + 1].unit_begin : U) - u_begin;
      pp_end = (int)(e < n_units ? e : n_units);
      const int64_t local = u - Q.unit_begin;
      if constexpr (WRAP) {
        const int64_t blk0 = local * 64;
        pp_nbx = Q.nbx;
        pp_by = (int)(blk0 / pp_nbx);
        pp_chunk = (int)(blk0 - (int64_t)pp_by * pp_nbx);
        pp_rem = (int64_t)Q.nbx * Q.nby - blk0;
      } else {
        pp_by = (int)(local / pp_chunks);
        pp_chunk = (int)(local - (int64_t)pp_by * pp_chunks);
      }
    }
    if constexpr (WRAP) {
      const int by0 = pp_by, bx0 = pp_chunk;
      const int rc = (int)(pp_rem < 64 ? pp_rem : 64);
      const int n0 = min(rc, pp_nbx - bx0), n1 = rc - n0;
      pp_rem -= 64;
      pp_chunk += 64;
      if (pp_chunk >= pp_nbx) {
        pp_chunk -= pp_nbx;
        ++pp_by;
      }
      const uint32_t bar = bars + 8 * s;
      const int k = lane & 7, seg = lane >> 3;  // lanes 0-7: segment 0, 8-15: segment 1
      const uint8_t* src = seg == 0 ? pp_img + (int64_t)(by0 * 8 + k) * pp_pitch + (int64_t)bx0 * 8
                                    : pp_img + (int64_t)((by0 + 1) * 8 + k) * pp_pitch;
      const uint32_t bytes = seg == 0 ? 8u * (uint32_t)n0 : 8u * (uint32_t)n1;
      const uint32_t dst_off = (uint32_t)k * 512u + (seg == 0 ? 0u : 8u * (uint32_t)n0);
      // order this warp's earlier generic reads of the slot before the async writes
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (lane == 0) mbar_arrive_expect_tx(bar, 64u * (uint32_t)rc);
      __syncwarp();
      const bool skip = hook && i == 0;
      if (lane < 16 && bytes > 0 && !skip)
        bulk_copy_g2s(smem_addr(ring + s * UB + dst_off), src, bytes, bar);
      issued |= 1u << s;
      return;
    }
    const int by = pp_by, chunk = pp_chunk;
    if (++pp_chunk == pp_chunks) {
      pp_chunk = 0;
      ++pp_by;
    }
    const uint32_t row_bytes = (uint32_t)min(512, pp_W - chunk * 512);
    const uint32_t bar = bars + 8 * s;
    const uint8_t* src = pp_img + (int64_t)(by * 8 + (lane & 7)) * pp_pitch + (int64_t)chunk * 512;
    uint32_t off = 0, bytes = row_bytes, total = 8u * row_bytes;
    if constexpr (SHIFT) {
      // row `lane` (< 8) of the unit: a row that starts 8 bytes past a
      // 16-byte boundary (the odd rows) is copied from 8 bytes earlier, and
      // every copy's length is rounded up to 16 bytes; the host admits such
      // planes only when those extra bytes lie in the plane's neighbouring
      // rows (base 16-byte aligned, W % 16 == 8, H % 8 == 0)
      off = (uint32_t)(reinterpret_cast<uintptr_t>(src) & 15u);
      bytes = lane < 8 ? ((row_bytes + off + 15u) & ~15u) : 0u;
      // even rows of a unit start on a boundary, odd rows 8 bytes past one
      // (an odd multiple of the pitch): four copies of each length
      total = 4u * (((row_bytes + 15u) & ~15u) + ((row_bytes + 8u + 15u) & ~15u));
    }
    // order this warp's earlier generic reads of the slot before the async writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (lane == 0) mbar_arrive_expect_tx(bar, total);
    __syncwarp();
    const bool skip = hook && i == 0;
    if (lane < 8 && !skip)
      bulk_copy_g2s(smem_addr(ring + s * UB + lane * RB), src - off, bytes, bar);
    issued |= 1u << s;
  };

  // Bounded wait for slot s; on failure record the timeout, drain the other
  // slots (bounded) and report false.
  auto wait_slot = [&](int s) -> bool {
    const bool ok = __all_sync(0xffffffffu,
                               mbar_wait_bounded(bars + 8 * s, (phase >> s) & 1u, cp.wait_limit));
    if (ok) {
      phase ^= 1u << s;
      issued &= ~(1u << s);
      return true;
    }
    if (lane == 0 && cp.status) atomicExch(cp.status, 4 /* TDCT_ETIMEOUT */);
    for (int o = 0; o < STAGES; ++o)
      if (o != s && (issued >> o & 1u)) mbar_wait_bounded(bars + 8 * o, (phase >> o) & 1u, cp.wait_limit);
    return false;
  };

  for (int k = 0; k < STAGES && pf < n_units; ++k) issue_next();

  int p = -1;
  int p_end = -1;
  PlaneDesc P;
  unsigned long long acc = 0;
  // The warp's SSE of plane p so far: added to the plane's accumulator, and
  // with per-plane closing (plans) also the warp's units of the plane.
  auto flush_plane = [&]() {
    acc = warp_sum_u64(acc);
    if (cp.fin_cnt) {
      if (lane == 0) {
        const int64_t first = P.unit_begin - u_begin;
        const int64_t end = (p + 1 < tab.n) ? tab.d[p + 1].unit_begin : U;
        close_plane_units(P.slot, (int64_t)P.H * P.W, acc,
                          (unsigned int)(p_end - (first > 0 ? first : 0)),
                          (unsigned int)(end - P.unit_begin), sse_out, cp);
      }
    } else if (lane == 0 && acc) {
      atomicAdd(sse_out + P.slot, acc);
    }
    acc = 0;
  };
  int by = 0, chunk = 0, s = 0;  // consumer cursor, advanced like the producer's
  int64_t rem = 0;               // WRAP: as pp_rem (chunk: the unit's first block column)
  bool failed = false;
  for (int i = 0; i < n_units; ++i) {
    if (i >= p_end) {
      if (p >= 0) flush_plane();
      const int64_t u = u_begin + i;
      p = find_plane(tab, u);
      P = tab.d ? tab.d[p] : tab.one;
      const int64_t e = ((p + 1 < tab.n) ? tab.d[p + 1].unit_begin : U) - u_begin;
      p_end = (int)(e < n_units ? e : n_units);
      const int64_t local = u - P.unit_begin;
      if constexpr (WRAP) {
        const int64_t blk0 = local * 64;
        by = (int)(blk0 / P.nbx);
        chunk = (int)(blk0 - (int64_t)by * P.nbx);
        rem = (int64_t)P.nbx * P.nby - blk0;
      } else {
        by = (int)(local / P.chunks);
        chunk = (int)(local - (int64_t)by * P.chunks);
      }
    }
    if constexpr (WRAP) {
      // the lane's pair: block 2 lane of the unit, in segment 0 or 1
      const int rc = (int)(rem < 64 ? rem : 64);
      const int n0 = min(rc, P.nbx - chunk), pb = 2 * lane;
      const bool has = pb < rc;
      const int lby = pb < n0 ? by : by + 1, lbx = pb < n0 ? chunk + pb : pb - n0;
      const int cur_s = s;
      rem -= 64;
      chunk += 64;
      if (chunk >= P.nbx) {
        chunk -= P.nbx;
        ++by;
      }
      s = s + 1 == STAGES ? 0 : s + 1;
      if (!wait_slot(cur_s)) {
        failed = true;
        break;
      }
      const uint8_t* slot = ring + cur_s * UB + lane * 16;
      if (has)
        acc += codec_pair_u8<R, true>(P, lby, lbx, RowsInSmem{slot}, RowsInSmem{slot + 8}, cp);
      __syncwarp();
      if (pf < n_units) issue_next();  // refill the slot just used
      continue;
    }
    const int bx0 = chunk * 64 + 2 * lane;
    const int cur_by = by, cur_s = s;
    if (++chunk == P.chunks) {
      chunk = 0;
      ++by;
    }
    s = s + 1 == STAGES ? 0 : s + 1;
    if (!wait_slot(cur_s)) {
      failed = true;
      break;
    }
    // the lane's two blocks stay in the slot: the forward reads them, the
    // epilogue reads them again for the SSE; the slot is refilled after
    const uint8_t* slot = ring + cur_s * UB + lane * 16;
    if constexpr (SHIFT) {
      // odd rows sit 8 bytes into their slot rows; the pair may lack its second block
      if (bx0 < P.nbx)
        acc += codec_pair_u8<R, true, RowsInRing, true>(P, cur_by, bx0, RowsInRing{slot, slot + 8},
                                                        RowsInRing{slot + 8, slot + 16}, cp);
    } else {
      if (bx0 < P.nbx)
        acc += codec_pair_u8<R, true>(P, cur_by, bx0, RowsInSmem{slot}, RowsInSmem{slot + 8}, cp);
    }
    __syncwarp();
    if (pf < n_units) issue_next();  // refill the slot just used
  }
  // A warp whose wait gave up flushes its partial sum (the status word
  // reports the launch as incomplete); with per-plane closing it still
  // counts every unit of its range, so that each plane closes and leaves
  // its accumulator at zero.
  if (p >= 0) flush_plane();
  if (failed && cp.fin_cnt) {
    for (int i = p_end; i < n_units;) {
      const int64_t u = u_begin + i;
      p = find_plane(tab, u);
      P = tab.d ? tab.d[p] : tab.one;
      const int64_t e = ((p + 1 < tab.n) ? tab.d[p + 1].unit_begin : U) - u_begin;
      p_end = (int)(e < n_units ? e : n_units);
      flush_plane();
      i = p_end;
    }
  }
}

// Slots per warp of the bulk-copy ring; a slot is refilled after its unit is
// done, so STAGES - 1 units stay in flight while one is computed.  Measured
// on GB300 (bench workload): 4 slots (3 CTAs x 4 warps x 4 x 4 KB = 192 KB
// per SM) for the classes up to 10, where the kernel runs near the memory
// side's limit; 3 slots for classes 15 to 32 (0.5-1.6 % faster there, the
// compute-bound range); 4 for the 2-CTA classes from 36.
template <int R>
__host__ __device__ constexpr int ring_stages() {
#ifdef TDCT_U8_STAGES
  return TDCT_U8_STAGES;
#else
  return (R >= 15 && R <= 32) ? 3 : 4;
#endif
}

// ---- u8 path with a staged-copy ring (rows 8-byte aligned) --------------------
//
// For u8 planes whose rows are 8-byte but not 16-byte aligned (or whose width
// is 8 mod 16), which the bulk-copy engine cannot take.  Same units, slots and
// work split as the bulk-copy ring, but each lane stages only its own two
// blocks: 16 `cp.async` copies of 8 bytes per unit (8 rows x 2 blocks), one
// commit group per unit, `cp.async.wait_group` before the unit is computed.
// A lane reads only what it copied, so no barrier or mbarrier is involved
// and every wait completes with the lane's own copies.  Planes need
// W % 8 == 0 (a lane whose second block lies past the right edge copies and
// codes the first only); rows past the bottom edge are zero-filled in shared
// memory, the pad of partial blocks.
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// (3 CTAs per SM below class 36 whatever ring_four_ctas says: at 128
// registers this kernel spills at class 21)
template <int R, int STAGES>
__global__ void __launch_bounds__(TDCT_RING_THREADS, R >= 36 ? 2 : 3)
    codec_u8_staged_kernel(const PlaneTable tab, const CodecParams cp,
                           unsigned long long* __restrict__ sse_out) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  uint8_t* ring = smem + (size_t)wid * STAGES * kUnitBytes;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t U = tab.total_units;
  const int64_t u_begin = (U * warp) / nwarps;
  const int n_units = (int)((U * (warp + 1)) / nwarps - u_begin);

  // producer cursor, as in the bulk-copy ring
  int64_t pp_pitch = 0;
  const uint8_t* pp_img = nullptr;
  int pp_end = -1, pp_W = 0, pp_H = 0, pp_chunks = 1, pp_by = 0, pp_chunk = 0, pp_s = 0;
  int pf = 0;
  // stage unit pf (if any) into its slot and close one commit group
  auto issue_next = [&]() {
    if (pf < n_units) {
      const int i = pf++;
      const int s = pp_s;
      pp_s = pp_s + 1 == STAGES ? 0 : pp_s + 1;
      if (i >= pp_end) {
        const int64_t u = u_begin + i;
        const int q = find_plane(tab, u);
        const PlaneDesc& Q = tab.d ? tab.d[q] : tab.one;
        pp_img = Q.img;
        pp_pitch = Q.pitch;
        pp_W = Q.W;
        pp_H = Q.H;
        pp_chunks = Q.chunks;
        const int64_t e = ((q + 1 < tab.n) ? tab.d[q + 1].unit_begin : U) - u_begin;
        pp_end = (int)(e < n_units ? e : n_units);
        const int64_t local = u - Q.unit_begin;
        pp_by = (int)(local / pp_chunks);
        pp_chunk = (int)(local - (int64_t)pp_by * pp_chunks);
      }
      const int by = pp_by, chunk = pp_chunk;
      if (++pp_chunk == pp_chunks) {
        pp_chunk = 0;
        ++pp_by;
      }
      const int off = chunk * 512 + 16 * lane;  // the lane's first block, bytes into the row
      if (off < pp_W) {
        const bool second = off + 8 < pp_W;
        const uint8_t* src = pp_img + (int64_t)(by * 8) * pp_pitch + off;
        uint8_t* slot = ring + s * kUnitBytes + lane * 16;
        const uint32_t dst = smem_addr(slot);
        const int rows = min(8, pp_H - by * 8);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          if (k < rows) {
            cp_async8(dst + k * 512, src + (int64_t)k * pp_pitch);
            if (second) cp_async8(dst + k * 512 + 8, src + (int64_t)k * pp_pitch + 8);
          } else {
            *reinterpret_cast<uint4*>(slot + k * 512) = make_uint4(0u, 0u, 0u, 0u);
          }
        }
      }
    }
    cp_async_commit();
  };

  for (int k = 0; k < STAGES - 1; ++k) issue_next();

  int p = -1;
  int p_end = -1;
  PlaneDesc P;
  int by = 0, chunk = 0, s = 0;  // consumer cursor
  unsigned long long acc = 0;
  for (int i = 0; i < n_units; ++i) {
    if (i >= p_end) {
      if (p >= 0) {
        acc = warp_sum_u64(acc);
        if (lane == 0 && acc) atomicAdd(sse_out + P.slot, acc);
        acc = 0;
      }
      const int64_t u = u_begin + i;
      p = find_plane(tab, u);
      P = tab.d ? tab.d[p] : tab.one;
      const int64_t e = ((p + 1 < tab.n) ? tab.d[p + 1].unit_begin : U) - u_begin;
      p_end = (int)(e < n_units ? e : n_units);
      const int64_t local = u - P.unit_begin;
      by = (int)(local / P.chunks);
      chunk = (int)(local - (int64_t)by * P.chunks);
    }
    const int bx0 = chunk * 64 + 2 * lane;
    const int cur_by = by, cur_s = s;
    if (++chunk == P.chunks) {
      chunk = 0;
      ++by;
    }
    s = s + 1 == STAGES ? 0 : s + 1;
    // unit i + STAGES - 1 goes to the slot of unit i - 1, which this lane has
    // finished reading; then unit i's group (STAGES - 1 groups older than the
    // newest) is complete
    issue_next();
    cp_async_wait<STAGES - 1>();
    const uint8_t* slot = ring + cur_s * kUnitBytes + lane * 16;
    if (bx0 < P.nbx)
      acc += codec_pair_u8<R, false>(P, cur_by, bx0, RowsInSmem{slot}, RowsInSmem{slot + 8}, cp);
  }
  cp_async_wait<0>();
  if (p >= 0) {
    acc = warp_sum_u64(acc);
    if (lane == 0 && acc) atomicAdd(sse_out + P.slot, acc);
  }
}

// int16 residual planes with 8-byte aligned rows and W % 8 == 0, any H: the
// staged-copy ring with 8 KB units (8 rows x 64 blocks x 16 B).  A lane
// stages its two blocks (32 copies of 8 bytes; rows past the bottom edge are
// zero-filled in shared memory, the residual pad) and codes them one after
// the other from the slot.  Two slots per warp (3 CTAs x 4 warps x 16 KB).
constexpr int kUnitBytesI16 = 8 * 1024;
constexpr int kStagesI16 = 2;
// Slots per warp of the int16 bulk-copy ring.  Measured on GB300 (256
// planes of 1088 x 1920 residuals): the classes up to 10 are bound by the
// bytes in flight and run faster with 3 slots (2 CTAs x 4 warps x 3 x 8 KB
// per SM; class 8: 0.61 -> 0.66 of the measured HBM peak), the larger
// classes by issue and run faster with 2 slots at 3 CTAs per SM (class 16:
// 0.64 with 2 slots, 0.60-0.62 with 3).
template <int R>
__host__ __device__ constexpr int i16_bulk_stages() {
#ifdef TDCT_I16_BULK_STAGES
  return TDCT_I16_BULK_STAGES;
#else
  return R <= 10 ? 3 : 2;
#endif
}

template <int R>
__global__ void __launch_bounds__(TDCT_RING_THREADS, 3)
    codec_i16_staged_kernel(const PlaneTable tab, const CodecParams cp,
                            unsigned long long* __restrict__ sse_out) {
  constexpr int STAGES = kStagesI16;
  extern __shared__ __align__(128) uint8_t smem[];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  uint8_t* ring = smem + (size_t)wid * STAGES * kUnitBytesI16;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t U = tab.total_units;
  const int64_t u_begin = (U * warp) / nwarps;
  const int n_units = (int)((U * (warp + 1)) / nwarps - u_begin);

  int64_t pp_pitch = 0;
  const uint8_t* pp_img = nullptr;
  int pp_end = -1, pp_W = 0, pp_H = 0, pp_chunks = 1, pp_by = 0, pp_chunk = 0, pp_s = 0;
  int pf = 0;
  auto issue_next = [&]() {
    if (pf < n_units) {
      const int i = pf++;
      const int s = pp_s;
      pp_s = pp_s + 1 == STAGES ? 0 : pp_s + 1;
      if (i >= pp_end) {
        const int64_t u = u_begin + i;
        const int q = find_plane(tab, u);
        const PlaneDesc& Q = tab.d ? tab.d[q] : tab.one;
        pp_img = Q.img;
        pp_pitch = Q.pitch;
        pp_W = Q.W;
        pp_H = Q.H;
        pp_chunks = Q.chunks;
        const int64_t e = ((q + 1 < tab.n) ? tab.d[q + 1].unit_begin : U) - u_begin;
        pp_end = (int)(e < n_units ? e : n_units);
        const int64_t local = u - Q.unit_begin;
        pp_by = (int)(local / pp_chunks);
        pp_chunk = (int)(local - (int64_t)pp_by * pp_chunks);
      }
      const int by = pp_by, chunk = pp_chunk;
      if (++pp_chunk == pp_chunks) {
        pp_chunk = 0;
        ++pp_by;
      }
      const int bx0 = chunk * 64 + 2 * lane;  // the lane's first block
      if (bx0 * 8 < pp_W) {
        const bool second = (bx0 + 1) * 8 < pp_W;
        const uint8_t* src = pp_img + (int64_t)(by * 8) * pp_pitch + (int64_t)bx0 * 16;
        uint8_t* slot = ring + s * kUnitBytesI16 + lane * 32;
        const uint32_t dst = smem_addr(slot);
        const int rows = min(8, pp_H - by * 8);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          if (k < rows) {
            const uint8_t* sk = src + (int64_t)k * pp_pitch;
            cp_async8(dst + k * 1024, sk);
            cp_async8(dst + k * 1024 + 8, sk + 8);
            if (second) {
              cp_async8(dst + k * 1024 + 16, sk + 16);
              cp_async8(dst + k * 1024 + 24, sk + 24);
            }
          } else {
            *reinterpret_cast<uint4*>(slot + k * 1024) = make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint4*>(slot + k * 1024 + 16) = make_uint4(0u, 0u, 0u, 0u);
          }
        }
      }
    }
    cp_async_commit();
  };

  for (int k = 0; k < STAGES - 1; ++k) issue_next();

  int p = -1;
  int p_end = -1;
  PlaneDesc P;
  int by = 0, chunk = 0, s = 0;
  unsigned long long acc = 0;
  for (int i = 0; i < n_units; ++i) {
    if (i >= p_end) {
      if (p >= 0) {
        acc = warp_sum_u64(acc);
        if (lane == 0 && acc) atomicAdd(sse_out + P.slot, acc);
        acc = 0;
      }
      const int64_t u = u_begin + i;
      p = find_plane(tab, u);
      P = tab.d ? tab.d[p] : tab.one;
      const int64_t e = ((p + 1 < tab.n) ? tab.d[p + 1].unit_begin : U) - u_begin;
      p_end = (int)(e < n_units ? e : n_units);
      const int64_t local = u - P.unit_begin;
      by = (int)(local / P.chunks);
      chunk = (int)(local - (int64_t)by * P.chunks);
    }
    const int bx0 = chunk * 64 + 2 * lane;
    const int cur_by = by, cur_s = s;
    if (++chunk == P.chunks) {
      chunk = 0;
      ++by;
    }
    s = s + 1 == STAGES ? 0 : s + 1;
    issue_next();  // into the slot of unit i - 1, which this lane has finished reading
    cp_async_wait<STAGES - 1>();
    const uint8_t* slot = ring + cur_s * kUnitBytesI16 + lane * 32;
    const int valid_rows = min(8, P.H - cur_by * 8);
#pragma unroll 1
    for (int b = 0; b < 2; ++b) {
      if (bx0 + b < P.nbx)
        acc += codec_block_i16<R>(P, cur_by, bx0 + b, I16RowsInSmem{slot + 16 * b}, cp, valid_rows, 8);
    }
  }
  cp_async_wait<0>();
  if (p >= 0) {
    acc = warp_sum_u64(acc);
    if (lane == 0 && acc) atomicAdd(sse_out + P.slot, acc);
  }
}

// int16 residual planes with a 16-byte aligned base and pitch and W % 8 == 0
// (any H): the bulk-copy ring with 8 KB units (8 rows x 64 blocks x 16 B).
// Lanes 0-7 copy one unit row each (cp.async.bulk, the TMA engine, one
// mbarrier per slot, bounded waits as the u8 ring); rows past the bottom
// edge are zero-filled in the slot by the consumer (the residual pad).  The
// lane's two blocks are coded one after the other from the slot, as in the
// staged-copy kernel; STAGES slots per warp, STAGES - 1 units in flight.
template <int R, int STAGES>
__global__ void __launch_bounds__(TDCT_RING_THREADS, 3)
    codec_i16_tma_kernel(const PlaneTable tab, const CodecParams cp,
                         unsigned long long* __restrict__ sse_out) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  uint8_t* ring = smem + (size_t)wid * STAGES * kUnitBytesI16;
  const uint32_t bars = smem_addr(smem + (size_t)(blockDim.x >> 5) * STAGES * kUnitBytesI16) +
                        (uint32_t)(wid * STAGES * 8);
  if (lane == 0) {
#pragma unroll
    for (int s = 0; s < STAGES; ++s) mbar_init(bars + 8 * s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t U = tab.total_units;
  const int64_t u_begin = (U * warp) / nwarps;
  const int n_units = (int)((U * (warp + 1)) / nwarps - u_begin);
  const bool hook = cp.test_hook == 1 && warp == 0;

  int64_t pp_pitch = 0;
  const uint8_t* pp_img = nullptr;
  int pp_end = -1, pp_W = 0, pp_H = 0, pp_chunks = 1, pp_by = 0, pp_chunk = 0, pp_s = 0;
  uint32_t issued = 0, phase = 0;
  int pf = 0;
  auto issue_next = [&]() {
    const int i = pf++;
    const int s = pp_s;
    pp_s = pp_s + 1 == STAGES ? 0 : pp_s + 1;
    if (i >= pp_end) {
      const int64_t u = u_begin + i;
      const int q = find_plane(tab, u);
      const PlaneDesc& Q = tab.d ? tab.d[q] : tab.one;
      pp_img = Q.img;
      pp_pitch = Q.pitch;
      pp_W = Q.W;
      pp_H = Q.H;
      pp_chunks = Q.chunks;
      const int64_t e = ((q + 1 < tab.n) ? tab.d[q + 1].unit_begin : U) - u_begin;
      pp_end = (int)(e < n_units ? e : n_units);
      const int64_t local = u - Q.unit_begin;
      pp_by = (int)(local / pp_chunks);
      pp_chunk = (int)(local - (int64_t)pp_by * pp_chunks);
    }
    const int by = pp_by, chunk = pp_chunk;
    if (++pp_chunk == pp_chunks) {
      pp_chunk = 0;
      ++pp_by;
    }
    const uint32_t row_bytes = (uint32_t)min(1024, 2 * pp_W - chunk * 1024);  // a multiple of 16
    const int rows = min(8, pp_H - by * 8);
    const uint32_t bar = bars + 8 * s;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)rows * row_bytes);
    __syncwarp();
    const bool skip = hook && i == 0;
    if (lane < rows && !skip) {
      const uint8_t* src = pp_img + (int64_t)(by * 8 + lane) * pp_pitch + (int64_t)chunk * 1024;
      bulk_copy_g2s(smem_addr(ring + s * kUnitBytesI16 + lane * 1024), src, row_bytes, bar);
    }
    issued |= 1u << s;
  };
  auto wait_slot = [&](int s) -> bool {
    const bool ok = __all_sync(0xffffffffu,
                               mbar_wait_bounded(bars + 8 * s, (phase >> s) & 1u, cp.wait_limit));
    if (ok) {
      phase ^= 1u << s;
      issued &= ~(1u << s);
      return true;
    }
    if (lane == 0 && cp.status) atomicExch(cp.status, 4 /* TDCT_ETIMEOUT */);
    for (int o = 0; o < STAGES; ++o)
      if (o != s && (issued >> o & 1u)) mbar_wait_bounded(bars + 8 * o, (phase >> o) & 1u, cp.wait_limit);
    return false;
  };

  for (int k = 0; k < STAGES && pf < n_units; ++k) issue_next();

  int p = -1, p_end = -1;
  PlaneDesc P;
  int by = 0, chunk = 0, s = 0;
  unsigned long long acc = 0;
  for (int i = 0; i < n_units; ++i) {
    if (i >= p_end) {
      if (p >= 0) {
        acc = warp_sum_u64(acc);
        if (lane == 0 && acc) atomicAdd(sse_out + P.slot, acc);
        acc = 0;
      }
      const int64_t u = u_begin + i;
      p = find_plane(tab, u);
      P = tab.d ? tab.d[p] : tab.one;
      const int64_t e = ((p + 1 < tab.n) ? tab.d[p + 1].unit_begin : U) - u_begin;
      p_end = (int)(e < n_units ? e : n_units);
      const int64_t local = u - P.unit_begin;
      by = (int)(local / P.chunks);
      chunk = (int)(local - (int64_t)by * P.chunks);
    }
    const int bx0 = chunk * 64 + 2 * lane;
    const int cur_by = by, cur_s = s;
    if (++chunk == P.chunks) {
      chunk = 0;
      ++by;
    }
    s = s + 1 == STAGES ? 0 : s + 1;
    if (!wait_slot(cur_s)) return;
    uint8_t* slot_all = ring + cur_s * kUnitBytesI16;
    const int valid_rows = min(8, P.H - cur_by * 8);
    if (valid_rows < 8) {  // the zero pad below the bottom edge (never copied)
      for (int e = valid_rows * 64 + lane; e < 8 * 64; e += 32)
        reinterpret_cast<uint4*>(slot_all)[e] = make_uint4(0u, 0u, 0u, 0u);
      __syncwarp();
    }
    const uint8_t* slot = slot_all + lane * 32;
    if constexpr (i16_packed_forward<R>()) {
      if (bx0 < P.nbx)
        acc += codec_pair_i16<R>(P, cur_by, bx0, slot, cp, valid_rows, bx0 + 1 < P.nbx);
    } else {
#pragma unroll 1
      for (int b = 0; b < 2; ++b) {
        if (bx0 + b < P.nbx)
          acc += codec_block_i16<R>(P, cur_by, bx0 + b, I16RowsInSmem{slot + 16 * b}, cp,
                                    valid_rows, 8);
      }
    }
    __syncwarp();
    if (pf < n_units) issue_next();  // refill the slot just used
  }
  if (p >= 0) {
    acc = warp_sum_u64(acc);
    if (lane == 0 && acc) atomicAdd(sse_out + P.slot, acc);
  }
}

inline int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return sms > 0 ? sms : 1;
}

// Host-side launcher of one instantiation (defined where instantiated).
// `max_ctas` > 0 caps the persistent grid (autotuning, tests).
template <int R, int DT>
cudaError_t launch_codec(const PlaneTable& tab, const CodecParams& cp, unsigned long long* sse,
                         int max_ctas, cudaStream_t s) {
  constexpr int kThreads = 256;
  constexpr int kRingThreads = TDCT_RING_THREADS;
  constexpr int kStages = ring_stages<R>();
  constexpr size_t kSmem = (size_t)(kRingThreads / 32) * kStages * (kUnitBytes + 8);
  constexpr size_t kSmemShift = (size_t)(kRingThreads / 32) * kStages * (kRingUnitBytes + 8);
  constexpr size_t kSmemStaged = (size_t)(kRingThreads / 32) * kStages * kUnitBytes;
  static int resident = 0, resident_bulk = 0, resident_staged = 0, resident_shift = 0;
  static int resident_wrap = 0;
  static int sms = 0;
  if (resident == 0) {
    sms = device_sms();
    cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, codec_kernel<R, DT>, kThreads, 0);
    if (e != cudaSuccess) return e;
    if (resident < 1) resident = 1;
    if constexpr (DT == 0) {
      e = cudaFuncSetAttribute(codec_u8_tma_kernel<R, kStages>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
      if (e != cudaSuccess) return e;
      e = cudaFuncSetAttribute(codec_u8_tma_kernel<R, kStages>,
                               cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
      if (e != cudaSuccess) return e;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &resident_bulk, codec_u8_tma_kernel<R, kStages>, kRingThreads, kSmem);
      if (e != cudaSuccess) return e;
      if (resident_bulk < 1) resident_bulk = 1;
      e = cudaFuncSetAttribute(codec_u8_tma_kernel<R, kStages, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemShift);
      if (e != cudaSuccess) return e;
      e = cudaFuncSetAttribute(codec_u8_tma_kernel<R, kStages, true>,
                               cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
      if (e != cudaSuccess) return e;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &resident_shift, codec_u8_tma_kernel<R, kStages, true>, kRingThreads, kSmemShift);
      if (e != cudaSuccess) return e;
      if (resident_shift < 1) resident_shift = 1;
      e = cudaFuncSetAttribute(codec_u8_tma_kernel<R, kStages, false, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
      if (e != cudaSuccess) return e;
      e = cudaFuncSetAttribute(codec_u8_tma_kernel<R, kStages, false, true>,
                               cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
      if (e != cudaSuccess) return e;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &resident_wrap, codec_u8_tma_kernel<R, kStages, false, true>, kRingThreads, kSmem);
      if (e != cudaSuccess) return e;
      if (resident_wrap < 1) resident_wrap = 1;
      e = cudaFuncSetAttribute(codec_u8_staged_kernel<R, kStages>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemStaged);
      if (e != cudaSuccess) return e;
      e = cudaFuncSetAttribute(codec_u8_staged_kernel<R, kStages>,
                               cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
      if (e != cudaSuccess) return e;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &resident_staged, codec_u8_staged_kernel<R, kStages>, kRingThreads, kSmemStaged);
      if (e != cudaSuccess) return e;
      if (resident_staged < 1) resident_staged = 1;
    }
  }
  if constexpr (DT == 1) {
    if (tab.any_bulk) {
      constexpr int kSt = i16_bulk_stages<R>();
      constexpr size_t kSmemI16B = (size_t)(kRingThreads / 32) * kSt * (kUnitBytesI16 + 8);
      static int resident_i16b = 0;
      if (resident_i16b == 0) {
        cudaError_t e = cudaFuncSetAttribute(codec_i16_tma_kernel<R, kSt>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kSmemI16B);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(codec_i16_tma_kernel<R, kSt>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident_i16b,
                                                          codec_i16_tma_kernel<R, kSt>,
                                                          kRingThreads, kSmemI16B);
        if (e != cudaSuccess) return e;
        if (resident_i16b < 1) resident_i16b = 1;
      }
      int per_sm = resident_i16b;
      if (cp.ctas_per_sm > 0 && cp.ctas_per_sm < per_sm) per_sm = cp.ctas_per_sm;
      int64_t grid = (int64_t)per_sm * sms;
      const int64_t by_work = (tab.total_units + kRingThreads / 32 - 1) / (kRingThreads / 32);
      if (by_work < grid) grid = by_work;
      if (max_ctas > 0 && grid > max_ctas) grid = max_ctas;
      if (grid < 1) grid = 1;
      codec_i16_tma_kernel<R, kSt><<<(unsigned)grid, kRingThreads, kSmemI16B, s>>>(tab, cp, sse);
      return cudaGetLastError();
    }
    if (tab.staged) {
      constexpr size_t kSmemI16 = (size_t)(kRingThreads / 32) * kStagesI16 * kUnitBytesI16;
      static int resident_i16 = 0;
      if (resident_i16 == 0) {
        cudaError_t e = cudaFuncSetAttribute(codec_i16_staged_kernel<R>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kSmemI16);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(codec_i16_staged_kernel<R>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident_i16, codec_i16_staged_kernel<R>,
                                                          kRingThreads, kSmemI16);
        if (e != cudaSuccess) return e;
        if (resident_i16 < 1) resident_i16 = 1;
      }
      int per_sm = resident_i16;
      if (cp.ctas_per_sm > 0 && cp.ctas_per_sm < per_sm) per_sm = cp.ctas_per_sm;
      int64_t grid = (int64_t)per_sm * sms;
      const int64_t by_work = (tab.total_units + kRingThreads / 32 - 1) / (kRingThreads / 32);
      if (by_work < grid) grid = by_work;
      if (max_ctas > 0 && grid > max_ctas) grid = max_ctas;
      if (grid < 1) grid = 1;
      codec_i16_staged_kernel<R><<<(unsigned)grid, kRingThreads, kSmemI16, s>>>(tab, cp, sse);
      return cudaGetLastError();
    }
  }
  const bool bulk = DT == 0 && tab.any_bulk;
  const bool staged = DT == 0 && !bulk && tab.staged;
  int per_sm = bulk ? (tab.shifted ? resident_shift : tab.wrap ? resident_wrap : resident_bulk)
                   : staged ? resident_staged : resident;
  if (cp.ctas_per_sm > 0 && cp.ctas_per_sm < per_sm) per_sm = cp.ctas_per_sm;
  int64_t grid = (int64_t)per_sm * sms;
  const int threads = (bulk || staged) ? kRingThreads : kThreads;
  const int64_t by_work = (tab.total_units + threads / 32 - 1) / (threads / 32);
  if (by_work < grid) grid = by_work;
  if (max_ctas > 0 && grid > max_ctas) grid = max_ctas;
  if (grid < 1) grid = 1;
  if constexpr (DT == 0) {
    if (bulk) {
      if (tab.shifted)
        codec_u8_tma_kernel<R, kStages, true>
            <<<(unsigned)grid, kRingThreads, kSmemShift, s>>>(tab, cp, sse);
      else if (tab.wrap)
        codec_u8_tma_kernel<R, kStages, false, true>
            <<<(unsigned)grid, kRingThreads, kSmem, s>>>(tab, cp, sse);
      else
        codec_u8_tma_kernel<R, kStages><<<(unsigned)grid, kRingThreads, kSmem, s>>>(tab, cp, sse);
      return cudaGetLastError();
    }
    if (staged) {
      codec_u8_staged_kernel<R, kStages><<<(unsigned)grid, kRingThreads, kSmemStaged, s>>>(tab, cp,
                                                                                         sse);
      return cudaGetLastError();
    }
  }
  codec_kernel<R, DT><<<(unsigned)grid, kThreads, 0, s>>>(tab, cp, sse);
  return cudaGetLastError();
}

}  // namespace tdct
