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
// as they are: the DC position is always kept and the kept-coefficient
// reconstruction is an orthogonal projection, so it maps X to
// 128 + P(X - 128) and |x'_exact - 128| <= ||X - 128||_F <= 128 B; then
// |2N + L^2 - 256 L^2| <= (256 B + 1) L^2 < 2^31 for B <= 32, and the
// column and row inverses run in 32-bit integers (wrapping intermediates,
// exact result).  For int16 residuals the row inverse runs in 64 bits.
//
// Work: a lane owns one row of a block (two 16x16 blocks or one 32x32 block
// side by side in a warp, NP such groups per iteration); rows are
// transformed in registers, columns after a transpose through a padded
// shared-memory tile (column-major, so the column stage moves whole columns
// with 16-byte accesses), and back.  Rows arrive through a per-warp ring of
// asynchronous copies.  Kernels are compiled per kept-extent class KE
// (every kept position (i, j) has i, j < KE): the row forward forms KE
// outputs, only the KE leading columns are transformed, and the row inverse
// has KE inputs; the exact r is applied at run time.  The kernel is bound by
// instruction issue and the integer multiply-add pipe (the multiply-highs of
// the rounding and most adds land there), so sign flips are written as
// logic-unit operations and the per-pixel arithmetic is kept to the
// transforms, one multiply-high, the packing and the byte SSE.
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
// The row inverse (second stage) in 32 bits: u8 samples, where the result
// 2N + L^2 + 128 * 2 L^2 lies within +-(256 B + 257) L^2 < 2^31 for B <= 32
// (the intermediates may wrap; the ring arithmetic mod 2^32 keeps the result
// exact).
template <int B, int DT>
constexpr bool kStageB32 = (DT == 0);

// A contiguous run of N tile entries (16-byte aligned) moved with 16-byte
// accesses: the low 32 bits of each entry in, full entries out.
template <typename TileT, int N>
__device__ __forceinline__ void col_load(const TileT* p, uint32_t* v) {
  const uint4* q = reinterpret_cast<const uint4*>(p);
  if constexpr (sizeof(TileT) == 4) {
#pragma unroll
    for (int i = 0; i < N / 4; ++i) {
      const uint4 t = q[i];
      v[4 * i] = t.x, v[4 * i + 1] = t.y, v[4 * i + 2] = t.z, v[4 * i + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      const uint4 t = q[i];
      v[2 * i] = t.x, v[2 * i + 1] = t.z;
    }
  }
}
template <typename TileT, int N, typename V>
__device__ __forceinline__ void col_store(TileT* p, const V* v) {
  uint4* q = reinterpret_cast<uint4*>(p);
  if constexpr (sizeof(TileT) == 4) {
#pragma unroll
    for (int i = 0; i < N / 4; ++i)
      q[i] = make_uint4((uint32_t)v[4 * i], (uint32_t)v[4 * i + 1], (uint32_t)v[4 * i + 2],
                        (uint32_t)v[4 * i + 3]);
  } else {
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      const unsigned long long a = (unsigned long long)(long long)v[2 * i];
      const unsigned long long b = (unsigned long long)(long long)v[2 * i + 1];
      q[i] = make_uint4((uint32_t)a, (uint32_t)(a >> 32), (uint32_t)b, (uint32_t)(b >> 32));
    }
  }
}

template <int B, int DT, int KE, int PF, int NP>
__global__ void __launch_bounds__(128) jam_codec_kernel(const PlaneDesc P, const JamParams jp,
                                                        unsigned long long* __restrict__ sse_out) {
  constexpr int BPW = 32 / B;   // blocks side by side in a warp (a lane per row)
  constexpr int BPI = BPW * NP;  // blocks per warp iteration: NP such groups
  constexpr int SB = DT == 0 ? 1 : 2;
  using VA = StageA<B, DT>;
  using VB = std::conditional_t<kStageB32<B, DT>, uint32_t, long long>;
  using TileT = std::conditional_t<std::is_same_v<VA, uint32_t>, int32_t, long long>;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int bsub = lane / B, k = lane % B;
  // a plane holds fewer than 2^30 blocks (the host checks), so block
  // indices, and one grid stride past them, fit in 32 bits
  const int nbx = (P.W + B - 1) / B, nby = (P.H + B - 1) / B;
  const int nb = nbx * nby;
  const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  // the column stage: two lanes per column when the kept extent allows at
  // 16x16 blocks (the two branches of the first JAM stage), four at 32x32 u8
  // blocks (the two branches of the first two stages) with 4 KE <= 32
  constexpr bool kSplit = B == 16 && 2 * KE <= B;
  constexpr bool kSplit4 = B == 32 && DT == 0 && 4 * KE <= B;
  // The block's KE leading columns, stored column by column (a column is
  // contiguous, so the column stage moves it with 16-byte accesses): column c
  // at c * kS, entry of row i at pos(i), where the split stages order the rows
  // so that each lane of a column's pair (quad) owns one contiguous half
  // (quarter) of the outputs: two lanes, rows 0..15 then 31 down to 16; four
  // lanes, rows 0..7, 15 down to 8, 31 down to 24, 16..23.  kS pads a column by 16 bytes; the blocks of a
  // warp sit 16 banks apart (row accesses of the two halves do not collide).
  constexpr int kEl = (int)sizeof(TileT);
  constexpr int kS = B + 16 / kEl;
  constexpr int kBlkWords = KE * kS * kEl / 4;
  constexpr int kBlk = (KE * kS + ((16 - kBlkWords % 32 + 32) % 32) * 4 / kEl);
  __shared__ __align__(16) TileT tile[4][NP][BPW][kBlk];
  const int pk_ = kSplit4 ? (k < 8 ? k : k < 16 ? 23 - k : k < 24 ? k + 8 : 47 - k)
                  : (kSplit && k >= B / 2) ? (3 * B / 2 - 1 - k) : k;  // pos(k)
  constexpr uint32_t kBlockMask = (2 * KE >= 32) ? 0xffffffffu : ((1u << (2 * KE)) - 1u);
  constexpr uint32_t kSplitMask = B == 16 ? (kBlockMask | (kBlockMask << 16)) : kBlockMask;
  constexpr uint32_t kQuadMask = (4 * KE >= 32) ? 0xffffffffu : ((1u << (4 * KE)) - 1u);
  // the lane's column in the column stage and its kept rows
  const int ccol = kSplit4 ? (k >> 2) : kSplit ? (k >> 1) : k;
  const int hk = kept_height(B, jp.r, ccol);
  // rounding bias folded into the DC input of the row inverse (T's first row
  // is all ones, so it reaches every output): L^2 for u8 samples; int16
  // residuals round half away from zero on |2N| instead
  const VB bias = DT == 0 ? (VB)jp.L2 : (VB)0;
  // the zonal mask and the doubled q_i of the column stage, per lane: entry i
  // multiplies the i-th output of the lane's column forward (zero where the
  // position is not kept); held in registers up to 8 entries.  With the
  // 32-bit row inverse the column's own q_c joins it (the row inverse then
  // takes V'[k][c] q_c straight from the tile; products wrap mod 2^32, the
  // result does not).
  constexpr bool kFoldQ = kStageB32<B, DT>;
  constexpr int kNQ = kSplit4 ? (KE + 3) / 4 : kSplit ? KE / 2 : KE;
  constexpr int kNQR = kNQ <= 8 ? kNQ : 1;
  int32_t qm2r[kNQR];
  const int qc = kFoldQ ? jp.q[min(ccol, KE - 1)] : 1;
  auto qm2_of = [&](int i) {
    // the row of Z that output i of the lane's last-stage forward is
    const int ifull = kSplit4 ? 4 * i + (k & 3) : kSplit ? 2 * i + (k & 1) : i;
    return ifull < hk ? (int32_t)((uint32_t)(2 * jp.q[ifull]) * (uint32_t)qc) : 0;
  };
#pragma unroll
  for (int i = 0; i < kNQR; ++i) qm2r[i] = qm2_of(i);
  auto qm2 = [&](int i) { return kNQ <= 8 ? qm2r[i < kNQR ? i : 0] : qm2_of(i); };
  unsigned long long acc = 0;
  // Geometry of the lane's blocks (indices base + p BPW + bsub at warp
  // position base, p < NP), stepped by the grid stride without a division
  // per iteration.
  struct __align__(8) Geo {
    int by, bx;
  };
  const int nbx_full = P.W / B, nby_full = P.H / B;
  const int stride = nwarps * BPI;
  const int sby = stride / nbx, sbx = stride - sby * nbx;
  auto step = [&](Geo& g) {
    g.bx += sbx;
    g.by += sby;
    if (g.bx >= nbx) {
      g.bx -= nbx;
      ++g.by;
    }
  };
  Geo gf[NP];  // the blocks being fetched
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int blk = warp * BPI + p * BPW + bsub;
    gf[p].by = blk / nbx;
    gf[p].bx = blk - gf[p].by * nbx;
  }
  // Rows reach the warp through a ring of PF slots in shared memory, filled by
  // asynchronous 16-byte copies (cp.async, one commit group per iteration):
  // the loads of the next PF iterations are in flight while one is
  // transformed.  Each lane reads back only the words it copied (or stored,
  // for blocks that cross the plane's edge), so the ring needs no barrier.
  extern __shared__ uint4 jam_ring[];
  constexpr int kW = RowRaw<B, DT>::kWords;
  // row p of slot s, per lane: + (s NP + p) 32 kW
  uint4* const ring = jam_ring + ((size_t)wid * PF * NP * 32 + lane) * kW;
  // the block geometry of each row, per lane, after the rows
  Geo* const ring_geo =
      reinterpret_cast<Geo*>(jam_ring + 4 * PF * NP * 32 * kW) + wid * PF * NP * 32 + lane;
  auto fetch_row = [&](const Geo& g, int slot, int p) {
    uint4* dst = ring + (slot * NP + p) * 32 * kW;
    ring_geo[(slot * NP + p) * 32] = g;
    const int fy = g.by * B + k;
    if (g.by < nby_full && g.bx < nbx_full && (jp.aligned & 1)) {
      const uint4* src =
          reinterpret_cast<const uint4*>(P.img + (int64_t)fy * P.pitch + (int64_t)g.bx * B * SB);
#pragma unroll
      for (int q = 0; q < kW; ++q)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(dst + q)),
                     "l"(src + q)
                     : "memory");
    } else {
      uint32_t u[4 * kW];
#pragma unroll
      for (int q = 0; q < 4 * kW; ++q) u[q] = 0u;
      if (g.by < nby) {
#pragma unroll
        for (int l = 0; l < B; ++l) {
          const uint32_t v = (uint32_t)load_px<DT>(P, fy, g.bx * B + l);
          if (DT == 0) u[l >> 2] |= (v & 0xffu) << (8 * (l & 3));
          else u[l >> 1] |= (v & 0xffffu) << (16 * (l & 1));
        }
      }
#pragma unroll
      for (int q = 0; q < kW; ++q) dst[q] = make_uint4(u[4 * q], u[4 * q + 1], u[4 * q + 2], u[4 * q + 3]);
    }
  };
#pragma unroll
  for (int s = 0; s < PF; ++s) {
    if (warp * BPI + s * stride < nb) {
#pragma unroll
      for (int p = 0; p < NP; ++p) fetch_row(gf[p], s, p);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
#pragma unroll
    for (int p = 0; p < NP; ++p) step(gf[p]);
  }
  int slot = 0;
  for (int base = warp * BPI; base < nb; base += stride) {
    asm volatile("cp.async.wait_group %0;" ::"n"(PF - 1) : "memory");
    RowRaw<B, DT> raws[NP];  // the raw rows stay for the error
    Geo gc[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
#pragma unroll
      for (int q = 0; q < kW; ++q) raws[p].w[q] = ring[(slot * NP + p) * 32 * kW + q];
      gc[p] = ring_geo[(slot * NP + p) * 32];
    }
    if (base + PF * stride < nb) {
#pragma unroll
      for (int p = 0; p < NP; ++p) fetch_row(gf[p], slot, p);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
#pragma unroll
    for (int p = 0; p < NP; ++p) step(gf[p]);
    slot = slot + 1 == PF ? 0 : slot + 1;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      TileT* const tl = tile[wid][p][bsub];
      const RowRaw<B, DT>& raw = raws[p];
      // rows: t = T x for row k of the block (KE leading outputs)
      if constexpr (DT == 0) {
        // u8: the mirrored samples x_m and x_(B-1-m) travel as one word
        // x_m + 2^16 x_(B-1-m) through the half-size forward T', whose outputs
        // are then f_i + 2^16 g_i with f = T' x_(0..B/2-1) and g = T' of the
        // mirrored half (both within +-12 * 255 * B / 16: exact in 16 bits).
        // The first JAM stage is linear, so t_(2i) = f_i + g_i and
        // t_(2i+1) = f_i - g_i.
        const uint32_t* ru = reinterpret_cast<const uint32_t*>(raw.w);
        uint32_t pk[B / 2], o[B / 2];
  #pragma unroll
        for (int m = 0; m < B / 2; m += 2) {
          const int l = B - 1 - m;  // l - 1 mirrors m + 1, in the same word as l
          // bytes x_m, x_(m+1), x_l, x_(l-1)
          const uint32_t w = __byte_perm(ru[m >> 2], ru[l >> 2],
                                         (uint32_t)((m & 3) | ((m & 3) + 1) << 4 |
                                                    (4 + (l & 3)) << 8 | (4 + (l & 3) - 1) << 12));
          pk[m] = __byte_perm(w, 0u, 0x4240u);
          pk[m + 1] = __byte_perm(w, 0u, 0x4341u);
        }
        jam_fwd<B / 2, uint32_t>(pk, o);
  #pragma unroll
        for (int i = 0; i < KE / 2; ++i) {
          const int32_t f = (int32_t)(int16_t)(o[i] & 0xffffu);
          const int32_t g = (int32_t)(o[i] + 0x8000u) >> 16;
          tl[(2 * i) * kS + pk_] = (TileT)(f + g);
          tl[(2 * i + 1) * kS + pk_] = (TileT)(f - g);
        }
      } else {
        uint32_t x[B], t[B];
  #pragma unroll
        for (int l = 0; l < B; ++l) x[l] = (uint32_t)raw.at(l);
        jam_fwd<B, uint32_t>(x, t);
  #pragma unroll
        for (int j = 0; j < KE; ++j) tl[j * kS + pk_] = (TileT)(int32_t)t[j];
      }
    }
    __syncwarp();
    // columns c < KE: Z[i][c] (i < KE), zonal mask with 2 q_i, inverse along
    // the column.  With 2 KE <= B = 16 two lanes share a column: lane half h takes
    // the sums (h = 0: even rows of Z) or the differences (h = 1: odd rows)
    // of the first JAM stage, the half-size forward and inverse, and the
    // pair combines u +- w by one exchange; otherwise one lane per column.
    // Lanes write only the column they read.
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      TileT* const tl = tile[wid][p][bsub];
      if constexpr (kSplit) {
        if (k < 2 * KE) {
          const int c = k >> 1;
          // sign flips as (x ^ hm) - hm (hm all ones for h = 1): logic-unit
          // operations, which leave the multiply-add pipe (the busier one here)
          // to the transforms
          const uint32_t hm = (k & 1) ? 0xffffffffu : 0u;
          uint32_t col[B], v[B / 2], zh[B / 2];
          col_load<TileT, B>(tl + c * kS, col);  // rows 0..B/2-1, then B-1 down to B/2
  #pragma unroll
          for (int m = 0; m < B / 2; ++m) v[m] = col[m] + (col[B / 2 + m] ^ hm) - hm;
          jam_fwd<B / 2, uint32_t>(v, zh);  // zh[i] = Z[2 i + h][c]
          VA w[B / 2], rh[B / 2];
  #pragma unroll
          for (int i = 0; i < B / 2; ++i) w[i] = i < kNQ ? (VA)(zh[i] * (uint32_t)qm2(i)) : (VA)0;
          jam_inv<B / 2, VA>(w, rh);  // h = 0: u, h = 1: w
          VA val[B / 2];
  #pragma unroll
          for (int m = 0; m < B / 2; ++m) {
            const VA pm = __shfl_xor_sync(kSplitMask, rh[m], 1);
            // h = 0: row m = u + w; h = 1: row B - 1 - m = u - w
            val[m] = pm + (rh[m] ^ hm) - hm;
          }
          col_store<TileT, B / 2>(tl + c * kS + (k & 1) * (B / 2), val);
        }
      } else if constexpr (kSplit4) {
        // four lanes per column: lane bit 0 picks the branch of the first JAM
        // stage (sums x_m + x_(31-m) or differences), bit 1 that of the
        // second on the resulting 16-point signal; each lane runs the 8-point
        // forward (Z rows 4 i + (k & 3)), the mask and the 8-point inverse, and
        // two exchanges (lane ^ 2, then lane ^ 1) rebuild the 16- and
        // 32-point inverses, a quarter of the column per lane
        if (k < 4 * KE) {
          const int c = k >> 2;
          const uint32_t s1 = (k & 1) ? 0xffffffffu : 1u, s2 = (k & 2) ? 0xffffffffu : 1u;
          uint32_t col[B], y8[8], z8[8];
          col_load<TileT, B>(tl + c * kS, col);  // rows 0..7, 15..8, 31..24, 16..23
  #pragma unroll
          for (int m = 0; m < 8; ++m)
            y8[m] = (col[m] + s1 * col[16 + m]) + s2 * (col[8 + m] + s1 * col[24 + m]);
          jam_fwd<8, uint32_t>(y8, z8);
          VA w[8], r8[8];
  #pragma unroll
          for (int i = 0; i < 8; ++i) w[i] = i < kNQ ? (VA)(z8[i] * (uint32_t)qm2(i)) : (VA)0;
          jam_inv<8, VA>(w, r8);
          VA v2[8], v1[8];
  #pragma unroll
          for (int m = 0; m < 8; ++m) v2[m] = __shfl_xor_sync(kQuadMask, r8[m], 2) + s2 * r8[m];
  #pragma unroll
          for (int m = 0; m < 8; ++m) v1[m] = __shfl_xor_sync(kQuadMask, v2[m], 1) + s1 * v2[m];
          col_store<TileT, 8>(tl + c * kS + 8 * (2 * (k & 1) + ((k >> 1) & 1)), v1);
        }
      } else if (k < KE) {
        uint32_t col[B], z[B];
        col_load<TileT, B>(tl + k * kS, col);
        jam_fwd<B, uint32_t>(col, z);
        VA w[B], u[B];
  #pragma unroll
        for (int i = 0; i < B; ++i) w[i] = i < kNQ ? (VA)((long long)(int32_t)z[i] * qm2(i)) : (VA)0;
        jam_inv<B, VA>(w, u);
        col_store<TileT, B>(tl + k * kS, u);
      }
    }
    __syncwarp();
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      TileT* const tl = tile[wid][p][bsub];
      const RowRaw<B, DT>& raw = raws[p];
      const int by = gc[p].by, bx = gc[p].bx;
      const bool valid = by < nby, full = by < nby_full && bx < nbx_full;
      const int y = by * B + k;
      // row k: 2N[k][l] + bias = sum_j q_j V'[k][j] T[j][l] (j < KE); round,
      // clamp, error, store
      {
        VB v[B], n2[B];
  #pragma unroll
        for (int j = 0; j < B; ++j)
          v[j] = j >= KE ? (VB)0 : kFoldQ ? (VB)tl[j * kS + pk_] : (VB)tl[j * kS + pk_] * (VB)jp.q[j];
        v[0] += bias;
        jam_inv<B, VB>(v, n2);
        RowRaw<B, DT> out;
        uint32_t* ou = reinterpret_cast<uint32_t*>(out.w);
  #pragma unroll
        for (int q = 0; q < 4 * RowRaw<B, DT>::kWords; ++q) ou[q] = 0u;
        uint32_t sse = 0;
        const bool row_in = valid && y < P.H;
        if constexpr (kStageB32<B, DT>) {
          // n2 = 2N + L^2 exactly (|n2 - 256 L^2| <= (256 B + 1) L^2); the signed
          // high product with magic16 carries floor(n2 / (2 L^2)) = x' in its
          // upper 16 bits for 0 <= n2 <= 256 * 2 L^2 (host-checked), at least
          // 256 above that (the product is monotone) and a negative value below
          // 0, all within 16 bits (|n2| < 2^31 keeps |x'| < 2^13); pairs are
          // clamped to [0, 255] as s16x2 and packed to bytes
          uint32_t h[B];
  #pragma unroll
          for (int l = 0; l < B; ++l) h[l] = (uint32_t)__mulhi((int32_t)n2[l], jp.magic16);
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
    }
    __syncwarp();
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0 && acc) atomicAdd(sse_out, acc);
}

// Kept-extent classes: the smallest class at least the extent of the first
// r zig-zag positions of a B x B block.
__host__ __device__ constexpr int jam_extent_class(int ext) {
  return ext <= 2 ? 2 : ext <= 4 ? 4 : ext <= 6 ? 6 : ext <= 8 ? 8 : ext <= 12 ? 12
       : ext <= 16 ? 16 : ext <= 24 ? 24 : 32;
}

// Ring depth (iterations of row loads in flight per warp).  The kernel is
// bound by instruction issue and the integer multiply-add pipe, not memory
// latency: 2 stages were fastest at both block sizes, 4 up to 4 % slower.
template <int B, int DT>
constexpr int jam_stages() {
#ifdef TDCT_JAM_STAGES
  return TDCT_JAM_STAGES;
#else
  return 2;
#endif
}

// Block groups per warp iteration: at 16x16 u8 blocks two amortise the
// ring, geometry and loop work of an iteration over twice the blocks (2 %
// faster); at 32x32 the registers of a second group cost resident warps (4 %
// slower), and int16 residuals (64-bit row inverse) keep one as well.
template <int B, int DT>
constexpr int jam_groups() {
#ifdef TDCT_JAM_GROUPS
  return TDCT_JAM_GROUPS;
#else
  return (B == 16 && DT == 0) ? 2 : 1;
#endif
}

template <int B, int DT, int KE>
cudaError_t launch_b(const PlaneDesc& P, const JamParams& jp, unsigned long long* sse,
                     cudaStream_t s) {
  constexpr int PF = jam_stages<B, DT>();
  constexpr int NP = jam_groups<B, DT>();
  constexpr int kThreads = 128;
  constexpr size_t kRing =
      (size_t)(kThreads / 32) * PF * NP * 32 * (RowRaw<B, DT>::kWords * 16 + 8);
  auto kern = jam_codec_kernel<B, DT, KE, PF, NP>;
  static int resident = 0, sms = 0;
  if (resident == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRing);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, kern, kThreads, kRing);
    if (e != cudaSuccess) return e;
    if (resident < 1) resident = 1;
    sms = device_sms();
  }
  const int64_t nb = (int64_t)((P.W + B - 1) / B) * ((P.H + B - 1) / B);
  const int64_t warps = (nb + (32 / B) * NP - 1) / ((32 / B) * NP);
  int64_t grid = (warps + kThreads / 32 - 1) / (kThreads / 32);
  if (grid > (int64_t)resident * sms) grid = (int64_t)resident * sms;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, kThreads, kRing, s>>>(P, jp, sse);
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
  // the kernel steps block indices in 32-bit integers
  if (B > 0 && (int64_t)((P.W + B - 1) / B) * ((P.H + B - 1) / B) >= ((int64_t)1 << 30))
    return cudaErrorInvalidValue;
  if (B == 16)
    return P.dtype == 0 ? launch_ke<16, 0>(ke, P, jp, sse, s) : launch_ke<16, 1>(ke, P, jp, sse, s);
  if (B == 32)
    return P.dtype == 0 ? launch_ke<32, 0>(ke, P, jp, sse, s) : launch_ke<32, 1>(ke, P, jp, sse, s);
  return cudaErrorInvalidValue;
}

}  // namespace tdct
