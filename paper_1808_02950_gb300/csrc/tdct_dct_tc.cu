// tdct_dct_tc.cu -- the exact-DCT comparison codec in BF16 on the tensor cores.
//
// The codec of §6.1 with the orthonormal DCT-II of §2 as two GEMMs per tile of
// 128 blocks (tcgen05.mma .kind::f16 with bf16 operands and FP32
// accumulation in tensor memory):
//
//   Y = A1 B1^T   A1: 128 x 64, row m = the 64 samples of block m (bf16,
//                     exact for 0..255);
//                 B1: N1 x 64, row n = C_i kron C_j (the weights
//                     C_i[k] C_j[l], rounded once to bf16) of the n-th kept
//                     coefficient (i, j) -- zig-zag order, zero rows from r on;
//   X' = A2 B2^T  A2: 128 x (N1 + 16), row m = Y of block m rounded to bf16,
//                     then the constant 1 (the bias column);
//                 B2: 64 x (N1 + 16), row p = (k, l): the same weights for
//                     the kept coefficients, then 1/2 in the bias column.
//
// so X' = C^T Y' C + 1/2 and the reconstructed sample is floor(X') clamped to
// [0, 255] (round half away from zero for u8).  The CUDA cores convert the
// samples to bf16, the FP32 coefficients to bf16 between the GEMMs, and run
// the epilogue (floor by the bit pattern of X' + 1.5 * 2^23 rounded toward
// -inf, two samples per FADD2; packed clamp; byte SSE; 8-byte stores).
// When the coefficients are requested, B1 holds all 64 weights in raster
// order, Y goes to d_coef, and the unkept coefficients are zeroed in A2.
//
// FP32-level accuracy (SPLIT = 3): B1 holds three bf16 terms of each weight
// (w = w1 + w2 + w3 to about 2^-24) and GEMM 1 runs three K = 64 passes into
// the same accumulator; A2 holds two bf16 terms of each coefficient
// (Y = y1 + y2 to about 2^-17) and GEMM 2 sums y1 w1 + y2 w1 + y1 w2 + 1/2
// (K slices of A2 = [y1 | y2 | bias] against B2 = [w1 | w2 | 1/2]).
//
// N1 = 16 ceil(r / 16).  One CTA of 128 threads per tile (thread t = row t =
// block t of the tile), 4 CTAs per SM, persistent over tiles; the samples of
// the next tile are loaded into registers while the GEMMs of the current one
// run.  Operands use the canonical no-swizzle K-major layout: element
// (row, k) of an R-row operand at byte (k / 8) (R 16) + 16 row + 2 (k % 8).
// Tensor memory: D1 in columns [0, N1), D2 in [64, 128).  Every mbarrier wait
// is bounded: one that gives up records TDCT_ETIMEOUT in the status word and
// the CTA leaves after releasing its tensor memory.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "tdct_dct_tc.h"
#include "tdct_tcgen05.cuh"

namespace tdct {

namespace {

constexpr int kDtThreads = 128;
constexpr int kDtTables = 65;  // r = 1..64 (zig-zag), raster (coefficients)

// K extent of A2 / B2: the coefficient terms, then one 16-wide bias slice.
__host__ __device__ constexpr int dt_k2(int N1, int SPLIT) {
  return (SPLIT == 1 ? N1 : 2 * N1) + 16;
}
// B1 (SPLIT x N1 x 64) + B2 (64 x K2) elements at the largest N1 = 64.
__host__ __device__ constexpr int dt_table_elems(int SPLIT) {
  return SPLIT * 64 * 64 + 64 * dt_k2(64, SPLIT) + 128;  // + 64 float offsets
}

// The weight tables of every r in the operand layout, built once per device.
__device__ __align__(16) uint16_t g_dct_tc_b[kDtTables][dt_table_elems(1)];
__device__ __align__(16) uint16_t g_dct_tc_b3[kDtTables][dt_table_elems(3)];

__host__ __device__ constexpr int dt_n1(int r) { return 16 * ((r + 15) / 16); }

// (row, k) -> element offset in the no-swizzle K-major layout of an R-row operand.
__host__ __device__ constexpr int kmajor(int R, int row, int k) {
  return (k / 8) * (R * 8) + row * 8 + (k % 8);
}

// Two floats -> packed bf16x2 (x in the low half), round to nearest even.
__device__ __forceinline__ uint32_t pack_bf16x2(float x, float y) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(y), "f"(x));
  return d;
}

// Eight u8 samples (one block row) -> eight bf16 (exact): each byte becomes
// the float 2^23 + x minus 2^23 (two at a time), whose upper half is its bf16.
__device__ __forceinline__ uint4 row_to_bf16(uint2 w) {
  uint32_t o[4];
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const uint32_t word = h < 2 ? w.x : w.y;
    const int b0 = 2 * (h & 1);
    const float2 f = __fadd2_rn(
        make_float2(__uint_as_float(__byte_perm(word, 0x4B000000u, 0x7650u + b0)),
                    __uint_as_float(__byte_perm(word, 0x4B000000u, 0x7650u + b0 + 1))),
        make_float2(-8388608.0f, -8388608.0f));
    o[h] = __byte_perm(__float_as_uint(f.x), __float_as_uint(f.y), 0x7632u);
  }
  return make_uint4(o[0], o[1], o[2], o[3]);
}

// Eight u8 samples (one block row) -> eight fp16 1024 + x (exact: fp16 has
// unit spacing on [1024, 2048)), one byte permute per two samples.
__device__ __forceinline__ uint4 row_to_f16_biased(uint2 w) {
  return make_uint4(__byte_perm(w.x, 0x64646464u, 0x4140u), __byte_perm(w.x, 0x64646464u, 0x4342u),
                    __byte_perm(w.y, 0x64646464u, 0x4140u), __byte_perm(w.y, 0x64646464u, 0x4342u));
}

template <int N1, bool COEF, int SPLIT>
__global__ void __launch_bounds__(kDtThreads, 4)
    dct_tc_kernel(const PlaneDesc P, const uint16_t* __restrict__ btab, uint64_t kept_mask,
                  float* __restrict__ coef, int* __restrict__ status, long long wait_limit,
                  unsigned long long* __restrict__ sse_out) {
  constexpr int K2 = dt_k2(N1, SPLIT);
  constexpr int KB = K2 - 16;  // K index of the bias column
  constexpr int A1_BYTES = 128 * 64 * 2, A2_BYTES = 128 * K2 * 2;
  constexpr int B1_BYTES = SPLIT * N1 * 64 * 2, B2_BYTES = 64 * K2 * 2;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* a1 = smem;
  uint8_t* a2 = a1 + A1_BYTES;
  uint8_t* b1 = a2 + A2_BYTES;
  uint8_t* b2 = b1 + B1_BYTES;
  float* off = reinterpret_cast<float*>(b2 + B2_BYTES);  // 64 offsets 1024 sum_p w_np (SPLIT 1)
  uint64_t* bar = reinterpret_cast<uint64_t*>(off + 64);   // [0] GEMM 1, [1] GEMM 2
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 2);

  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tmem_slot)),
                 "r"(128u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    mbar_init(smem_addr(bar), 1);
    mbar_init(smem_addr(bar + 1), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // weights (and the offsets), once per CTA
  for (int e = t; e < (B1_BYTES + B2_BYTES + 256) / 16; e += kDtThreads)
    reinterpret_cast<uint4*>(b1)[e] = __ldg(reinterpret_cast<const uint4*>(btab) + e);
  // the bias column of A2 (K index KB = 1.0, the rest of its slice 0)
  {
    uint16_t* a2e = reinterpret_cast<uint16_t*>(a2);
#pragma unroll
    for (int k = KB; k < K2; ++k) a2e[kmajor(128, t, k)] = k == KB ? 0x3F80u : 0u;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t trow = tmem + ((uint32_t)(wid * 32) << 16);
  const uint32_t a1s = smem_addr(a1), a2s = smem_addr(a2), b1s = smem_addr(b1),
                 b2s = smem_addr(b2);
  const uint32_t bar1 = smem_addr(bar), bar2 = smem_addr(bar + 1);

  const int64_t nb = (int64_t)P.nbx * P.nby;
  const int64_t tiles = (nb + 127) / 128;
  const bool vec = (P.vec16 & 1) != 0, vec_out = P.recon && (P.vec16 & 2);

  // the 8 rows of block b (zero outside the plane)
  auto load_rows = [&](int64_t b, uint2 (&rw)[8]) {
#pragma unroll
    for (int k = 0; k < 8; ++k) rw[k] = make_uint2(0u, 0u);
    if (b >= nb) return;
    const int by = (int)(b / P.nbx), bx = (int)(b - (int64_t)by * P.nbx);
    const uint8_t* base = P.img + (int64_t)(by * 8) * P.pitch + (int64_t)bx * 8;
    const int vr = min(8, P.H - by * 8), vc = min(8, P.W - bx * 8);
    if (vr == 8 && vc == 8 && vec) {
#pragma unroll
      for (int k = 0; k < 8; ++k) rw[k] = __ldg(reinterpret_cast<const uint2*>(base + k * P.pitch));
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        uint8_t v[8];
#pragma unroll
        for (int l = 0; l < 8; ++l) v[l] = (k < vr && l < vc) ? __ldg(base + k * P.pitch + l) : 0;
        rw[k] = *reinterpret_cast<const uint2*>(v);
      }
    }
  };

  unsigned long long acc = 0;
  uint32_t phase = 0;
  uint2 rw[8];
  int64_t tile = blockIdx.x;
  load_rows(tile * 128 + t, rw);
  for (; tile < tiles; tile += gridDim.x) {
    const int64_t b = tile * 128 + t;
    // A1 row t: chunk k = row k of the block (SPLIT 1: fp16 1024 + x; the
    // bf16 weights are exact in fp16, and the offset 1024 sum_p w_np of each
    // coefficient is subtracted after the read-back)
#pragma unroll
    for (int k = 0; k < 8; ++k)
      *reinterpret_cast<uint4*>(a1 + k * 2048 + t * 16) =
          SPLIT == 1 ? row_to_f16_biased(rw[k]) : row_to_bf16(rw[k]);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
#pragma unroll
      for (int w = 0; w < SPLIT; ++w)  // the weight terms, one K = 64 pass each
#pragma unroll
        for (int q = 0; q < 4; ++q)
          mma_f16(tmem, smem_desc(a1s + 2 * q * 2048, 2048, 128),
                  smem_desc(b1s + w * (N1 * 128) + 2 * q * (N1 * 16), N1 * 16, 128),
                  SPLIT == 1 ? idesc_f16(128, N1) : idesc_bf16(128, N1),
                  (w > 0 || q > 0) ? 1u : 0u);
      mma_commit(bar1);
    }
    // the samples of this block stay in x, the next tile's load is in flight
    uint2 x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = rw[k];
    load_rows(b + (int64_t)gridDim.x * 128, rw);
    bool ok = __syncthreads_and(mbar_wait_sleep_bounded(bar1, phase, wait_limit));
    if (!ok) {
      if (t == 0 && status) atomicExch(status, 4 /* TDCT_ETIMEOUT */);
      break;
    }
    tc_fence_after();
    // Y of this block -> bf16 -> A2 row t (and the coefficients, if requested)
    {
      uint32_t y[N1];
#pragma unroll
      for (int g = 0; g < N1 / 16; ++g) tmem_ld16(trow + 16 * g, y + 16 * g);
      tmem_wait_ld();
      if constexpr (SPLIT == 1) {
#pragma unroll
        for (int n = 0; n < N1; n += 2) {
          const float2 o = *reinterpret_cast<const float2*>(off + n);
          const float2 v = __fadd2_rn(make_float2(__uint_as_float(y[n]), __uint_as_float(y[n + 1])),
                                      make_float2(-o.x, -o.y));
          y[n] = __float_as_uint(v.x);
          y[n + 1] = __float_as_uint(v.y);
        }
      }
      if constexpr (COEF) {
        if (b < nb) {
          if ((reinterpret_cast<uintptr_t>(coef) & 15) == 0) {
            float4* dst = reinterpret_cast<float4*>(coef + b * 64);
#pragma unroll
            for (int g = 0; g < 16; ++g)
              dst[g] = make_float4(__uint_as_float(y[4 * g]), __uint_as_float(y[4 * g + 1]),
                                   __uint_as_float(y[4 * g + 2]), __uint_as_float(y[4 * g + 3]));
          } else {
#pragma unroll
            for (int n = 0; n < 64; ++n) coef[b * 64 + n] = __uint_as_float(y[n]);
          }
        }
#pragma unroll
        for (int n = 0; n < N1; ++n)
          if (!((kept_mask >> n) & 1ull)) y[n] = 0u;
      }
#pragma unroll
      for (int c = 0; c < N1 / 8; ++c) {
        uint32_t hi[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
          hi[e] = pack_bf16x2(__uint_as_float(y[8 * c + 2 * e]), __uint_as_float(y[8 * c + 2 * e + 1]));
        *reinterpret_cast<uint4*>(a2 + c * 2048 + t * 16) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        if constexpr (SPLIT == 3) {
          // y2 = bf16(Y - y1); Y - y1 is exact in FP32 (y1 is Y to 8 bits)
          uint32_t lo[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float2 d = __fadd2_rn(
                make_float2(__uint_as_float(y[8 * c + 2 * e]), __uint_as_float(y[8 * c + 2 * e + 1])),
                make_float2(-__uint_as_float(hi[e] << 16), -__uint_as_float(hi[e] & 0xffff0000u)));
            lo[e] = pack_bf16x2(d.x, d.y);
          }
          *reinterpret_cast<uint4*>(a2 + (N1 / 8 + c) * 2048 + t * 16) =
              make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
      // (A2 K slice, B2 K slice) pairs in 16-wide slices: SPLIT 1: y w + bias;
      // SPLIT 3: y1 w1, y2 w1, y1 w2, bias
      constexpr int S = N1 / 16;
      int n = 0;
      auto slice = [&](int sa, int sb) {
        mma_f16(tmem + 64, smem_desc(a2s + 2 * sa * 2048, 2048, 128),
                smem_desc(b2s + 2 * sb * (64 * 16), 64 * 16, 128), idesc_bf16(128, 64),
                n++ > 0 ? 1u : 0u);
      };
#pragma unroll
      for (int q = 0; q < S; ++q) slice(q, q);
      if constexpr (SPLIT == 3) {
#pragma unroll
        for (int q = 0; q < S; ++q) slice(S + q, q);
#pragma unroll
        for (int q = 0; q < S; ++q) slice(q, S + q);
      }
      slice(K2 / 16 - 1, K2 / 16 - 1);  // the bias
      mma_commit(bar2);
    }
    ok = __syncthreads_and(mbar_wait_sleep_bounded(bar2, phase, wait_limit));
    phase ^= 1u;
    if (!ok) {
      if (t == 0 && status) atomicExch(status, 4 /* TDCT_ETIMEOUT */);
      break;
    }
    tc_fence_after();
    // X' + 1/2 of this block, row by row: floor, clamp, SSE, store.  The
    // tensor-memory loads are warp-collective (.sync.aligned): every lane
    // executes them, also the lanes whose block lies past the plane's end.
    {
      const bool has = b < nb;
      const int by = has ? (int)(b / P.nbx) : 0, bx = has ? (int)(b - (int64_t)by * P.nbx) : 0;
      const int vr = min(8, P.H - by * 8), vc = min(8, P.W - bx * 8);
      const bool full = vr == 8 && vc == 8;
      uint8_t* out = (P.recon && has)
                         ? P.recon + (int64_t)(by * 8) * P.recon_pitch + (int64_t)bx * 8
                         : nullptr;
      uint32_t sse = 0;
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        uint32_t v[16];
        tmem_ld16(trow + 64 + 16 * h, v);
        tmem_wait_ld();
        if (!has) continue;
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
          const int k = 2 * h + rr;
          uint32_t f[8];
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const float2 s = __fadd2_rd(make_float2(__uint_as_float(v[8 * rr + 2 * m]),
                                                    __uint_as_float(v[8 * rr + 2 * m + 1])),
                                        make_float2(12582912.0f, 12582912.0f));
            f[2 * m] = __float_as_uint(s.x);
            f[2 * m + 1] = __float_as_uint(s.y);
          }
          const uint32_t c01 = min_relu_s16x2(__byte_perm(f[0], f[1], 0x5410u), 0x00ff00ffu);
          const uint32_t c23 = min_relu_s16x2(__byte_perm(f[2], f[3], 0x5410u), 0x00ff00ffu);
          const uint32_t c45 = min_relu_s16x2(__byte_perm(f[4], f[5], 0x5410u), 0x00ff00ffu);
          const uint32_t c67 = min_relu_s16x2(__byte_perm(f[6], f[7], 0x5410u), 0x00ff00ffu);
          uint2 yk = make_uint2(__byte_perm(c01, c23, 0x6420u), __byte_perm(c45, c67, 0x6420u));
          if (!full) {
            const uint64_t m = k < vr ? (vc >= 8 ? ~0ull : ((1ull << (8 * vc)) - 1ull)) : 0ull;
            yk.x = (yk.x & (uint32_t)m) | (x[k].x & ~(uint32_t)m);
            yk.y = (yk.y & (uint32_t)(m >> 32)) | (x[k].y & ~(uint32_t)(m >> 32));
          }
          const uint32_t d0 = __vabsdiffu4(x[k].x, yk.x), d1 = __vabsdiffu4(x[k].y, yk.y);
          sse = __dp4a(d0, d0, __dp4a(d1, d1, sse));
          if (out) {
            if (full && vec_out) {
              *reinterpret_cast<uint2*>(out + (int64_t)k * P.recon_pitch) = yk;
            } else if (k < vr) {
#pragma unroll
              for (int l = 0; l < 8; ++l)
                if (l < vc)
                  out[(int64_t)k * P.recon_pitch + l] =
                      (uint8_t)(((l < 4 ? yk.x : yk.y) >> (8 * (l & 3))) & 0xffu);
            }
          }
        }
      }
      acc += sse;
    }
    tc_fence_before();
    __syncthreads();  // A1, A2 and the accumulators are free for the next tile
  }
  acc = warp_sum_u64(acc);
  if (lane == 0 && acc) atomicAdd(sse_out, acc);
  tc_fence_before();
  __syncthreads();
  if (wid == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u)
                 : "memory");
  }
}

float bf16_round(double v) {
  // the float, then round to nearest even on its upper 16 bits (finite values)
  float f = (float)v;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7fffu + ((u >> 16) & 1u);
  u &= 0xffff0000u;
  std::memcpy(&f, &u, 4);
  return f;
}

// fp16 bits of a value that fp16 represents exactly (a bf16-rounded weight:
// 8 significant bits, magnitude in [2^-14, 2^15)); 0 for 0.
uint16_t f16_bits_exact(double v) {
  if (v == 0.0) return 0;
  const uint16_t sign = v < 0 ? 0x8000u : 0u;
  double a = std::fabs(v);
  int e = 0;
  const double m = std::frexp(a, &e);  // a = m 2^e, m in [0.5, 1)
  const int E = e - 1 + 15;            // biased exponent of 1.f x 2^(e-1)
  const uint32_t frac = (uint32_t)std::lround((m * 2.0 - 1.0) * 1024.0);
  return (uint16_t)(sign | ((uint32_t)E << 10) | frac);
}

uint16_t bf16_bits(double v) {
  const float f = bf16_round(v);
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return (uint16_t)(u >> 16);
}

// The weight tables of table index `ti` (0..63: r = ti + 1 in zig-zag order;
// 64: all 64 coefficients in raster order), in the operand layout, with
// SPLIT bf16 terms of each weight in B1 (w1, w2 = bf16(w - w1), ...) and,
// for SPLIT 3, B2 = [w1 | w2 | 1/2].
void build_table(int ti, int SPLIT, uint16_t* out) {
  double C[8][8];
  for (int k = 0; k < 8; ++k)
    for (int j = 0; j < 8; ++j)
      C[k][j] = (k == 0 ? std::sqrt(1.0 / 8.0) : std::sqrt(2.0 / 8.0)) *
                std::cos(M_PI * (2.0 * j + 1.0) * k / 16.0);
  const bool raster = ti == 64;
  const int r = raster ? 64 : ti + 1;
  const int N1 = raster ? 64 : dt_n1(r), K2 = dt_k2(N1, SPLIT), KB = K2 - 16;
  int pos[64];  // column n -> position i * 8 + j
  for (int n = 0; n < 64; ++n) pos[n] = n;
  if (!raster)
    for (int i = 0; i < 8; ++i)
      for (int j = 0; j < 8; ++j) pos[zz_index(i, j)] = 8 * i + j;
  std::memset(out, 0, sizeof(uint16_t) * dt_table_elems(SPLIT));
  uint16_t* B1 = out;
  uint16_t* B2 = out + SPLIT * N1 * 64;
  double off64[64] = {};  // SPLIT 1: 1024 sum_p w_np (GEMM 1 takes the samples as 1024 + x)
  for (int n = 0; n < N1; ++n) {
    if (n >= r) continue;
    const int i = pos[n] / 8, j = pos[n] % 8;
    for (int k = 0; k < 8; ++k)
      for (int l = 0; l < 8; ++l) {
        double rest = C[i][k] * C[j][l];
        for (int w = 0; w < SPLIT; ++w) {
          const double term = bf16_round(rest);
          // SPLIT 1: the bf16 weight re-encoded exactly as fp16 for GEMM 1
          B1[w * N1 * 64 + kmajor(N1, n, 8 * k + l)] =
              SPLIT == 1 ? f16_bits_exact(term) : bf16_bits(term);
          if (SPLIT == 1) off64[n] += 1024.0 * term;
          if (w == 0) B2[kmajor(64, 8 * k + l, n)] = bf16_bits(term);
          if (w == 1 && SPLIT == 3) B2[kmajor(64, 8 * k + l, N1 + n)] = bf16_bits(term);
          rest -= term;
        }
      }
  }
  for (int p = 0; p < 64; ++p) B2[kmajor(64, p, KB)] = 0x3F00u;  // 1/2
  float off[64];
  for (int n = 0; n < 64; ++n) off[n] = (float)off64[n];
  std::memcpy(B2 + 64 * K2, off, sizeof off);
}

template <int N1, bool COEF, int SPLIT>
cudaError_t launch_one(const PlaneDesc& P, const uint16_t* tab, uint64_t kept_mask, float* coef,
                       int* status, unsigned long long* sse, cudaStream_t s) {
  constexpr int K2 = dt_k2(N1, SPLIT);
  // at least 56 KB of shared memory per CTA: then at most 4 CTAs share an SM,
  // whose 512 tensor-memory columns hold exactly 4 allocations of 128
  constexpr size_t kUsed =
      128 * 64 * 2 + 128 * K2 * 2 + SPLIT * N1 * 64 * 2 + 64 * K2 * 2 + 256 + 64;
  constexpr size_t kSmem = kUsed < 56 * 1024 ? 56 * 1024 : kUsed;
  static int sms = 0, per_sm = 0;
  if (sms == 0) {
    const cudaError_t e = cudaFuncSetAttribute(dct_tc_kernel<N1, COEF, SPLIT>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kSmem);
    if (e != cudaSuccess) return e;
    sms = device_sms();
    int dev = 0, smem_sm = 233472, reserved = 1024;
    if (cudaGetDevice(&dev) == cudaSuccess) {
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    }
    per_sm = (int)(smem_sm / (kSmem + reserved));
    if (per_sm > 4) per_sm = 4;
    if (per_sm < 1) per_sm = 1;
  }
  const int64_t tiles = ((int64_t)P.nbx * P.nby + 127) / 128;
  // at most 4 CTAs of 128 tensor-memory columns per SM (its 512 columns)
  int64_t grid = (int64_t)per_sm * sms;
  if (grid > tiles) grid = tiles;
  if (grid < 1) grid = 1;
  dct_tc_kernel<N1, COEF, SPLIT><<<(unsigned)grid, kDtThreads, kSmem, s>>>(
      P, tab, kept_mask, coef, status, 2000000000ll, sse);
  return cudaGetLastError();
}

}  // namespace

cudaError_t dct_tc_prepare(int split, const uint16_t** tables) {
  static std::mutex mu;
  static void* addr[2][256] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256 || (split != 1 && split != 3)) return cudaErrorInvalidValue;
  const int si = split == 3 ? 1 : 0;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[si][dev]) {
    const int elems = dt_table_elems(split);
    std::vector<uint16_t> host((size_t)kDtTables * elems);
    for (int ti = 0; ti < kDtTables; ++ti) build_table(ti, split, host.data() + (size_t)ti * elems);
    void* p = nullptr;
    if (split == 3) {
      e = cudaMemcpyToSymbol(g_dct_tc_b3, host.data(), host.size() * sizeof(uint16_t));
      if (e == cudaSuccess) e = cudaGetSymbolAddress(&p, g_dct_tc_b3);
    } else {
      e = cudaMemcpyToSymbol(g_dct_tc_b, host.data(), host.size() * sizeof(uint16_t));
      if (e == cudaSuccess) e = cudaGetSymbolAddress(&p, g_dct_tc_b);
    }
    if (e != cudaSuccess) return e;
    addr[si][dev] = p;
  }
  *tables = static_cast<const uint16_t*>(addr[si][dev]);
  return cudaSuccess;
}

namespace {
template <int SPLIT>
cudaError_t launch_split(const PlaneDesc& P, float* coef, int* status, unsigned long long* sse,
                         cudaStream_t s) {
  const uint16_t* all = nullptr;
  cudaError_t e = dct_tc_prepare(SPLIT, &all);
  if (e != cudaSuccess) return e;
  const int r = P.r;
  const size_t elems = (size_t)dt_table_elems(SPLIT);
  uint64_t kept_mask = 0;
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j)
      if (kept(r, i, j)) kept_mask |= 1ull << (8 * i + j);
  if (coef)
    return launch_one<64, true, SPLIT>(P, all + 64 * elems, kept_mask, coef, status, sse, s);
  const uint16_t* tab = all + (size_t)(r - 1) * elems;
  switch (dt_n1(r)) {
    case 16: return launch_one<16, false, SPLIT>(P, tab, 0, nullptr, status, sse, s);
    case 32: return launch_one<32, false, SPLIT>(P, tab, 0, nullptr, status, sse, s);
    case 48: return launch_one<48, false, SPLIT>(P, tab, 0, nullptr, status, sse, s);
    default: return launch_one<64, false, SPLIT>(P, tab, 0, nullptr, status, sse, s);
  }
}
}  // namespace

cudaError_t launch_dct_tc(const PlaneDesc& P, int split, float* coef, int* status,
                          unsigned long long* sse, cudaStream_t s) {
  return split == 3 ? launch_split<3>(P, coef, status, sse, s)
                    : launch_split<1>(P, coef, status, sse, s);
}

}  // namespace tdct
