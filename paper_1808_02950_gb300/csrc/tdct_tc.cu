// tdct_tc.cu -- the forward transform on the 5th-generation tensor cores.
//
// For u8 planes the integer coefficients Z = T1 X T1^T of the kept zig-zag
// positions are a linear map of the 64 pixels with weights
// (t_i kron t_j)[k][l] in {0, +-1, +-2, +-4}.  sm_103a has no int8 MMA
// (tcgen05.mma .kind::i8 is rejected for this target), so the GEMM runs as
// .kind::f16 with exact integer arithmetic: each pixel enters as the fp16
// value 1024 + x (exact: fp16 has unit spacing on [1024, 2048)), the weights
// are exact in fp16, every product and partial sum is an integer below 2^20
// and is therefore exact in the FP32 accumulator.  The bias contributes
// 1024 * sum(weights) = 65536 to Z_00 and nothing elsewhere (the other rows of
// T1 sum to zero); it is subtracted after the read-back.
//
// Tile = 4 units = 128 lane pairs = 256 blocks, one CTA of 4 warps:
//   A (M = 128 rows, K = 128 fp16): row m = the block pair of lane m % 32 of
//     unit m / 32; K-chunk ch = 2 k + h (8 elements) = row k of block h.
//   B (NH rows, K = 64): row n = the weights of kept coefficient n.
//   Two MMAs per tile, one per block h of the pairs: A restricted to the
//     K-chunks 2k + h (4096 B apart) times B gives D_h = the coefficients of
//     block h (M x NH, FP32) in tensor-memory columns [h NH, h NH + NH);
//     tcgen05.ld gives each lane its pair's 2 NH coefficients.  Scaling, inverse, rounding and the error run
//     on the CUDA cores exactly as in the butterfly path.
// Shared memory uses the canonical no-swizzle K-major UMMA layout: core
// matrices of 8 rows x 16 bytes with rows 16 B apart; 8-row groups 128 B
// apart (SBO); K-chunks of one block 4096 B apart for A and NH * 16 B apart
// for B (LBO).
// CTAs are persistent over tiles; tensor memory is allocated once per CTA
// (at most 128 columns, 4 CTAs per SM) and released on every exit path.
// Every mbarrier wait is bounded and records TDCT_ETIMEOUT when it gives up.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "tdct_classes.h"
#include "tdct_kernels.cuh"
#include "tdct_tc.h"
#include "tdct_tcgen05.cuh"

namespace tdct {

namespace {

constexpr int kTcThreads = 128;
constexpr int kATileBytes = 16 * 2048;  // 16 K-chunks x 128 rows x 16 bytes

// Columns per block (a valid N of an M = 128 MMA: a multiple of 16).
__host__ __device__ constexpr int nh_of(int R) { return R <= 16 ? 16 : (R <= 32 ? 32 : 64); }
__host__ __device__ constexpr int tmem_cols_of(int N) { return N < 32 ? 32 : N; }

// fp16 pair (1024 + a, 1024 + b) from bytes of w selected by `sel`.
__device__ __forceinline__ uint32_t biased_f16x2(uint32_t w, uint32_t sel) {
  return __byte_perm(w, 0x64646464u, sel);
}

// CTAs per SM each tensor kernel is compiled for (128 or 168 registers per
// thread; measured): the one-tile kernel keeps 4 up to class 16, the
// pipelined kernel and the larger classes run faster without spills at 3.
// The launcher derives the actual residency from the compiled kernel.
template <int R, bool PIPE>
__host__ __device__ constexpr int tc_min_blocks() {
#ifdef TDCT_TC_MINB
  return TDCT_TC_MINB;
#else
  return (PIPE || R > 16) ? 3 : 4;
#endif
}

template <int R>
__global__ void __launch_bounds__(kTcThreads, tc_min_blocks<R, false>())
    codec_u8_tc_kernel(const PlaneTable tab, const CodecParams cp,
                       const uint16_t* __restrict__ b_global,
                       unsigned long long* __restrict__ sse_out) {
  constexpr int NH = nh_of(R);
  constexpr int N = 2 * NH;
  constexpr int COLS = tmem_cols_of(N);
  constexpr int B_BYTES = NH * 128;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* a_tile = smem;                          // 32 KB fp16 A operand
  uint8_t* raw_all = smem + kATileBytes;           // 4 warps x 8 rows x 512 B
  uint8_t* b_mat = raw_all + 4 * kUnitBytes;       // NH x 64 fp16
  uint64_t* bar = reinterpret_cast<uint64_t*>(b_mat + B_BYTES);  // [0] mma, [1..4] raw
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 5);

  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  const uint32_t bar_mma = smem_addr(bar);
  const uint32_t bar_raw = smem_addr(bar + 1 + wid);
  uint8_t* raw = raw_all + wid * kUnitBytes;

  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tmem_slot)),
                 "r"((uint32_t)COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    mbar_init(bar_mma, 1);
    for (int w = 0; w < 4; ++w) mbar_init(smem_addr(bar + 1 + w), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // B once per CTA (L2-resident table built per r)
  for (int e = threadIdx.x; e < B_BYTES / 16; e += kTcThreads)
    reinterpret_cast<uint4*>(b_mat)[e] = __ldg(reinterpret_cast<const uint4*>(b_global) + e);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t trow = tmem + ((uint32_t)(wid * 32) << 16);
  const uint32_t a0 = smem_addr(a_tile), b0 = smem_addr(b_mat);
  constexpr uint32_t idesc = idesc_f16(128, NH);

  const int64_t tiles = (tab.total_units + 3) / 4;
  const int64_t t_begin = (tiles * blockIdx.x) / gridDim.x;
  const int64_t t_end = (tiles * (blockIdx.x + 1)) / gridDim.x;

  // Prefetch of this warp's unit of tile t into `raw` (8 bulk row copies).
  int64_t pf_end = -1, pf_ubegin = 0, pf_pitch = 0;
  const uint8_t* pf_img = nullptr;
  int pf_W = 0, pf_chunks = 1;
  uint32_t raw_phase = 0;
  auto prefetch = [&](int64_t t) -> bool {
    const int64_t u = t * 4 + wid;
    if (t >= t_end || u >= tab.total_units) return false;
    if (u >= pf_end) {
      const int q = find_plane(tab, u);
      const PlaneDesc& Q = tab.d ? tab.d[q] : tab.one;
      pf_img = Q.img;
      pf_pitch = Q.pitch;
      pf_W = Q.W;
      pf_chunks = Q.chunks;
      pf_ubegin = Q.unit_begin;
      pf_end = (q + 1 < tab.n) ? tab.d[q + 1].unit_begin : tab.total_units;
    }
    const int64_t local = u - pf_ubegin;
    const int by = (int)(local / pf_chunks);
    const int chunk = (int)(local - (int64_t)by * pf_chunks);
    const uint32_t row_bytes = (uint32_t)min(512, pf_W - chunk * 512);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (lane == 0) mbar_arrive_expect_tx(bar_raw, 8u * row_bytes);
    __syncwarp();
    if (lane < 8) {
      const uint8_t* src = pf_img + (int64_t)(by * 8 + lane) * pf_pitch + (int64_t)chunk * 512;
      bulk_copy_g2s(smem_addr(raw + lane * 512), src, row_bytes, bar_raw);
    }
    return true;
  };
  bool in_flight = prefetch(t_begin);

  int p = -1;
  int64_t p_end = -1;
  PlaneDesc P;
  unsigned long long acc = 0;
  uint32_t phase = 0;
  for (int64_t t = t_begin; t < t_end; ++t) {
    const int64_t u = t * 4 + wid;
    const bool has_unit = u < tab.total_units;
    int by = 0, bx0 = 0;
    bool has_pair = false;
    if (has_unit) {
      if (u >= p_end) {
        if (p >= 0) {
          acc = warp_sum_u64(acc);
          if (lane == 0 && acc) atomicAdd(sse_out + P.slot, acc);
          acc = 0;
        }
        p = find_plane(tab, u);
        P = tab.d ? tab.d[p] : tab.one;
        p_end = (p + 1 < tab.n) ? tab.d[p + 1].unit_begin : tab.total_units;
      }
      const int64_t local = u - P.unit_begin;
      by = (int)(local / P.chunks);
      const int chunk = (int)(local - (int64_t)by * P.chunks);
      bx0 = chunk * 64 + 2 * lane;
      has_pair = bx0 < P.nbx;
    }
    // this warp's rows of tile t (in flight since the previous tile)
    bool ok = true;
    if (in_flight) {
      ok = __all_sync(0xffffffffu, mbar_wait_sleep_bounded(bar_raw, raw_phase, cp.wait_limit));
      raw_phase ^= 1u;
      in_flight = false;
    }
    uint4 rw[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
      rw[k] = (has_pair && ok) ? *reinterpret_cast<const uint4*>(raw + k * 512 + lane * 16)
                               : make_uint4(0u, 0u, 0u, 0u);
    __syncwarp();
    if (ok) in_flight = prefetch(t + 1);  // the next unit loads during this tile
    // A rows of this lane's pair: chunk 2k + h holds row k of block h
    uint8_t* arow = a_tile + (wid * 32 + lane) * 16;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint4 lo = make_uint4(biased_f16x2(rw[k].x, 0x4140u), biased_f16x2(rw[k].x, 0x4342u),
                                  biased_f16x2(rw[k].y, 0x4140u), biased_f16x2(rw[k].y, 0x4342u));
      const uint4 hi = make_uint4(biased_f16x2(rw[k].z, 0x4140u), biased_f16x2(rw[k].z, 0x4342u),
                                  biased_f16x2(rw[k].w, 0x4140u), biased_f16x2(rw[k].w, 0x4342u));
      *reinterpret_cast<uint4*>(arow + (2 * k) * 2048) = lo;
      *reinterpret_cast<uint4*>(arow + (2 * k + 1) * 2048) = hi;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    if (!__syncthreads_and(ok)) {  // a row copy did not arrive in time
      if (threadIdx.x == 0 && cp.status) atomicExch(cp.status, 4 /* TDCT_ETIMEOUT */);
      break;
    }
    // timeout test hook: CTA 0 never issues its first tile's MMAs
    const bool hook = cp.test_hook == 1 && blockIdx.x == 0 && t == t_begin;
    if (threadIdx.x == 0 && !hook) {
      tc_fence_after();
      // block h uses the K-chunks 2k + h (4096 B apart) and TMEM columns h NH
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint64_t ad = smem_desc(a0 + (4 * q + h) * 2048, 4096, 128);
          const uint64_t bd = smem_desc(b0 + q * 2 * (NH * 16), NH * 16, 128);
          mma_f16(tmem + h * NH, ad, bd, idesc, q > 0 ? 1u : 0u);
        }
      mma_commit(bar_mma);
    }
    // CTA-uniform decision: every thread waits (bounded), all agree
    const bool done = __syncthreads_and(mbar_wait_sleep_bounded(bar_mma, phase, cp.wait_limit));
    phase ^= 1u;
    if (!done) {
      if (threadIdx.x == 0 && cp.status) atomicExch(cp.status, 4 /* TDCT_ETIMEOUT */);
      break;
    }
    tc_fence_after();
    uint32_t zf[2][NH];
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int g = 0; g < NH / 8; ++g) tmem_ld8(trow + b * NH + 8 * g, zf[b] + 8 * g);
    tmem_wait_ld();
    tc_fence_before();
    __syncthreads();  // A tile and accumulator free for the next tile
    if (has_pair) {
      uint2 xa[8], xb[8];
      uint32_t sse = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        xa[k] = make_uint2(rw[k].x, rw[k].y);
        xb[k] = make_uint2(rw[k].z, rw[k].w);
#if !TDCT_SSE_ABSDIFF  // the epilogue's terms then need sum x^2
        sse = __dp4a(xa[k].x, xa[k].x, sse);
        sse = __dp4a(xa[k].y, xa[k].y, sse);
        sse = __dp4a(xb[k].x, xb[k].x, sse);
        sse = __dp4a(xb[k].y, xb[k].y, sse);
#endif
      }
      const bool store = P.recon != nullptr;
      const int64_t rp = P.recon_pitch;
      uint2* out0 = store ? reinterpret_cast<uint2*>(P.recon + (int64_t)(by * 8) * rp +
                                                     (int64_t)bx0 * 8)
                          : nullptr;
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        uint32_t w[64];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int pz = 8 * i + j;
            if (kept(R, i, j)) {
              int32_t z = __float2int_rn(__uint_as_float(zf[b][zz_index(i, j)]));
              if (pz == 0) z -= 65536;  // the 1024 bias of the 64 pixels
              w[pz] = (uint32_t)z * (uint32_t)cp.cmul2[pz];
            } else {
              w[pz] = 0u;
            }
          }
        w[0] += kL2;
        sse += inverse_epilogue_u8_any<R>(w, RowsInRegs{b == 0 ? xa : xb}, store ? out0 + b : nullptr, rp, store,
                                      true, 8, 8);
      }
      acc += sse;
    }
  }
  // drain a prefetch still in flight (bounded) before the shared memory goes
  if (in_flight) __all_sync(0xffffffffu, mbar_wait_sleep_bounded(bar_raw, raw_phase, cp.wait_limit));
  if (p >= 0) {
    acc = warp_sum_u64(acc);
    if (lane == 0 && acc) atomicAdd(sse_out + P.slot, acc);
  }
  tc_fence_before();
  __syncthreads();
  if (wid == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)COLS)
                 : "memory");
  }
}

// Software-pipelined variant: the MMA of tile t + 1 runs while tile t is
// computed.  Per iteration: wait for MMA(t) and read its accumulator (the A
// tile is then free), convert the prefetched rows of tile t + 1 into A,
// issue MMA(t + 1) into the other accumulator, then compute tile t, reading
// its pixels again from global memory (an L2 hit: they were fetched by the
// prefetch one tile earlier) instead of holding them in registers across
// the MMA.  Two tensor-memory accumulators of N columns, one mbarrier each.
template <int R>
__global__ void __launch_bounds__(kTcThreads, tc_min_blocks<R, true>())
    codec_u8_tc_pipe_kernel(const PlaneTable tab, const CodecParams cp,
                            const uint16_t* __restrict__ b_global,
                            unsigned long long* __restrict__ sse_out) {
  constexpr int NH = nh_of(R);
  constexpr int N = 2 * NH;
  constexpr int COLS = tmem_cols_of(2 * N);
  constexpr int B_BYTES = NH * 128;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* a_tile = smem;
  uint8_t* raw_all = smem + kATileBytes;  // [warp][8 rows x 512 B]
  uint8_t* b_mat = raw_all + 4 * kUnitBytes;
  uint64_t* bar = reinterpret_cast<uint64_t*>(b_mat + B_BYTES);  // [0,1] mma, [2..5] raw
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 6);

  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  uint8_t* raw = raw_all + wid * kUnitBytes;  // this warp's rows of the next tile
  const uint32_t bar_raw = smem_addr(bar + 2 + wid);

  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tmem_slot)),
                 "r"((uint32_t)COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < 6; ++i) mbar_init(smem_addr(bar + i), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int e = threadIdx.x; e < B_BYTES / 16; e += kTcThreads)
    reinterpret_cast<uint4*>(b_mat)[e] = __ldg(reinterpret_cast<const uint4*>(b_global) + e);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t trow = tmem + ((uint32_t)(wid * 32) << 16);
  const uint32_t a0 = smem_addr(a_tile), b0 = smem_addr(b_mat);
  constexpr uint32_t idesc = idesc_f16(128, NH);

  const int64_t tiles = (tab.total_units + 3) / 4;
  const int64_t t_begin = (tiles * blockIdx.x) / gridDim.x;
  const int64_t t_end = (tiles * (blockIdx.x + 1)) / gridDim.x;

  // prefetch cursor: this warp's unit of a tile -> its rows into its raw slot
  int64_t pf_end = -1, pf_ubegin = 0, pf_pitch = 0;
  const uint8_t* pf_img = nullptr;
  int pf_W = 0, pf_chunks = 1;
  uint32_t raw_phase = 0;
  auto prefetch = [&](int64_t t) -> bool {
    const int64_t u = t * 4 + wid;
    if (t >= t_end || u >= tab.total_units) return false;
    if (u >= pf_end) {
      const int q = find_plane(tab, u);
      const PlaneDesc& Q = tab.d ? tab.d[q] : tab.one;
      pf_img = Q.img;
      pf_pitch = Q.pitch;
      pf_W = Q.W;
      pf_chunks = Q.chunks;
      pf_ubegin = Q.unit_begin;
      pf_end = (q + 1 < tab.n) ? tab.d[q + 1].unit_begin : tab.total_units;
    }
    const int64_t local = u - pf_ubegin;
    const int by = (int)(local / pf_chunks);
    const int chunk = (int)(local - (int64_t)by * pf_chunks);
    const uint32_t row_bytes = (uint32_t)min(512, pf_W - chunk * 512);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (lane == 0) mbar_arrive_expect_tx(bar_raw, 8u * row_bytes);
    __syncwarp();
    if (lane < 8) {
      const uint8_t* src = pf_img + (int64_t)(by * 8 + lane) * pf_pitch + (int64_t)chunk * 512;
      bulk_copy_g2s(smem_addr(raw + lane * 512), src, row_bytes, bar_raw);
    }
    return true;
  };

  // Convert the rows in `raw` (the next tile) into A (bounded wait).
  bool in_flight = false;
  auto stage_tile = [&]() -> bool {
    bool ok = true;
    if (in_flight) {
      ok = __all_sync(0xffffffffu, mbar_wait_sleep_bounded(bar_raw, raw_phase, cp.wait_limit));
      raw_phase ^= 1u;
      in_flight = false;
    }
    uint4 rw[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) rw[k] = *reinterpret_cast<const uint4*>(raw + k * 512 + lane * 16);
    __syncwarp();
    uint8_t* arow = a_tile + (wid * 32 + lane) * 16;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint4 lo = make_uint4(biased_f16x2(rw[k].x, 0x4140u), biased_f16x2(rw[k].x, 0x4342u),
                                  biased_f16x2(rw[k].y, 0x4140u), biased_f16x2(rw[k].y, 0x4342u));
      const uint4 hi = make_uint4(biased_f16x2(rw[k].z, 0x4140u), biased_f16x2(rw[k].z, 0x4342u),
                                  biased_f16x2(rw[k].w, 0x4140u), biased_f16x2(rw[k].w, 0x4342u));
      *reinterpret_cast<uint4*>(arow + (2 * k) * 2048) = lo;
      *reinterpret_cast<uint4*>(arow + (2 * k + 1) * 2048) = hi;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    return ok;
  };
  auto issue_mma = [&](int buf, bool hook) {
    if (threadIdx.x == 0 && !hook) {
      tc_fence_after();
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint64_t ad = smem_desc(a0 + (4 * q + h) * 2048, 4096, 128);
          const uint64_t bd = smem_desc(b0 + q * 2 * (NH * 16), NH * 16, 128);
          mma_f16(tmem + buf * N + h * NH, ad, bd, idesc, q > 0 ? 1u : 0u);
        }
      mma_commit(smem_addr(bar + buf));
    }
  };

  uint32_t mma_phase = 0;  // bit b: parity of accumulator b's next completion
  bool mma_pending[2] = {false, false};
  bool alive = t_begin < t_end;
  if (alive) {
    in_flight = prefetch(t_begin);
    bool ok = stage_tile();
    if (ok) in_flight = prefetch(t_begin + 1);
    tc_fence_before();
    alive = __syncthreads_and(ok);
    if (alive) {
      issue_mma(0, cp.test_hook == 1 && blockIdx.x == 0);
      mma_pending[0] = true;
    } else if (threadIdx.x == 0 && cp.status) {
      atomicExch(cp.status, 4 /* TDCT_ETIMEOUT */);
    }
  }

  int p = -1;
  int64_t p_end = -1;
  PlaneDesc P;
  unsigned long long acc = 0;
  for (int64_t t = t_begin; t < t_end && alive; ++t) {
    const int b = (int)((t - t_begin) & 1);
    // accumulator of tile t
    // warp-uniform: stage_tile below contains warp-collective operations
    bool ok = __all_sync(0xffffffffu,
                         mbar_wait_sleep_bounded(smem_addr(bar + b), (mma_phase >> b) & 1u, cp.wait_limit));
    mma_phase ^= 1u << b;
    mma_pending[b] = false;
    tc_fence_after();
    uint32_t zf[2][NH];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int g = 0; g < NH / 8; ++g) tmem_ld8(trow + b * N + h * NH + 8 * g, zf[h] + 8 * g);
    tmem_wait_ld();
    // A is free: stage tile t + 1 and start its MMA before computing tile t
    const bool more = t + 1 < t_end;
    if (more && ok) {
      ok = stage_tile();
      if (ok) in_flight = prefetch(t + 2);
    }
    tc_fence_before();
    if (!__syncthreads_and(ok)) {
      if (threadIdx.x == 0 && cp.status) atomicExch(cp.status, 4 /* TDCT_ETIMEOUT */);
      alive = false;
      break;
    }
    if (more) {
      issue_mma(b ^ 1, false);
      mma_pending[b ^ 1] = true;
    }
    // compute tile t
    const int64_t u = t * 4 + wid;
    if (u < tab.total_units) {
      if (u >= p_end) {
        if (p >= 0) {
          acc = warp_sum_u64(acc);
          if (lane == 0 && acc) atomicAdd(sse_out + P.slot, acc);
          acc = 0;
        }
        p = find_plane(tab, u);
        P = tab.d ? tab.d[p] : tab.one;
        p_end = (p + 1 < tab.n) ? tab.d[p + 1].unit_begin : tab.total_units;
      }
      const int64_t local = u - P.unit_begin;
      const int by = (int)(local / P.chunks);
      const int chunk = (int)(local - (int64_t)by * P.chunks);
      const int bx0 = chunk * 64 + 2 * lane;
      if (bx0 < P.nbx) {
        const uint8_t* src = P.img + (int64_t)(by * 8) * P.pitch + (int64_t)bx0 * 8;
        uint2 xa[8], xb[8];
        uint32_t sse = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const uint4 v = __ldg(reinterpret_cast<const uint4*>(src + k * P.pitch));
          xa[k] = make_uint2(v.x, v.y);
          xb[k] = make_uint2(v.z, v.w);
#if !TDCT_SSE_ABSDIFF  // the epilogue's terms then need sum x^2
          sse = __dp4a(xa[k].x, xa[k].x, sse);
          sse = __dp4a(xa[k].y, xa[k].y, sse);
          sse = __dp4a(xb[k].x, xb[k].x, sse);
          sse = __dp4a(xb[k].y, xb[k].y, sse);
#endif
        }
        const bool store = P.recon != nullptr;
        const int64_t rp = P.recon_pitch;
        uint2* out0 = store ? reinterpret_cast<uint2*>(P.recon + (int64_t)(by * 8) * rp +
                                                       (int64_t)bx0 * 8)
                            : nullptr;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t w[64];
#pragma unroll
          for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int pz = 8 * i + j;
              if (kept(R, i, j)) {
                int32_t z = __float2int_rn(__uint_as_float(zf[h][zz_index(i, j)]));
                if (pz == 0) z -= 65536;  // the 1024 bias of the 64 pixels
                w[pz] = (uint32_t)z * (uint32_t)cp.cmul2[pz];
              } else {
                w[pz] = 0u;
              }
            }
          w[0] += kL2;
          sse += inverse_epilogue_u8_any<R>(w, RowsInRegs{h == 0 ? xa : xb}, store ? out0 + h : nullptr, rp,
                                        store, true, 8, 8);
        }
        acc += sse;
      }
    }
  }
  // drain: copies and MMAs still in flight (bounded) before the memory goes
  if (in_flight) mbar_wait_sleep_bounded(bar_raw, raw_phase, cp.wait_limit);
  for (int b = 0; b < 2; ++b)
    if (mma_pending[b]) mbar_wait_sleep_bounded(smem_addr(bar + b), (mma_phase >> b) & 1u, cp.wait_limit);
  if (p >= 0) {
    acc = warp_sum_u64(acc);
    if (lane == 0 && acc) atomicAdd(sse_out + P.slot, acc);
  }
  tc_fence_before();
  __syncthreads();
  if (wid == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)COLS)
                 : "memory");
  }
}

// B matrices for every r: slot r - 1 holds [row k (8)][coefficient n (NH)]
// [column l (8) fp16] = (t_i kron t_j)[k][l] for the n-th kept zig-zag
// position (i, j) (zero for n >= r), NH = nh(class(r)); written once per
// device from the host.
__device__ __align__(128) uint16_t g_tc_b[64][128 * 128];

}  // namespace

namespace {
const int8_t kT1Host[64] = {1, 1, 1,  1,  1,  1,  1,  1,  2,  2,  1,  0,  0,  -1, -2, -2,
                            2, 1, -1, -2, -2, -1, 1,  2,  1,  0,  -2, -2, 2,  2,  0,  -1,
                            1, -1, -1, 1, 1,  -1, -1, 1,  2,  -2, 0,  1,  -1, 0,  2,  -2,
                            1, -2, 2, -1, -1, 2,  -2, 1,  0,  -1, 2,  -2, 2,  -2, 1,  0};

uint16_t f16_bits_of_small_int(int v) {
  switch (v) {
    case 0: return 0x0000;
    case 1: return 0x3c00;
    case 2: return 0x4000;
    case 4: return 0x4400;
    case -1: return 0xbc00;
    case -2: return 0xc000;
    case -4: return 0xc400;
    default: return 0x7e00;  // not reachable: T1 kron T1 entries are 0, +-1, +-2, +-4
  }
}
}  // namespace

// Build (once per device, synchronously, outside any capture) and return
// the device address of the B table.
cudaError_t tc_prepare(const uint16_t** table) {
  static std::mutex mu;
  static void* addr[256] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidValue;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    std::vector<uint16_t> host((size_t)64 * 128 * 128, 0);
    for (int r = 1; r <= 64; ++r) {
      const int NH = nh_of(r_class(r));
      uint16_t* dst = host.data() + (size_t)(r - 1) * 128 * 128;
      for (int e2 = 0; e2 < NH * 64; ++e2) {
        const int k = e2 / (NH * 8), idx = (e2 / 8) % NH, l = e2 % 8;
        int v = 0;
        if (idx < r) {
          int pos = 0;
          for (int q = 0; q < 64; ++q)
            if (zz_index(q >> 3, q & 7) == idx) pos = q;
          v = kT1Host[(pos >> 3) * 8 + k] * kT1Host[(pos & 7) * 8 + l];
        }
        dst[e2] = f16_bits_of_small_int(v);
      }
    }
    e = cudaMemcpyToSymbol(g_tc_b, host.data(), host.size() * sizeof(uint16_t));
    if (e != cudaSuccess) return e;
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_tc_b);
    if (e != cudaSuccess) return e;
    addr[dev] = p;
  }
  *table = static_cast<const uint16_t*>(addr[dev]);
  return cudaSuccess;
}

template <int R>
cudaError_t launch_codec_tc(const PlaneTable& tab, const CodecParams& cp, int r_exact,
                            unsigned long long* sse, cudaStream_t s) {
  constexpr int N = 4 * nh_of(R);  // accumulator columns of the pipelined variant (the larger)
#ifndef TDCT_TC_SMEM_PAD
#define TDCT_TC_SMEM_PAD 0
#endif
  constexpr size_t kSmem =
      kATileBytes + 4 * kUnitBytes + (size_t)nh_of(R) * 128 + 128 + TDCT_TC_SMEM_PAD;
  // at most 512 / COLS CTAs may hold tensor memory on one SM at a time
  constexpr int kMaxPerSm = 512 / tmem_cols_of(N);
  // variant 1: software-pipelined (wins at large r); 0: one tile at a time
  const bool pipe = cp.tc_variant == 1;
  auto kernel = pipe ? codec_u8_tc_pipe_kernel<R> : codec_u8_tc_kernel<R>;
  static int resident_v[2] = {0, 0}, sms = 0;
  int& resident = resident_v[pipe ? 1 : 0];
  if (resident == 0) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    // residency from registers and shared memory (the occupancy query
    // under-reports kernels that hold tensor memory)
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    int dev = 0, regs_sm = 65536, smem_sm = 233472, reserved = 1024;
    if (cudaGetDevice(&dev) == cudaSuccess) {
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    }
    const int by_regs = regs_sm / (kTcThreads * (fa.numRegs > 0 ? fa.numRegs : 255));
    const int by_smem = smem_sm / (int)(kSmem + fa.sharedSizeBytes + reserved);
    resident = by_regs < by_smem ? by_regs : by_smem;
    if (resident < 1) resident = 1;
    if (resident > kMaxPerSm) resident = kMaxPerSm;
    sms = device_sms();
  }
  // an explicit request may exceed the occupancy query (which reports one
  // CTA per SM for this kernel) but never the tensor-memory budget
  int per_sm = cp.ctas_per_sm > 0 ? cp.ctas_per_sm : resident;
  if (per_sm > kMaxPerSm) per_sm = kMaxPerSm;
  const uint16_t* table = nullptr;
  cudaError_t eb = tc_prepare(&table);
  if (eb != cudaSuccess) return eb;
  const uint16_t* bmat = table + (size_t)(r_exact - 1) * 128 * 128;
  const int64_t tiles = (tab.total_units + 3) / 4;
  if (tiles < 1) return cudaSuccess;
  int64_t grid = (int64_t)per_sm * sms;
  if (grid > tiles) grid = tiles;
  kernel<<<(unsigned)grid, kTcThreads, kSmem, s>>>(tab, cp, bmat, sse);
  return cudaGetLastError();
}

#define TDCT_TC_INST(R)                                                                   \
  template cudaError_t launch_codec_tc<R>(const PlaneTable&, const CodecParams&, int,     \
                                          unsigned long long*, cudaStream_t);
TDCT_FOR_EACH_CLASS(TDCT_TC_INST)
#undef TDCT_TC_INST

}  // namespace tdct
