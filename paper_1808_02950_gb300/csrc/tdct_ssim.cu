// tdct_ssim.cu -- mean SSIM of u8 plane pairs on the CUDA cores (§6.1 rates
// the reconstructions with the index of Wang et al. 2004).
//
// At every window position (the 11x11 window inside the plane):
//   mx = sum w x, sx^2 = sum w x^2 - mx^2, sxy = sum w x y - mx my,
//   SSIM = ((2 mx my + C1)(2 sxy + C2)) / ((mx^2 + my^2 + C1)(sx^2 + sy^2 + C2)).
// The window is separable, w = g g^T, so each of the five moment maps
// (x, y, x^2, y^2, x y) is filtered by 11 taps along rows, then 11 along
// columns.  Samples are centred (x - 128) before filtering: the variances and
// the covariance do not change, the means shift back by 128, and the squares
// stay below 2^14, which keeps the FP32 differences E[x^2] - mx^2 accurate.
//
// Work: a unit is a strip of 64 output columns (two adjacent ones per lane)
// by 512 output rows of one plane; units are dealt to persistent warps as
// contiguous ranges.  For each input row the warp stages its 74 centred
// (x, y) pairs in shared memory (each sample loaded one row ahead of its
// use); each lane reads its 12 input columns once, forms their squares and
// products once, and the horizontal sums of both its columns; the last 11
// of those stay in registers (rings whose slots are compile-time indices of
// an 11-way unrolled row loop) and, once 11 rows are in, give the vertical
// sums and the SSIM of two outputs.  (x, y) and (x^2, y^2) are carried as
// FP32x2 pairs (FFMA2 / FMUL2).
#include "tdct_ssim.h"

namespace tdct {

namespace {

__device__ __forceinline__ int find_ssim_plane(const SsimDesc* d, int n, int64_t u) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&d[mid].unit_begin) <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ float2 centred_pair(uint32_t x, uint32_t y) {
  // 2^23 + v as an FP32 bit pattern, minus 2^23 + 128: v - 128 exactly
  const float2 f = make_float2(__uint_as_float(0x4B000000u | x), __uint_as_float(0x4B000000u | y));
  return __fadd2_rn(f, make_float2(-8388736.0f, -8388736.0f));
}

// Per output column: horizontal sums of one input row.
struct HSums {
  float2 A;  // (sum g x, sum g y), centred samples
  float2 B;  // (sum g x^2, sum g y^2)
  float C;   // sum g x y
};

// One ring step: the new row's horizontal sums go to slot K; when 11 rows
// are in, the vertical sums over slots K+1 .. K (oldest first).  One
// instantiation per slot keeps the ring in registers; the row loop itself
// stays rolled (its body appears once), which keeps the code within the
// instruction cache.
template <int K>
__device__ __forceinline__ void ring_step(HSums (&r0)[kSsimWin], HSums (&r1)[kSsimWin],
                                          const HSums& n0, const HSums& n1, bool ready,
                                          const SsimParams& sp, HSums& v0, HSums& v1) {
  r0[K] = n0;
  r1[K] = n1;
  if (!ready) return;
  v0 = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), 0.f};
  v1 = v0;
#pragma unroll
  for (int i = 0; i < kSsimWin; ++i) {
    const int sl = (K + 1 + i) % kSsimWin;
    const float2 g = make_float2(sp.g[i], sp.g[i]);
    v0.A = __ffma2_rn(g, r0[sl].A, v0.A);
    v0.B = __ffma2_rn(g, r0[sl].B, v0.B);
    v0.C = fmaf(sp.g[i], r0[sl].C, v0.C);
    v1.A = __ffma2_rn(g, r1[sl].A, v1.A);
    v1.B = __ffma2_rn(g, r1[sl].B, v1.B);
    v1.C = fmaf(sp.g[i], r1[sl].C, v1.C);
  }
}

__global__ void __launch_bounds__(128, 2)
    ssim_kernel(const SsimDesc* __restrict__ descs, int n, int64_t total_units,
                const SsimParams sp, double* __restrict__ out) {
  // per warp, two row buffers of 64 + 10 (+2 pad) centred (x, y) pairs
  __shared__ __align__(16) float2 rowbuf[4][2][kSsimStrip + kSsimWin + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t u_begin = (total_units * warp) / nwarps;
  const int64_t u_end = (total_units * (warp + 1)) / nwarps;
  int p = -1;
  int64_t p_end = -1;
  SsimDesc P;
  double acc = 0.0;
  for (int64_t u = u_begin; u < u_end; ++u) {
    if (u >= p_end) {
      if (p >= 0) {
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0 && acc != 0.0) atomicAdd(out + P.slot, acc);
        acc = 0.0;
      }
      p = find_ssim_plane(descs, n, u);
      P = descs[p];
      p_end = (p + 1 < n) ? descs[p + 1].unit_begin : total_units;
    }
    const int local = (int)(u - P.unit_begin);
    const int band = local / P.strips, strip = local - band * P.strips;
    const int c0 = strip * kSsimStrip, o0 = band * kSsimBand;
    const int out_rows = min(kSsimBand, P.H - (kSsimWin - 1) - o0);
    const int r_end = o0 + out_rows + kSsimWin - 1;
    const int cl = 2 * lane;                 // the lane's first column within the strip
    const int outW = P.W - (kSsimWin - 1);
    const bool ok0 = c0 + cl < outW, ok1 = c0 + cl + 1 < outW;
    // staged columns: lane l writes columns 2l, 2l+1 and lanes 0..4 the halo 64..73
    const int s0 = c0 + cl, s1 = s0 + 1, h0 = c0 + kSsimStrip + cl, h1 = h0 + 1;
    HSums r0[kSsimWin], r1[kSsimWin];
    float lane_sum = 0.0f;
    uint32_t nx0 = 0, nx1 = 0, ny0 = 0, ny1 = 0, nhx0 = 0, nhx1 = 0, nhy0 = 0, nhy1 = 0;
    auto load_row = [&](int row) {
      const uint8_t* xr = P.x + (int64_t)row * P.xpitch;
      const uint8_t* yr = P.y + (int64_t)row * P.ypitch;
      nx0 = s0 < P.W ? __ldg(xr + s0) : 0u;
      nx1 = s1 < P.W ? __ldg(xr + s1) : 0u;
      ny0 = s0 < P.W ? __ldg(yr + s0) : 0u;
      ny1 = s1 < P.W ? __ldg(yr + s1) : 0u;
      if (lane < (kSsimWin - 1) / 2) {
        nhx0 = h0 < P.W ? __ldg(xr + h0) : 0u;
        nhx1 = h1 < P.W ? __ldg(xr + h1) : 0u;
        nhy0 = h0 < P.W ? __ldg(yr + h0) : 0u;
        nhy1 = h1 < P.W ? __ldg(yr + h1) : 0u;
      }
    };
    load_row(o0);
    int kslot = 0;  // ring slot of the current row: (row - o0) mod 11
#pragma unroll 1
    for (int row = o0; row < r_end; ++row) {
      float2* buf = rowbuf[wid][row & 1];
      const float2 a0 = centred_pair(nx0, ny0), a1 = centred_pair(nx1, ny1);
      float2 ha0, ha1;
      if (lane < (kSsimWin - 1) / 2) {
        ha0 = centred_pair(nhx0, nhy0);
        ha1 = centred_pair(nhx1, nhy1);
      }
      if (row + 1 < r_end) load_row(row + 1);  // one row ahead
      *reinterpret_cast<float4*>(buf + cl) = make_float4(a0.x, a0.y, a1.x, a1.y);
      if (lane < (kSsimWin - 1) / 2)
        *reinterpret_cast<float4*>(buf + kSsimStrip + cl) = make_float4(ha0.x, ha0.y, ha1.x, ha1.y);
      __syncwarp();
      // the lane's 12 input columns (cl .. cl + 11), their squares and products
      float2 a[kSsimWin + 1], q[kSsimWin + 1];
      float c[kSsimWin + 1];
#pragma unroll
      for (int t = 0; t < (kSsimWin + 1) / 2; ++t) {
        const float4 v = *reinterpret_cast<const float4*>(buf + cl + 2 * t);
        a[2 * t] = make_float2(v.x, v.y);
        a[2 * t + 1] = make_float2(v.z, v.w);
      }
#pragma unroll
      for (int t = 0; t <= kSsimWin; ++t) {
        q[t] = __fmul2_rn(a[t], a[t]);
        c[t] = a[t].x * a[t].y;
      }
      HSums n0 = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), 0.f};
      HSums n1 = n0;
#pragma unroll
      for (int j = 0; j < kSsimWin; ++j) {
        const float2 g = make_float2(sp.g[j], sp.g[j]);
        n0.A = __ffma2_rn(g, a[j], n0.A);
        n0.B = __ffma2_rn(g, q[j], n0.B);
        n0.C = fmaf(sp.g[j], c[j], n0.C);
        n1.A = __ffma2_rn(g, a[j + 1], n1.A);
        n1.B = __ffma2_rn(g, q[j + 1], n1.B);
        n1.C = fmaf(sp.g[j], c[j + 1], n1.C);
      }
      const bool ready = row - o0 >= kSsimWin - 1;
      HSums v0, v1;
      switch (kslot) {
#define TDCT_SSIM_SLOT(K) \
  case K:                 \
    ring_step<K>(r0, r1, n0, n1, ready, sp, v0, v1); \
    break;
        TDCT_SSIM_SLOT(0) TDCT_SSIM_SLOT(1) TDCT_SSIM_SLOT(2) TDCT_SSIM_SLOT(3)
        TDCT_SSIM_SLOT(4) TDCT_SSIM_SLOT(5) TDCT_SSIM_SLOT(6) TDCT_SSIM_SLOT(7)
        TDCT_SSIM_SLOT(8) TDCT_SSIM_SLOT(9) TDCT_SSIM_SLOT(10)
#undef TDCT_SSIM_SLOT
        default:
          break;
      }
      kslot = kslot == kSsimWin - 1 ? 0 : kslot + 1;
      if (ready) {
        auto ssim_of = [&](const HSums& v) {
          const float mx = v.A.x + 128.0f, my = v.A.y + 128.0f;
          const float sxx = v.B.x - v.A.x * v.A.x, syy = v.B.y - v.A.y * v.A.y;
          const float sxy = v.C - v.A.x * v.A.y;
          const float num = (2.0f * mx * my + sp.C1) * (2.0f * sxy + sp.C2);
          const float den = (mx * mx + my * my + sp.C1) * (sxx + syy + sp.C2);
          return __fdividef(num, den);
        };
        if (ok0) lane_sum += ssim_of(v0);
        if (ok1) lane_sum += ssim_of(v1);
      }
    }
    acc += (double)lane_sum;
  }
  if (p >= 0) {
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0 && acc != 0.0) atomicAdd(out + P.slot, acc);
  }
}

// Mean over the window positions.
__global__ void ssim_finalize(const SsimDesc* __restrict__ descs, int n, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const SsimDesc d = descs[i];
  out[d.slot] /= (double)(d.H - (kSsimWin - 1)) * (double)(d.W - (kSsimWin - 1));
}

}  // namespace

cudaError_t launch_ssim(const SsimDesc* d_descs, int n, int64_t total_units,
                        const SsimParams& sp, double* d_out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(d_out, 0, sizeof(double) * n, s);
  if (e != cudaSuccess) return e;
  static int resident = 0, sms = 0;
  if (resident == 0) {
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, ssim_kernel, 128, 0)) !=
        cudaSuccess)
      return e;
    if (resident < 1) resident = 1;
  }
  int64_t grid = (int64_t)resident * sms;
  const int64_t by_work = (total_units + 3) / 4;
  if (by_work < grid) grid = by_work;
  if (grid < 1) grid = 1;
  ssim_kernel<<<(unsigned)grid, 128, 0, s>>>(d_descs, n, total_units, sp, d_out);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  ssim_finalize<<<(n + 255) / 256, 256, 0, s>>>(d_descs, n, d_out);
  return cudaGetLastError();
}

}  // namespace tdct
