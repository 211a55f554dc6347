// tdct_abi.cu -- the extern "C" boundary of libtdct (declared in include/tdct.h).
//
// Host side: argument validation, the block-offset tables of ragged batches,
// launch dispatch over the compiled r-classes, batch plans replayed as CUDA
// graphs, the device status word.  Also the small non-fused kernels: the
// forward-only and inverse-only transforms and the FP64 PSNR finalisation.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/tdct.h"
#include "tdct_classes.h"
#include "tdct_dct.h"
#include "tdct_dct_tc.h"
#include "tdct_generic.cuh"
#include "tdct_jam.h"
#include "tdct_kernels.cuh"
#include "tdct_search.h"
#include "tdct_ssim.h"
#include "tdct_sweep.h"
#include "tdct_tc.h"

namespace tdct {

// Instantiated in tdct_inst_*.cu.
#define TDCT_EXTERN(R)                                                                       \
  extern template cudaError_t launch_codec<R, 0>(const PlaneTable&, const CodecParams&,      \
                                                 unsigned long long*, int, cudaStream_t);    \
  extern template cudaError_t launch_codec<R, 1>(const PlaneTable&, const CodecParams&,      \
                                                 unsigned long long*, int, cudaStream_t);
TDCT_FOR_EACH_CLASS(TDCT_EXTERN)
#undef TDCT_EXTERN

// Device status word (bounded waits and internal checks record a code here).
__device__ int g_status;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(TDCT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// T1 of §4.1, row-major.
constexpr int8_t kT1[64] = {
    1, 1, 1,  1,  1,  1,  1,  1,  2, 2,  1,  0,  0,  -1, -2, -2, 2, 1,  -1, -2, -2, -1,
    1, 2, 1,  0,  -2, -2, 2,  2,  0, -1, 1,  -1, -1, 1,  1,  -1, -1, 1, 2,  -2, 0,  1,
    -1, 0, 2, -2, 1,  -2, 2,  -1, -1, 2, -2, 1,  0,  -1, 2,  -2, 2,  -2, 1, 0};

// The transform of a call.  T1 runs on the fused kernels (fast algorithm of
// §5.1, both engines); any other orthogonal T on the generic kernels, whose
// parameters are built here.
struct Transform {
  bool t1 = true;
  GenericParams base;  // T, L^2 and the rounding division constant; cmul2 per r
  int32_t q[8];        // q_k = L / n_k
};

int64_t gcd64(int64_t a, int64_t b) {
  while (b) {
    const int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

// T T^T == diag(n) (Eq. (2) with a diagonal S); builds the generic parameters
// when T is not T1.
//
// Bounds of the generic kernels.  A reconstructed sample is the orthogonal
// projection of the block onto the kept basis functions, so |N / L^2| <=
// ||block||_2 <= 8 * 255 = 2040 for u8 and int16 planes; the kernels form 2N
// in wrapping 32-bit arithmetic, exact when |2N| + L^2 < 2^31, i.e.
// 4082 L^2 < 2^31 (L <= 725).  Rounding divides a = |2N| + L^2 (or 2N + L^2)
// by 2 L^2 as (a * magic) >> (32 + shift) with magic = ceil(2^k / (2 L^2)) <
// 2^31; with e = magic * 2 L^2 - 2^k the quotient is exact for 0 <= a < A when
// e * A < 2^k, and it is checked here for A = 4082 L^2.
int resolve_transform(const int8_t* T, const int32_t* n, Transform* tr) {
  if (!T || !n) return fail(TDCT_EINVAL, "T and n must not be NULL");
  for (int a = 0; a < 8; ++a)
    for (int b = 0; b < 8; ++b) {
      int64_t dot = 0;
      for (int l = 0; l < 8; ++l) dot += (int64_t)T[a * 8 + l] * T[b * 8 + l];
      const int64_t want = a == b ? n[a] : 0;
      if (dot != want)
        return fail(TDCT_ENOTORTHO, "(T T^T)[%d][%d] = %lld but diag(n) gives %lld", a, b,
                    (long long)dot, (long long)want);
    }
  for (int k = 0; k < 8; ++k)
    if (n[k] < 1) return fail(TDCT_ENOTORTHO, "row %d of T is zero (n_%d = 0)", k, k);
  tr->t1 = std::memcmp(T, kT1, 64) == 0;
  if (tr->t1) return TDCT_OK;
  int64_t L = 1;
  for (int k = 0; k < 8; ++k) {
    L = L / gcd64(L, n[k]) * n[k];
    if (L > 725)
      return fail(TDCT_EUNSUPPORTED,
                  "lcm of the row norms n exceeds 725: the exact 32-bit reconstruction needs "
                  "4082 L^2 < 2^31");
  }
  const int64_t L2 = L * L, d = 2 * L2, A = 4082 * L2;
  int k = 32;
  while (k < 62 && (((int64_t)1 << (k + 1)) + d - 1) / d < ((int64_t)1 << 31)) ++k;
  const int64_t magic = (((int64_t)1 << k) + d - 1) / d;
  const int64_t e = magic * d - ((int64_t)1 << k);
  if (magic >= ((int64_t)1 << 31) || (unsigned __int128)e * (unsigned __int128)A >=
                                         ((unsigned __int128)1 << k))
    return fail(TDCT_EUNSUPPORTED, "no exact 32-bit division constant for L = %lld",
                (long long)L);
  std::memset(&tr->base, 0, sizeof tr->base);
  for (int i = 0; i < 64; ++i) tr->base.T[i] = T[i];
  tr->base.L2 = (int32_t)L2;
  tr->base.magic = (int32_t)magic;
  tr->base.shift = k - 32;
  for (int i = 0; i < 8; ++i) tr->q[i] = (int32_t)(L / n[i]);
  // even rows symmetric and odd rows antisymmetric: the even/odd kernels
  bool sym = true;
  for (int k = 0; k < 8; ++k)
    for (int l = 0; l < 8; ++l)
      if (T[8 * k + 7 - l] != ((k & 1) ? -T[8 * k + l] : T[8 * k + l])) sym = false;
  // two u8 blocks per register in the forward: every |Z_ij| of u8 samples,
  // 255 * max(sum of positive, sum of negative entries of t_i kron t_j), fits
  // a signed 16-bit lane, except Z_00 when t_0 >= 0, which may use the
  // unsigned lane range
  bool pack = sym, dc_u16 = false;
  for (int i = 0; i < 8 && pack; ++i)
    for (int j = 0; j < 8 && pack; ++j) {
      int64_t pos = 0, neg = 0;
      for (int k = 0; k < 8; ++k)
        for (int l = 0; l < 8; ++l) {
          const int64_t w = (int64_t)T[8 * i + k] * T[8 * j + l];
          (w > 0 ? pos : neg) += w > 0 ? w : -w;
        }
      const int64_t bound = 255 * (pos > neg ? pos : neg);
      if (bound <= 32767) continue;
      if (i == 0 && j == 0 && neg == 0 && bound <= 65535) dc_u16 = true;
      else pack = false;
    }
  tr->base.flags = (sym ? kGenSym : 0) | (pack ? kGenPackU8 : 0) | (pack && dc_u16 ? kGenDcU16 : 0);
  return TDCT_OK;
}

// Generic parameters for retention r: cmul2 = 2 q_i q_j on the first r
// zig-zag positions (Eq. (11) mask), else 0.
GenericParams generic_for_r(const Transform& tr, int r) {
  GenericParams gp = tr.base;
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j) gp.cmul2[8 * i + j] = kept(r, i, j) ? 2 * tr.q[i] * tr.q[j] : 0;
  return gp;
}

int check_engine(const Transform& tr, int path) {
  if (path < TDCT_PATH_AUTO || path > TDCT_PATH_TENSOR_PIPELINED)
    return fail(TDCT_EUNSUPPORTED, "path %d is not a tdct_path", path);
  if (!tr.t1 && (path == TDCT_PATH_TENSOR || path == TDCT_PATH_TENSOR_PIPELINED))
    return fail(TDCT_EUNSUPPORTED,
                "the tensor-core engine implements T1 only; use TDCT_PATH_AUTO or "
                "TDCT_PATH_BUTTERFLY for another T");
  return TDCT_OK;
}

int sample_bytes(int dtype) { return dtype == TDCT_I16 ? 2 : 1; }

int check_plane(const void* img, int64_t pitch, int H, int W, int dtype, const char* what) {
  if (dtype != TDCT_U8 && dtype != TDCT_I16) return fail(TDCT_EINVAL, "%s: bad dtype %d", what, dtype);
  if (!img) return fail(TDCT_EINVAL, "%s: NULL plane pointer", what);
  if (H < 1 || W < 1 || H > (1 << 28) || W > (1 << 28))
    return fail(TDCT_EINVAL, "%s: bad size %d x %d", what, H, W);
  if (pitch < (int64_t)W * sample_bytes(dtype))
    return fail(TDCT_EINVAL, "%s: pitch %lld < W * sample size", what, (long long)pitch);
  if (dtype == TDCT_I16 && ((reinterpret_cast<uintptr_t>(img) | (uintptr_t)pitch) & 1))
    return fail(TDCT_EINVAL, "%s: int16 plane must be 2-byte aligned", what);
  return TDCT_OK;
}

int check_r(int r) {
  if (r < 1 || r > 64) return fail(TDCT_EINVAL, "r = %d outside 1..64", r);
  return TDCT_OK;
}

// One-shot test hook: the next codec launch withholds one bulk copy so that
// its bounded wait runs out (see tdct_debug_inject_wait_timeout).
std::atomic<int> g_inject_timeout{0};
std::atomic<int> g_search_hit_cap{kSearchHitCap};

int* status_word() {
  static void* addr[256] = {};
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev] && cudaGetSymbolAddress(&addr[dev], g_status) != cudaSuccess) addr[dev] = nullptr;
  return static_cast<int*>(addr[dev]);
}

CodecParams make_params(int r, int ctas_per_sm = 0, int tc_variant = 0) {
  CodecParams cp;
  std::memset(&cp, 0, sizeof cp);
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j) {
      cp.cmul[8 * i + j] = kept(r, i, j) ? q_of(i) * q_of(j) : 0;
      cp.cmul2[8 * i + j] = 2 * cp.cmul[8 * i + j];
      cp.cmul2h[8 * i + j] = cp.cmul2[8 * i + j] * 65536;
    }
  cp.status = status_word();
  cp.wait_limit = 2000000000ll;  // about a second of SM clock
  cp.ctas_per_sm = ctas_per_sm;
  cp.tc_variant = tc_variant;
  if (const char* env = std::getenv("TDCT_CTAS_PER_SM")) cp.ctas_per_sm = std::atoi(env);
  if (g_inject_timeout.exchange(0)) {
    cp.test_hook = 1;
    cp.wait_limit = 20000000ll;
  }
  return cp;
}

bool aligned8(const void* p, int64_t pitch) {
  return ((reinterpret_cast<uintptr_t>(p) | (uintptr_t)pitch) & 7) == 0;
}

PlaneDesc make_desc(const void* img, int64_t pitch, int H, int W, int dtype, int r, void* recon,
                    int64_t recon_pitch, int slot) {
  PlaneDesc d;
  std::memset(&d, 0, sizeof d);
  d.img = static_cast<const uint8_t*>(img);
  d.recon = static_cast<uint8_t*>(recon);
  d.pitch = pitch;
  d.recon_pitch = recon_pitch;
  d.H = H;
  d.W = W;
  d.nbx = (W + 7) / 8;
  d.nby = (H + 7) / 8;
  d.chunks = (d.nbx + 63) / 64;
  d.dtype = dtype;
  d.r = r;
  // bulk-copy ring: 16-byte aligned base, H % 8 == 0, and either 16-byte
  // aligned rows with W % 16 == 0, or a pitch of 8 mod 16 with W % 16 == 8
  // (odd rows then start 8 bytes past a boundary; their copies reach 8 bytes
  // into the previous row, and even rows' last copies 8 bytes into the next)
  const bool base16 = (reinterpret_cast<uintptr_t>(img) & 15) == 0;
  const bool shifted = (pitch & 15) == 8 && W % 16 == 8;
  const bool bulk8 = dtype == TDCT_U8 && base16 && H % 8 == 0 &&
                     (((pitch & 15) == 0 && W % 16 == 0) || shifted) &&
                     (!recon || aligned8(recon, recon_pitch));
  // int16: 16-byte aligned base and pitch and W % 8 == 0 (rows of 16-byte
  // multiples), any H (rows past the bottom edge are zero-filled in the slot)
  const bool bulk16 = dtype == TDCT_I16 && base16 && (pitch & 15) == 0 && W % 8 == 0 &&
                      (!recon || aligned8(recon, recon_pitch));
  const bool bulk = bulk8 || bulk16;
  // staged-copy rings: planes that miss the bulk-copy conditions, with 8-byte
  // aligned rows and W % 8 == 0, any height (rows past the bottom edge are
  // zero-filled in shared memory)
  const bool staged = !bulk && aligned8(img, pitch) && W % 8 == 0 &&
                      (!recon || aligned8(recon, recon_pitch));
  d.vec16 = (aligned8(img, pitch) ? 1 : 0) | ((recon && aligned8(recon, recon_pitch)) ? 2 : 0) |
            (bulk ? 4 : 0) | (staged ? 8 : 0) | ((bulk8 && shifted) ? 16 : 0);
  d.slot = slot;
  return d;
}

// Units of a plane: per block row ceil(nbx / 64), or, for planes whose units
// run on across block rows (vec16 bit 5), ceil(nbx nby / 64).
int64_t units_of(const PlaneDesc& d) {
  if (d.vec16 & 32) return ((int64_t)d.nbx * d.nby + 63) / 64;
  return (int64_t)d.nby * d.chunks;
}

// Bulk-copy u8 planes (rows 16-byte aligned) at least 64 blocks wide whose
// width is not a multiple of 64 blocks take units that run on across block
// rows (no nearly empty unit at the end of each block row), at r > 10, where
// the kernel is bound by issue.  Measured on GB300 (512 planes of 1024 x 1040,
// a third unit of 2 blocks per block row): r = 16 from 0.46 to 0.64 of the
// HBM peak; at r = 4, bound by memory, from 0.71 to 0.64 (the copies of
// segments that start inside a row), so the classes up to 10 keep per-row
// units.
bool wants_wrap(const PlaneDesc& d) {
  return d.dtype == TDCT_U8 && (d.vec16 & 4) && !(d.vec16 & 16) && d.nbx >= 64 &&
         d.nbx % 64 != 0 && d.r > 10;
}

cudaError_t dispatch_codec_tc(int r, const PlaneTable& tab, unsigned long long* sse,
                              cudaStream_t s, int ctas_per_sm = 0, int tc_variant = 0) {
  const CodecParams cp = make_params(r, ctas_per_sm, tc_variant);
  switch (r_class(r)) {
#define TDCT_CASE(R) \
  case R:            \
    return launch_codec_tc<R>(tab, cp, r, sse, s);
    TDCT_FOR_EACH_CLASS(TDCT_CASE)
#undef TDCT_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t dispatch_codec_generic(int r, int dtype, const PlaneTable& tab, const Transform& tr,
                                   unsigned long long* sse, cudaStream_t s) {
  const GenericParams gp = generic_for_r(tr, r);
  switch (r_class(r)) {
#define TDCT_CASE(R)                                                          \
  case R:                                                                     \
    return dtype == TDCT_U8 ? launch_codec_generic<R, 0>(tab, gp, sse, s)     \
                            : launch_codec_generic<R, 1>(tab, gp, sse, s);
    TDCT_FOR_EACH_CLASS(TDCT_CASE)
#undef TDCT_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

// fin_cnt (plans whose launches all run the u8 bulk-copy ring kernel): the
// kernel closes each plane itself (sse is then the plan's accumulator; see
// CodecParams::fin_cnt).
cudaError_t dispatch_codec(int r, int dtype, const PlaneTable& tab, unsigned long long* sse,
                           int max_ctas, cudaStream_t s, int ctas_per_sm = 0,
                           unsigned long long* fin_sse = nullptr, double* fin_psnr = nullptr,
                           unsigned int* fin_cnt = nullptr) {
  CodecParams cp = make_params(r, ctas_per_sm);
  cp.fin_sse = fin_sse;
  cp.fin_psnr = fin_psnr;
  cp.fin_cnt = fin_cnt;
  switch (r_class(r)) {
#define TDCT_CASE(R)                                                     \
  case R:                                                                \
    return dtype == TDCT_U8 ? launch_codec<R, 0>(tab, cp, sse, max_ctas, s) \
                            : launch_codec<R, 1>(tab, cp, sse, max_ctas, s);
    TDCT_FOR_EACH_CLASS(TDCT_CASE)
#undef TDCT_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace

// ---- forward / inverse only kernels ------------------------------------------

// Forward only: one block per thread; the 32 blocks of a warp are staged in
// shared memory so that the warp writes its 8 KB of coefficients as
// contiguous 16-byte stores (blocks are consecutive in the output).
template <int DT>
__global__ void __launch_bounds__(128) forward_kernel(const PlaneDesc P, int32_t* __restrict__ coef,
                                                      int coef_vec) {
  __shared__ __align__(16) int32_t stage[4][32 * 68];  // 68-word block stride: bank skew
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t* st = stage[wid];
  const int64_t nb = (int64_t)P.nbx * P.nby;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + wid * 32); base < nb; base += step) {
    const int64_t b = base + lane;
    if (b < nb) {
      const int by = (int)(b / P.nbx), bx = (int)(b - (int64_t)by * P.nbx);
      const bool interior = (by * 8 + 8 <= P.H) && ((bx + 1) * 8 <= P.W) && (P.vec16 & 1);
      RowWords<DT> rw;
      load_block<DT>(P, by, bx, interior, rw);
      uint32_t x[64], z[64];
#pragma unroll
      for (int k = 0; k < 8; ++k) unpack_row<DT>(rw, k, x + 8 * k);
      fwd2d<uint32_t>(x, z);
#pragma unroll
      for (int i = 0; i < 16; ++i)
        *reinterpret_cast<int4*>(st + lane * 68 + 4 * i) =
            make_int4((int)z[4 * i], (int)z[4 * i + 1], (int)z[4 * i + 2], (int)z[4 * i + 3]);
    }
    __syncwarp();
    const int64_t nblk = min((int64_t)32, nb - base);
    int32_t* dst = coef + base * 64;
    if (coef_vec) {
      for (int e = lane; e < nblk * 16; e += 32) {
        const int blk = e >> 4, i = e & 15;
        reinterpret_cast<int4*>(dst)[e] =
            *reinterpret_cast<const int4*>(st + blk * 68 + 4 * i);
      }
    } else {
      for (int e = lane; e < nblk * 64; e += 32) {
        const int blk = e >> 6, i = e & 63;
        dst[e] = st[blk * 68 + i];
      }
    }
    __syncwarp();
  }
}

template <int DT>
__global__ void __launch_bounds__(128) inverse_kernel(const int32_t* __restrict__ coef,
                                                      const PlaneDesc P, const CodecParams cp,
                                                      int coef_vec) {
  const int64_t nb = (int64_t)P.nbx * P.nby;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int by = (int)(b / P.nbx), bx = (int)(b - (int64_t)by * P.nbx);
    const int32_t* src = coef + b * 64;
    uint32_t w[64];
    if (coef_vec) {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int4 v = __ldg(reinterpret_cast<const int4*>(src) + i);
        w[4 * i] = (uint32_t)v.x;
        w[4 * i + 1] = (uint32_t)v.y;
        w[4 * i + 2] = (uint32_t)v.z;
        w[4 * i + 3] = (uint32_t)v.w;
      }
    } else {
#pragma unroll
      for (int p = 0; p < 64; ++p) w[p] = (uint32_t)__ldg(src + p);
    }
#pragma unroll
    for (int p = 0; p < 64; ++p) w[p] *= (uint32_t)cp.cmul[p];
    int32_t out[64];
    reconstruct<DT>(w, out);
    const bool fast = (by * 8 + 8 <= P.H) && ((bx + 1) * 8 <= P.W) && (P.vec16 & 2);
    store_block<DT>(P, by, bx, fast, out);
  }
}

// PSNR = 10 log10(255^2 npix / SSE) in FP64; +inf when SSE = 0 (§6.1).
__global__ void psnr_kernel(const unsigned long long* __restrict__ sse,
                            const int64_t* __restrict__ npix, int64_t npix_one,
                            double* __restrict__ psnr, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long s = sse[i];
  const double np = (double)(npix ? npix[i] : npix_one);
  psnr[i] = s == 0ull ? (double)INFINITY : 10.0 * log10(65025.0 * np / (double)s);
}

// PSNR of every (plane, r) entry of a sweep: entry e belongs to plane e / 64.
__global__ void psnr_sweep_kernel(const unsigned long long* __restrict__ sse,
                                  const int64_t* __restrict__ npix, double* __restrict__ psnr,
                                  int n) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const unsigned long long v = sse[e];
  psnr[e] = v == 0ull ? (double)INFINITY : 10.0 * log10(65025.0 * (double)npix[e / 64] / (double)v);
}

namespace {

int grid_for(int64_t items, int threads) {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t g = (items + threads - 1) / threads;
  const int64_t cap = (int64_t)sms * 16;
  if (g > cap) g = cap;
  return (int)std::max<int64_t>(g, 1);
}

// A ragged batch as per-(dtype, r) groups, each a contiguous slice of the
// descriptor array with its own unit prefix sums.
struct Group {
  int dtype, r;
  int first, count;
  int64_t units;
  int any_bulk;     // the planes take the bulk-copy ring
  int staged;       // the planes take the staged-copy ring
  int any_shifted;  // bulk planes with rows 8 mod 16 (their own launch; not the tensor engine)
  int wrap;         // bulk planes with units across block rows (their own launch; not the tensor engine)
};

// allow_wrap: the launches of this batch run the T1 ring kernels (the units
// of the generic-T and tensor-core kernels stay per block row).
int build_batch(const tdct_plane* planes, int nplanes, std::vector<PlaneDesc>& descs,
                std::vector<Group>& groups, std::vector<int64_t>& npix, bool allow_wrap) {
  if (!planes || nplanes < 1 || nplanes > (1 << 20))
    return fail(TDCT_EINVAL, "nplanes = %d outside 1..2^20 (or planes is NULL)", nplanes);
  std::map<std::tuple<int, int, int>, std::vector<int>> by_key;
  npix.resize(nplanes);
  for (int i = 0; i < nplanes; ++i) {
    const tdct_plane& p = planes[i];
    char what[64];
    std::snprintf(what, sizeof what, "plane %d", i);
    int rc = check_plane(p.img, p.pitch, p.H, p.W, p.dtype, what);
    if (rc) return rc;
    if (p.r < 1 || p.r > 64) return fail(TDCT_EINVAL, "plane %d: r = %d outside 1..64", i, p.r);
    if (p.recon && p.recon_pitch < (int64_t)p.W * sample_bytes(p.dtype))
      return fail(TDCT_EINVAL, "plane %d: recon pitch too small", i);
    const PlaneDesc probe = make_desc(p.img, p.pitch, p.H, p.W, p.dtype, p.r, p.recon, p.recon_pitch, i);
    // load path: 1 bulk-copy ring (3: its 8 mod 16 rows variant, 4: units
    // across block rows), 2 staged, 0 plain
    const int load = (probe.vec16 & 4)
                         ? ((probe.vec16 & 16) ? 3 : (allow_wrap && wants_wrap(probe)) ? 4 : 1)
                         : (probe.vec16 & 8) ? 2 : 0;
    by_key[{p.dtype, p.r, load}].push_back(i);
    npix[i] = (int64_t)p.H * p.W;
  }
  descs.clear();
  groups.clear();
  for (auto& kv : by_key) {
    const int load = std::get<2>(kv.first);
    Group g{std::get<0>(kv.first), std::get<1>(kv.first), (int)descs.size(),
            (int)kv.second.size(), 0, (load == 1 || load == 3 || load == 4) ? 1 : 0,
            load == 2 ? 1 : 0, load == 3 ? 1 : 0, load == 4 ? 1 : 0};
    for (int i : kv.second) {
      const tdct_plane& p = planes[i];
      PlaneDesc d = make_desc(p.img, p.pitch, p.H, p.W, p.dtype, p.r, p.recon, p.recon_pitch, i);
      if (load == 4) d.vec16 |= 32;
      d.unit_begin = g.units;
      g.units += units_of(d);
      descs.push_back(d);
    }
    groups.push_back(g);
  }
  return TDCT_OK;
}

// Whether a batch coded with transform tr on engine `path` may use units
// across block rows: the T1 ring kernels take them, the generic-T and
// tensor-core kernels do not (under TDCT_PATH_AUTO such groups run on the
// butterfly engine whatever the autotuner picks).
bool wrap_allowed(const Transform& tr, int path) {
  return tr.t1 && path != TDCT_PATH_TENSOR && path != TDCT_PATH_TENSOR_PIPELINED;
}

// Whether group g of a batch coded with transform tr on engine `path` runs
// the u8 bulk-copy ring kernel (the kernel that can close its planes itself).
bool group_on_u8_ring(const Transform& tr, const Group& g, int path) {
  const bool tensor = path == TDCT_PATH_TENSOR || path == TDCT_PATH_TENSOR_PIPELINED;
  return tr.t1 && g.dtype == TDCT_U8 && g.any_bulk && !(tensor && !g.any_shifted && !g.wrap);
}

// A plan's accumulators for launches that close their planes themselves:
// SSE and finished units per plane (both zero between launches).
struct PlanFinal {
  unsigned long long* acc;
  unsigned int* cnt;
};

// Streams on which the groups of a plan's graph run side by side (so that
// one group's launch tail overlaps the next group's start).
constexpr int kPlanBranches = 4;
struct Branches {
  cudaStream_t stream[kPlanBranches] = {};
  cudaEvent_t fork = nullptr, join[kPlanBranches] = {};
};

// Enqueue the kernels of a batch whose descriptors live at d_descs (device).
// With `br`, the groups are distributed round-robin over its streams between a
// fork and a join on s (graph capture: parallel branches).  With `fin` (every
// group on the u8 bulk-copy ring), the codec launches write SSE and PSNR
// themselves: no reset of `sse` before them and no PSNR kernel after.
cudaError_t enqueue_batch(const Transform& tr, const std::vector<Group>& groups,
                          const PlaneDesc* d_descs, const int64_t* d_npix, int nplanes,
                          unsigned long long* sse, double* psnr, cudaStream_t s,
                          int path = TDCT_PATH_AUTO, int ctas_per_sm = 0, int tc_variant = 0,
                          const Branches* br = nullptr, const PlanFinal* fin = nullptr) {
  cudaError_t e = cudaSuccess;
  if (fin) {
    for (const Group& g : groups)
      if (!group_on_u8_ring(tr, g, path)) return cudaErrorInvalidValue;
  } else {
    e = cudaMemsetAsync(sse, 0, sizeof(unsigned long long) * nplanes, s);
    if (e != cudaSuccess) return e;
  }
  const int nbr = (br && groups.size() > 1) ? (int)std::min<size_t>(groups.size(), kPlanBranches) : 0;
  if (nbr > 0) {
    if ((e = cudaEventRecord(br->fork, s)) != cudaSuccess) return e;
    for (int b = 0; b < nbr; ++b)
      if ((e = cudaStreamWaitEvent(br->stream[b], br->fork, 0)) != cudaSuccess) return e;
  }
  int gi = 0;
  for (const Group& g : groups) {
    const cudaStream_t gs = nbr > 0 ? br->stream[gi % nbr] : s;
    ++gi;
    PlaneTable tab;
    std::memset(&tab, 0, sizeof tab);
    tab.d = d_descs + g.first;
    tab.n = g.count;
    tab.total_units = g.units;
    tab.any_bulk = g.any_bulk;
    tab.shifted = g.any_shifted;
    tab.staged = g.staged;
    tab.wrap = g.wrap;
    const bool tensor = path == TDCT_PATH_TENSOR || path == TDCT_PATH_TENSOR_PIPELINED;
    if (!tr.t1)
      e = dispatch_codec_generic(g.r, g.dtype, tab, tr, sse, gs);
    else if (tensor && g.any_bulk && !g.any_shifted && !g.wrap && g.dtype == TDCT_U8)
      e = dispatch_codec_tc(g.r, tab, sse, gs, ctas_per_sm,
                            path == TDCT_PATH_TENSOR_PIPELINED ? 1 : tc_variant);
    else if (fin)
      e = dispatch_codec(g.r, g.dtype, tab, fin->acc, 0, gs, ctas_per_sm, sse, psnr, fin->cnt);
    else
      e = dispatch_codec(g.r, g.dtype, tab, sse, 0, gs, ctas_per_sm);
    if (e != cudaSuccess) return e;
  }
  for (int b = 0; b < nbr; ++b) {
    if ((e = cudaEventRecord(br->join[b], br->stream[b])) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s, br->join[b], 0)) != cudaSuccess) return e;
  }
  if (psnr && !fin) {
    psnr_kernel<<<(nplanes + 255) / 256, 256, 0, s>>>(sse, d_npix, 0, psnr, nplanes);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace
}  // namespace tdct

using namespace tdct;

// ---- plans ----------------------------------------------------------------------

struct tdct_plan {
  Transform tr;
  std::vector<Group> groups;
  int path = TDCT_PATH_AUTO;   // engine used by launches (never AUTO after creation)
  int ctas_per_sm = 0;         // launch shape (0 = the library default)
  int tc_variant = 0;          // tensor engine: 0 one tile at a time, 1 pipelined
  float tuned_ms = 0.f;        // time of the chosen configuration (autotuned plans)
  int nplanes = 0;
  PlaneDesc* d_descs = nullptr;
  int64_t* d_npix = nullptr;
  cudaStream_t capture_stream = nullptr;
  Branches branches;           // the groups' parallel branches in the graph (2+ groups)
  bool has_branches = false;
  PlanFinal fin{nullptr, nullptr};  // accumulators of launches that close themselves
  cudaGraphExec_t exec = nullptr;
  unsigned long long* exec_sse = nullptr;
  double* exec_psnr = nullptr;
  std::mutex mu;
};

namespace {

// Autotuner of TDCT_PATH_AUTO plans: runs every candidate (engine x CTAs per
// SM) on the plan's own planes (reconstructions are written, SSE goes to a
// scratch buffer) and keeps the fastest.  Two untimed runs, then the median
// of three timed runs per candidate, on the plan's private stream.
int autotune_plan(tdct_plan* plan) {
  bool any_u8_bulk = false;
  for (const Group& g : plan->groups) any_u8_bulk |= (g.any_bulk && g.dtype == TDCT_U8);
  struct Cand { int path, cps, variant; };
  std::vector<Cand> cands = {{TDCT_PATH_BUTTERFLY, 0, 0}, {TDCT_PATH_BUTTERFLY, 2, 0}};
  if (any_u8_bulk) {
    const uint16_t* table = nullptr;
    if (tc_prepare(&table) == cudaSuccess) {
      cands.push_back({TDCT_PATH_TENSOR, 0, 0});
      cands.push_back({TDCT_PATH_TENSOR, 3, 0});
      cands.push_back({TDCT_PATH_TENSOR, 0, 1});
    }
  }
  cudaStream_t s = plan->capture_stream;
  unsigned long long* sse = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&sse),
                                  sizeof(unsigned long long) * plan->nplanes, s);
  if (e != cudaSuccess) return fail(TDCT_ENOMEM, "autotune scratch: %s", cudaGetErrorString(e));
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  float best = 3.4e38f;
  Cand pick = cands[0];
  for (const Cand& c : cands) {
    float t[3] = {0, 0, 0};
    for (int it = 0; it < 5 && e == cudaSuccess; ++it) {
      if (it >= 2) e = cudaEventRecord(ev0, s);
      if (e == cudaSuccess)
        e = enqueue_batch(plan->tr, plan->groups, plan->d_descs, plan->d_npix, plan->nplanes, sse,
                          nullptr, s, c.path, c.cps, c.variant);
      if (e == cudaSuccess && it >= 2) e = cudaEventRecord(ev1, s);
      if (e == cudaSuccess && it >= 2) e = cudaEventSynchronize(ev1);
      if (e == cudaSuccess && it >= 2) e = cudaEventElapsedTime(&t[it - 2], ev0, ev1);
    }
    if (e != cudaSuccess) break;
    std::sort(t, t + 3);
    if (t[1] < best) {
      best = t[1];
      pick = c;
    }
  }
  cudaFreeAsync(sse, s);
  const cudaError_t es = cudaStreamSynchronize(s);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (e != cudaSuccess) return cuda_fail(e, "autotune");
  if (es != cudaSuccess) return cuda_fail(es, "autotune");
  plan->path = pick.path == TDCT_PATH_TENSOR && pick.variant == 1 ? TDCT_PATH_TENSOR_PIPELINED
                                                                   : pick.path;
  plan->ctas_per_sm = pick.cps;
  plan->tc_variant = pick.variant;
  plan->tuned_ms = best;
  return TDCT_OK;
}

}  // namespace

extern "C" {

const char* tdct_last_error(void) { return g_err.c_str(); }

const char* tdct_version(void) { return "tdct 0.1 (sm_103a)"; }

int tdct_forward(const void* d_img, int64_t pitch, int H, int W, int dtype, const int8_t T[64],
                 const int32_t n[8], int32_t* d_coef, tdct_stream_t stream) {
  Transform tr;
  int rc = resolve_transform(T, n, &tr);
  if (rc) return rc;
  if ((rc = check_plane(d_img, pitch, H, W, dtype, "tdct_forward"))) return rc;
  if (!d_coef || (reinterpret_cast<uintptr_t>(d_coef) & 3))
    return fail(TDCT_EINVAL, "tdct_forward: d_coef NULL or not 4-byte aligned");
  const PlaneDesc P = make_desc(d_img, pitch, H, W, dtype, 64, nullptr, 0, 0);
  const int vec = (reinterpret_cast<uintptr_t>(d_coef) & 15) == 0;
  const int grid = grid_for((int64_t)P.nbx * P.nby, 128);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!tr.t1) {
    const cudaError_t eg = launch_forward_generic(P, generic_for_r(tr, 64), d_coef, s, grid);
    return eg == cudaSuccess ? TDCT_OK : cuda_fail(eg, "tdct_forward launch");
  }
  if (dtype == TDCT_U8) forward_kernel<0><<<grid, 128, 0, s>>>(P, d_coef, vec);
  else forward_kernel<1><<<grid, 128, 0, s>>>(P, d_coef, vec);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TDCT_OK : cuda_fail(e, "tdct_forward launch");
}

int tdct_zonal_inverse(const int32_t* d_coef, int H, int W, int dtype, const int8_t T[64],
                       const int32_t n[8], int r, void* d_out, int64_t out_pitch,
                       tdct_stream_t stream) {
  Transform tr;
  int rc = resolve_transform(T, n, &tr);
  if (rc) return rc;
  if ((rc = check_r(r))) return rc;
  if ((rc = check_plane(d_out, out_pitch, H, W, dtype, "tdct_zonal_inverse"))) return rc;
  if (!d_coef || (reinterpret_cast<uintptr_t>(d_coef) & 3))
    return fail(TDCT_EINVAL, "tdct_zonal_inverse: d_coef NULL or not 4-byte aligned");
  const PlaneDesc P = make_desc(d_out, out_pitch, H, W, dtype, r, d_out, out_pitch, 0);
  const int vec = (reinterpret_cast<uintptr_t>(d_coef) & 15) == 0;
  const int grid = grid_for((int64_t)P.nbx * P.nby, 128);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!tr.t1) {
    const cudaError_t eg = launch_inverse_generic(d_coef, P, generic_for_r(tr, r), s, grid);
    return eg == cudaSuccess ? TDCT_OK : cuda_fail(eg, "tdct_zonal_inverse launch");
  }
  const CodecParams cp = make_params(r);
  if (dtype == TDCT_U8) inverse_kernel<0><<<grid, 128, 0, s>>>(d_coef, P, cp, vec);
  else inverse_kernel<1><<<grid, 128, 0, s>>>(d_coef, P, cp, vec);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TDCT_OK : cuda_fail(e, "tdct_zonal_inverse launch");
}

int tdct_codec_error(const void* d_img, int64_t pitch, int H, int W, int dtype,
                     const int8_t T[64], const int32_t n[8], int r, void* d_recon,
                     int64_t recon_pitch, uint64_t* d_sse, double* d_psnr,
                     tdct_stream_t stream) {
  Transform tr;
  int rc = resolve_transform(T, n, &tr);
  if (rc) return rc;
  if ((rc = check_r(r))) return rc;
  if ((rc = check_plane(d_img, pitch, H, W, dtype, "tdct_codec_error"))) return rc;
  if (d_recon && (rc = check_plane(d_recon, recon_pitch, H, W, dtype, "recon"))) return rc;
  if (!d_sse || (reinterpret_cast<uintptr_t>(d_sse) & 7))
    return fail(TDCT_EINVAL, "d_sse NULL or not 8-byte aligned");
  if (d_psnr && (reinterpret_cast<uintptr_t>(d_psnr) & 7))
    return fail(TDCT_EINVAL, "d_psnr not 8-byte aligned");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  PlaneTable tab;
  std::memset(&tab, 0, sizeof tab);
  tab.d = nullptr;
  tab.n = 1;
  tab.one = make_desc(d_img, pitch, H, W, dtype, r, d_recon, recon_pitch, 0);
  tab.total_units = units_of(tab.one);
  tab.any_bulk = (tab.one.vec16 & 4) ? 1 : 0;
  tab.shifted = (tab.one.vec16 & 16) ? 1 : 0;
  tab.staged = (tab.one.vec16 & 8) ? 1 : 0;
  unsigned long long* sse = reinterpret_cast<unsigned long long*>(d_sse);
  cudaError_t e = cudaMemsetAsync(sse, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return cuda_fail(e, "tdct_codec_error memset");
  e = tr.t1 ? dispatch_codec(r, dtype, tab, sse, 0, s)
            : dispatch_codec_generic(r, dtype, tab, tr, sse, s);
  if (e != cudaSuccess) return cuda_fail(e, "tdct_codec_error launch");
  if (d_psnr) {
    psnr_kernel<<<1, 32, 0, s>>>(sse, nullptr, (int64_t)H * W, d_psnr, 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "psnr launch");
  }
  return TDCT_OK;
}

int tdct_codec_error_batched(const tdct_plane* planes, int nplanes, const int8_t T[64],
                             const int32_t n[8], uint64_t* d_sse, double* d_psnr, int path,
                             tdct_stream_t stream) {
  Transform tr;
  int rc = resolve_transform(T, n, &tr);
  if (rc) return rc;
  if ((rc = check_engine(tr, path))) return rc;
  if (!d_sse || (reinterpret_cast<uintptr_t>(d_sse) & 7))
    return fail(TDCT_EINVAL, "d_sse NULL or not 8-byte aligned");
  std::vector<PlaneDesc> descs;
  std::vector<Group> groups;
  std::vector<int64_t> npix;
  if ((rc = build_batch(planes, nplanes, descs, groups, npix, wrap_allowed(tr, path)))) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (path == TDCT_PATH_TENSOR || path == TDCT_PATH_TENSOR_PIPELINED) {
    const uint16_t* table = nullptr;
    const cudaError_t et = tc_prepare(&table);
    if (et != cudaSuccess) return cuda_fail(et, "tensor-core weight tables");
  }
  // Stream-ordered scratch for the block-offset table, freed after the kernels.
  const size_t bytes_desc = sizeof(PlaneDesc) * descs.size();
  const size_t bytes_npix = sizeof(int64_t) * npix.size();
  void* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, bytes_desc + bytes_npix, s);
  if (e != cudaSuccess) return fail(TDCT_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e));
  PlaneDesc* d_descs = static_cast<PlaneDesc*>(scratch);
  int64_t* d_npix = reinterpret_cast<int64_t*>(static_cast<char*>(scratch) + bytes_desc);
  if ((e = cudaMemcpyAsync(d_descs, descs.data(), bytes_desc, cudaMemcpyHostToDevice, s)) ==
          cudaSuccess &&
      (e = cudaMemcpyAsync(d_npix, npix.data(), bytes_npix, cudaMemcpyHostToDevice, s)) ==
          cudaSuccess)
    e = enqueue_batch(tr, groups, d_descs, d_npix, nplanes,
                      reinterpret_cast<unsigned long long*>(d_sse), d_psnr, s, path);
  const cudaError_t ef = cudaFreeAsync(scratch, s);
  if (e != cudaSuccess) return cuda_fail(e, "tdct_codec_error_batched");
  if (ef != cudaSuccess) return cuda_fail(ef, "cudaFreeAsync");
  return TDCT_OK;
}

int tdct_plan_create(const tdct_plane* planes, int nplanes, const int8_t T[64],
                     const int32_t n[8], int path, tdct_plan** out_plan) {
  if (!out_plan) return fail(TDCT_EINVAL, "out_plan is NULL");
  *out_plan = nullptr;
  Transform tr;
  int rc = resolve_transform(T, n, &tr);
  if (rc) return rc;
  if ((rc = check_engine(tr, path))) return rc;
  std::vector<PlaneDesc> descs;
  std::vector<int64_t> npix;
  tdct_plan* plan = new (std::nothrow) tdct_plan;
  if (!plan) return fail(TDCT_ENOMEM, "host allocation failed");
  plan->tr = tr;
  if ((rc = build_batch(planes, nplanes, descs, plan->groups, npix, wrap_allowed(tr, path)))) {
    delete plan;
    return rc;
  }
  plan->nplanes = nplanes;
  plan->path = path;
  if (path == TDCT_PATH_TENSOR || path == TDCT_PATH_TENSOR_PIPELINED) {
    const uint16_t* table = nullptr;
    const cudaError_t et = tc_prepare(&table);
    if (et != cudaSuccess) {
      delete plan;
      return cuda_fail(et, "tensor-core weight tables");
    }
  }
  cudaError_t e = cudaMalloc(&plan->d_descs, sizeof(PlaneDesc) * descs.size());
  if (e == cudaSuccess) e = cudaMalloc(&plan->d_npix, sizeof(int64_t) * npix.size());
  if (e == cudaSuccess) e = cudaMalloc(&plan->fin.acc, sizeof(unsigned long long) * nplanes);
  if (e == cudaSuccess) e = cudaMalloc(&plan->fin.cnt, sizeof(unsigned int) * nplanes);
  if (e == cudaSuccess) e = cudaMemset(plan->fin.acc, 0, sizeof(unsigned long long) * nplanes);
  if (e == cudaSuccess) e = cudaMemset(plan->fin.cnt, 0, sizeof(unsigned int) * nplanes);
  if (e != cudaSuccess) {
    tdct_plan_destroy(plan);
    return fail(TDCT_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
  }
  e = cudaMemcpy(plan->d_descs, descs.data(), sizeof(PlaneDesc) * descs.size(),
                 cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(plan->d_npix, npix.data(), sizeof(int64_t) * npix.size(),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&plan->capture_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess && plan->groups.size() > 1) {
    plan->has_branches = true;
    e = cudaEventCreateWithFlags(&plan->branches.fork, cudaEventDisableTiming);
    for (int b = 0; b < kPlanBranches && e == cudaSuccess; ++b) {
      e = cudaStreamCreateWithFlags(&plan->branches.stream[b], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&plan->branches.join[b], cudaEventDisableTiming);
    }
  }
  if (e != cudaSuccess) {
    tdct_plan_destroy(plan);
    return cuda_fail(e, "tdct_plan_create");
  }
  if (path == TDCT_PATH_AUTO) {
    plan->path = TDCT_PATH_BUTTERFLY;
    // another T has one engine (the generic kernels): nothing to tune
    if (tr.t1 && (rc = autotune_plan(plan))) {
      tdct_plan_destroy(plan);
      return rc;
    }
  }
  *out_plan = plan;
  return TDCT_OK;
}

int tdct_plan_config(const tdct_plan* plan, int* path, int* ctas_per_sm, float* tuned_ms) {
  if (!plan) return fail(TDCT_EINVAL, "plan is NULL");
  if (path) *path = plan->path;
  if (ctas_per_sm) *ctas_per_sm = plan->ctas_per_sm;
  if (tuned_ms) *tuned_ms = plan->tuned_ms;
  return TDCT_OK;
}

int tdct_plan_groups(const tdct_plan* plan, tdct_plan_group* out, int max, int* count) {
  if (!plan || !count || max < 0) return fail(TDCT_EINVAL, "plan or count NULL, or max < 0");
  const int n = (int)plan->groups.size();
  *count = n;
  for (int i = 0; i < n && i < max && out; ++i) {
    const Group& g = plan->groups[i];
    out[i].dtype = g.dtype;
    out[i].r = g.r;
    out[i].load = !plan->tr.t1 ? TDCT_LOAD_PLAIN
                  : g.any_bulk ? TDCT_LOAD_BULK
                  : g.staged   ? TDCT_LOAD_STAGED
                               : TDCT_LOAD_PLAIN;
    out[i].planes = g.count;
  }
  return TDCT_OK;
}

}  // extern "C"

namespace {
// Whether every launch of the plan runs the u8 bulk-copy ring kernel, which
// then writes SSE and PSNR itself (one kernel node per group, nothing else).
bool plan_self_closing(const tdct_plan* plan) {
  for (const Group& g : plan->groups)
    if (!group_on_u8_ring(plan->tr, g, plan->path)) return false;
  return true;
}
}  // namespace

extern "C" {

int tdct_plan_kernel_count(const tdct_plan* plan) {
  if (!plan) return 0;
  return (int)plan->groups.size() + (plan_self_closing(plan) ? 0 : 1);
}

int tdct_plan_launch(tdct_plan* plan, uint64_t* d_sse, double* d_psnr, tdct_stream_t stream) {
  if (!plan) return fail(TDCT_EINVAL, "plan is NULL");
  if (!d_sse || (reinterpret_cast<uintptr_t>(d_sse) & 7))
    return fail(TDCT_EINVAL, "d_sse NULL or not 8-byte aligned");
  std::lock_guard<std::mutex> lock(plan->mu);
  unsigned long long* sse = reinterpret_cast<unsigned long long*>(d_sse);
  cudaError_t e = cudaSuccess;
  if (!plan->exec || plan->exec_sse != sse || plan->exec_psnr != d_psnr) {
    if (plan->exec) {
      cudaGraphExecDestroy(plan->exec);
      plan->exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(plan->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    const cudaError_t ee = enqueue_batch(plan->tr, plan->groups, plan->d_descs, plan->d_npix,
                                         plan->nplanes, sse, d_psnr, plan->capture_stream,
                                         plan->path, plan->ctas_per_sm, plan->tc_variant,
                                         plan->has_branches ? &plan->branches : nullptr,
                                         plan_self_closing(plan) ? &plan->fin : nullptr);
    e = cudaStreamEndCapture(plan->capture_stream, &graph);
    if (ee != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(ee, "plan capture");
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&plan->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      plan->exec = nullptr;
      return cuda_fail(e, "cudaGraphInstantiate");
    }
    plan->exec_sse = sse;
    plan->exec_psnr = d_psnr;
  }
  e = cudaGraphLaunch(plan->exec, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? TDCT_OK : cuda_fail(e, "cudaGraphLaunch");
}

void tdct_plan_destroy(tdct_plan* plan) {
  if (!plan) return;
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->capture_stream) cudaStreamDestroy(plan->capture_stream);
  for (int b = 0; b < kPlanBranches; ++b) {
    if (plan->branches.stream[b]) cudaStreamDestroy(plan->branches.stream[b]);
    if (plan->branches.join[b]) cudaEventDestroy(plan->branches.join[b]);
  }
  if (plan->branches.fork) cudaEventDestroy(plan->branches.fork);
  if (plan->d_descs) cudaFree(plan->d_descs);
  if (plan->d_npix) cudaFree(plan->d_npix);
  if (plan->fin.acc) cudaFree(plan->fin.acc);
  if (plan->fin.cnt) cudaFree(plan->fin.cnt);
  delete plan;
}

// ---- batch without device allocation -------------------------------------------
// The block-offset table of tdct_codec_error_batched_noalloc: descriptors,
// then the per-plane sample counts, in one fixed device array.
}  // extern "C"

namespace {
constexpr size_t kNoAllocDescBytes = sizeof(tdct::PlaneDesc) * TDCT_NOALLOC_MAX_PLANES;
constexpr size_t kNoAllocBytes = kNoAllocDescBytes + sizeof(int64_t) * TDCT_NOALLOC_MAX_PLANES;
}  // namespace
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_addr[256] = {};
// Held by each no-alloc call from its first table copy to its last launch,
// so that calls from several host threads enqueue their table and their
// kernels as one sequence (the table is shared).
std::mutex g_noalloc_call_mu;

// Device address of g_noalloc_scratch on the current device (looked up once
// per device; the host-side symbol is not a device address).
int noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 256) return fail(TDCT_EINVAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc table)");
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return TDCT_OK;
}

// Library-owned transfer streams of tdct_codec_error_batched_host, one pair
// per device, created on first use.
struct HostStreams {
  cudaStream_t h2d = nullptr, d2h = nullptr;
};
std::mutex g_host_mu;
HostStreams g_host_streams[256];

int host_streams(HostStreams* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 256) return fail(TDCT_EINVAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_host_mu);
  HostStreams& hs = g_host_streams[dev];
  if (!hs.h2d && (e = cudaStreamCreateWithFlags(&hs.h2d, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e, "transfer stream");
  if (!hs.d2h && (e = cudaStreamCreateWithFlags(&hs.d2h, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e, "transfer stream");
  *out = hs;
  return TDCT_OK;
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Copies between host planes and their staged images: planes whose rows are
// contiguous and that follow each other without a gap both on the host and
// in the staging buffer are merged into one linear copy (one DMA request
// instead of one per plane); other planes take a 2-D copy each.
// `host_of(i)` / `host_pitch(i)` give plane i's host side (input or
// reconstruction).
template <typename HostOf, typename PitchOf>
cudaError_t copy_planes(const tdct_plane* planes, int first, int count, uint8_t* staged,
                        const std::vector<size_t>& off, const std::vector<int64_t>& dpitch,
                        HostOf host_of, PitchOf host_pitch, bool to_device, cudaStream_t st,
                        int* failed_plane) {
  int k = 0;
  while (k < count) {
    const int i = first + k;
    const tdct_plane& p = planes[i];
    const size_t row = (size_t)p.W * (p.dtype == TDCT_I16 ? 2 : 1);
    uint8_t* h = static_cast<uint8_t*>(const_cast<void*>(host_of(i)));
    if (!h) {
      ++k;
      continue;
    }
    const bool linear = (size_t)host_pitch(i) == row && (size_t)dpitch[i] == row;
    if (!linear) {
      const cudaError_t e =
          to_device ? cudaMemcpy2DAsync(staged + off[i], (size_t)dpitch[i], h, (size_t)host_pitch(i),
                                        row, (size_t)p.H, cudaMemcpyHostToDevice, st)
                    : cudaMemcpy2DAsync(h, (size_t)host_pitch(i), staged + off[i], (size_t)dpitch[i],
                                        row, (size_t)p.H, cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) {
        *failed_plane = i;
        return e;
      }
      ++k;
      continue;
    }
    size_t bytes = row * (size_t)p.H;
    int m = k + 1;
    while (m < count) {
      const int j = first + m;
      const tdct_plane& q = planes[j];
      const size_t qrow = (size_t)q.W * (q.dtype == TDCT_I16 ? 2 : 1);
      const uint8_t* hq = static_cast<const uint8_t*>(host_of(j));
      if (!hq || (size_t)host_pitch(j) != qrow || (size_t)dpitch[j] != qrow || hq != h + bytes ||
          off[j] != off[i] + bytes)
        break;
      bytes += qrow * (size_t)q.H;
      ++m;
    }
    auto linear_copy = [&](int j, size_t n) {
      uint8_t* hj = static_cast<uint8_t*>(const_cast<void*>(host_of(j)));
      return to_device ? cudaMemcpyAsync(staged + off[j], hj, n, cudaMemcpyHostToDevice, st)
                       : cudaMemcpyAsync(hj, staged + off[j], n, cudaMemcpyDeviceToHost, st);
    };
    cudaError_t e = linear_copy(i, bytes);
    if (e == cudaErrorInvalidValue && m > k + 1) {
      // Adjacent planes from different host allocations: the CUDA driver rejects
      // a range that crosses page-locked allocations (argument check,
      // nothing enqueued).  Clear that error and copy the run plane by plane.
      (void)cudaGetLastError();
      e = cudaSuccess;
      for (int t = k; t < m && e == cudaSuccess; ++t) {
        const tdct_plane& q = planes[first + t];
        e = linear_copy(first + t, (size_t)q.W * (q.dtype == TDCT_I16 ? 2 : 1) * (size_t)q.H);
        if (e != cudaSuccess) *failed_plane = first + t;
      }
      if (e != cudaSuccess) return e;
    } else if (e != cudaSuccess) {
      *failed_plane = i;
      return e;
    }
    k = m;
  }
  return cudaSuccess;
}
}  // namespace

extern "C" {

int tdct_codec_error_batched_noalloc(const tdct_plane* planes, int nplanes, const int8_t T[64],
                                     const int32_t n[8], uint64_t* d_sse, double* d_psnr,
                                     tdct_stream_t stream) {
  Transform tr;
  int rc = resolve_transform(T, n, &tr);
  if (rc) return rc;
  if (nplanes > TDCT_NOALLOC_MAX_PLANES)
    return fail(TDCT_EINVAL,
                "tdct_codec_error_batched_noalloc: %d planes exceed its fixed table of %d planes "
                "(use tdct_codec_error_batched or split the batch)",
                nplanes, TDCT_NOALLOC_MAX_PLANES);
  if (!d_sse || (reinterpret_cast<uintptr_t>(d_sse) & 7))
    return fail(TDCT_EINVAL, "d_sse NULL or not 8-byte aligned");
  std::vector<PlaneDesc> descs;
  std::vector<Group> groups;
  std::vector<int64_t> npix;
  if ((rc = build_batch(planes, nplanes, descs, groups, npix, wrap_allowed(tr, TDCT_PATH_AUTO))))
    return rc;
  void* scratch = nullptr;
  if ((rc = noalloc_scratch(&scratch))) return rc;
  PlaneDesc* d_descs = static_cast<PlaneDesc*>(scratch);
  int64_t* d_npix = reinterpret_cast<int64_t*>(static_cast<char*>(scratch) + kNoAllocDescBytes);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> call_lock(g_noalloc_call_mu);
  cudaError_t e = cudaMemcpyAsync(d_descs, descs.data(), sizeof(PlaneDesc) * descs.size(),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_npix, npix.data(), sizeof(int64_t) * npix.size(),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = enqueue_batch(tr, groups, d_descs, d_npix, nplanes,
                      reinterpret_cast<unsigned long long*>(d_sse), d_psnr, s);
  return e == cudaSuccess ? TDCT_OK : cuda_fail(e, "tdct_codec_error_batched_noalloc");
}

int tdct_codec_error_batched_host(const tdct_plane* planes, int nplanes, const int8_t T[64],
                                  const int32_t n[8], uint64_t* h_sse, double* h_psnr,
                                  size_t chunk_bytes, tdct_stream_t stream) {
  Transform tr;
  int rc = resolve_transform(T, n, &tr);
  if (rc) return rc;
  if (!planes || nplanes < 1 || nplanes > (1 << 20))
    return fail(TDCT_EINVAL, "nplanes = %d outside 1..2^20 (or planes is NULL)", nplanes);
  if (!h_sse) return fail(TDCT_EINVAL, "h_sse is NULL");
  if (chunk_bytes == 0) chunk_bytes = (size_t)64 << 20;

  // Staged layout: each plane row-contiguous with a 16-byte multiple pitch
  // (u8 planes with W % 16 == 0 and H % 8 == 0 then take the bulk-copy
  // ring), 256-byte aligned, packed into chunks of consecutive planes.
  std::vector<size_t> off(nplanes);
  std::vector<int64_t> dpitch(nplanes);
  std::vector<int> chunk_first;
  size_t cur = 0, max_chunk = 0;
  bool any_recon = false;
  for (int i = 0; i < nplanes; ++i) {
    const tdct_plane& p = planes[i];
    char what[64];
    std::snprintf(what, sizeof what, "plane %d", i);
    if ((rc = check_plane(p.img, p.pitch, p.H, p.W, p.dtype, what))) return rc;
    if (p.r < 1 || p.r > 64) return fail(TDCT_EINVAL, "plane %d: r = %d outside 1..64", i, p.r);
    if (p.recon && p.recon_pitch < (int64_t)p.W * sample_bytes(p.dtype))
      return fail(TDCT_EINVAL, "plane %d: recon pitch too small", i);
    dpitch[i] = (int64_t)round_up((size_t)p.W * sample_bytes(p.dtype), 16);
    const size_t bytes = round_up((size_t)dpitch[i] * p.H, 256);
    if (i == 0 || (cur > 0 && cur + bytes > chunk_bytes)) {
      chunk_first.push_back(i);
      cur = 0;
    }
    off[i] = cur;
    cur += bytes;
    max_chunk = std::max(max_chunk, cur);
    any_recon |= p.recon != nullptr;
  }
  const int nchunks = (int)chunk_first.size();
  chunk_first.push_back(nplanes);

  HostStreams hs;
  if ((rc = host_streams(&hs))) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

  // One stream-ordered block: 2 input buffers, 2 reconstruction buffers (if
  // any), the descriptor table and sample counts, SSE and PSNR.
  const size_t bytes_desc = round_up(sizeof(PlaneDesc) * nplanes, 256);
  const size_t bytes_npix = round_up(sizeof(int64_t) * nplanes, 256);
  const size_t bytes_res = round_up(sizeof(uint64_t) * nplanes, 256);
  const size_t nbuf = any_recon ? 4 : 2;
  const size_t total = nbuf * max_chunk + bytes_desc + bytes_npix + 2 * bytes_res;
  void* block = nullptr;
  cudaError_t e = cudaMallocAsync(&block, total, s);
  if (e != cudaSuccess) return fail(TDCT_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e));
  uint8_t* base = static_cast<uint8_t*>(block);
  uint8_t* in_buf[2] = {base, base + max_chunk};
  uint8_t* out_buf[2] = {any_recon ? base + 2 * max_chunk : nullptr,
                         any_recon ? base + 3 * max_chunk : nullptr};
  PlaneDesc* d_descs = reinterpret_cast<PlaneDesc*>(base + nbuf * max_chunk);
  int64_t* d_npix = reinterpret_cast<int64_t*>(base + nbuf * max_chunk + bytes_desc);
  unsigned long long* d_sse =
      reinterpret_cast<unsigned long long*>(base + nbuf * max_chunk + bytes_desc + bytes_npix);
  double* d_psnr = reinterpret_cast<double*>(base + nbuf * max_chunk + bytes_desc + bytes_npix +
                                             bytes_res);

  // Per-chunk block-offset tables over the staged planes (slots relative to
  // the chunk), all uploaded at once.
  std::vector<PlaneDesc> descs(nplanes);
  std::vector<int64_t> npix(nplanes);
  std::vector<std::vector<Group>> groups(nchunks);
  for (int c = 0; c < nchunks && rc == TDCT_OK; ++c) {
    const int first = chunk_first[c], count = chunk_first[c + 1] - first;
    std::vector<tdct_plane> staged(count);
    for (int k = 0; k < count; ++k) {
      const tdct_plane& p = planes[first + k];
      staged[k] = p;
      staged[k].img = in_buf[c & 1] + off[first + k];
      staged[k].pitch = dpitch[first + k];
      staged[k].recon = p.recon ? out_buf[c & 1] + off[first + k] : nullptr;
      staged[k].recon_pitch = p.recon ? dpitch[first + k] : 0;
    }
    std::vector<PlaneDesc> dc;
    std::vector<int64_t> nc;
    rc = build_batch(staged.data(), count, dc, groups[c], nc, wrap_allowed(tr, TDCT_PATH_AUTO));
    if (rc == TDCT_OK) {
      std::copy(dc.begin(), dc.end(), descs.begin() + first);
      std::copy(nc.begin(), nc.end(), npix.begin() + first);
    }
  }
  cudaEvent_t ev_start = nullptr, ev_end_d2h = nullptr, ev_h2d[2] = {}, ev_comp[2] = {},
              ev_d2h[2] = {};
  auto make_events = [&]() -> cudaError_t {
    cudaError_t x = cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming);
    if (x == cudaSuccess) x = cudaEventCreateWithFlags(&ev_end_d2h, cudaEventDisableTiming);
    for (int b = 0; b < 2 && x == cudaSuccess; ++b) {
      x = cudaEventCreateWithFlags(&ev_h2d[b], cudaEventDisableTiming);
      if (x == cudaSuccess) x = cudaEventCreateWithFlags(&ev_comp[b], cudaEventDisableTiming);
      if (x == cudaSuccess) x = cudaEventCreateWithFlags(&ev_d2h[b], cudaEventDisableTiming);
    }
    return x;
  };
  int bad_plane = -1;
  const char* what = "setup";
  if (rc == TDCT_OK) {
    e = make_events();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_descs, descs.data(), sizeof(PlaneDesc) * nplanes,
                          cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_npix, npix.data(), sizeof(int64_t) * nplanes, cudaMemcpyHostToDevice,
                          s);
    if (e == cudaSuccess) e = cudaEventRecord(ev_start, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hs.h2d, ev_start, 0);
    if (e == cudaSuccess && any_recon) e = cudaStreamWaitEvent(hs.d2h, ev_start, 0);
    for (int c = 0; c < nchunks && e == cudaSuccess; ++c) {
      const int b = c & 1, first = chunk_first[c], count = chunk_first[c + 1] - first;
      // input buffer b is free once chunk c - 2 has been coded
      if (c >= 2) e = cudaStreamWaitEvent(hs.h2d, ev_comp[b], 0);
      if (e == cudaSuccess)
        e = copy_planes(
            planes, first, count, in_buf[b], off, dpitch,
            [&](int i) { return planes[i].img; }, [&](int i) { return planes[i].pitch; }, true,
            hs.h2d, &bad_plane);
      if (e != cudaSuccess) what = "copy to the device";
      if (e == cudaSuccess) e = cudaEventRecord(ev_h2d[b], hs.h2d);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_h2d[b], 0);
      // reconstruction buffer b is free once chunk c - 2's copies back are done
      if (e == cudaSuccess && any_recon && c >= 2) e = cudaStreamWaitEvent(s, ev_d2h[b], 0);
      if (e == cudaSuccess) {
        e = enqueue_batch(tr, groups[c], d_descs + first, d_npix + first, count, d_sse + first,
                          h_psnr ? d_psnr + first : nullptr, s);
        if (e != cudaSuccess) what = "codec launch";
      }
      if (e == cudaSuccess) e = cudaEventRecord(ev_comp[b], s);
      if (e == cudaSuccess && any_recon) {
        e = cudaStreamWaitEvent(hs.d2h, ev_comp[b], 0);
        if (e == cudaSuccess)
          e = copy_planes(
              planes, first, count, out_buf[b], off, dpitch,
              [&](int i) { return static_cast<const void*>(planes[i].recon); },
              [&](int i) { return planes[i].recon_pitch; }, false, hs.d2h, &bad_plane);
        if (e != cudaSuccess) what = "copy of the reconstruction";
        if (e == cudaSuccess) e = cudaEventRecord(ev_d2h[b], hs.d2h);
      }
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h_sse, d_sse, sizeof(uint64_t) * nplanes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && h_psnr)
      e = cudaMemcpyAsync(h_psnr, d_psnr, sizeof(double) * nplanes, cudaMemcpyDeviceToHost, s);
  }
  // `stream` waits for everything the transfer streams hold (also after a
  // failed enqueue), so the block is released in stream order after its
  // last use.
  cudaError_t ew = cudaSuccess;
  if (ev_start) {
    ew = cudaEventRecord(ev_h2d[0], hs.h2d);
    if (ew == cudaSuccess) ew = cudaStreamWaitEvent(s, ev_h2d[0], 0);
    if (ew == cudaSuccess && any_recon) ew = cudaEventRecord(ev_end_d2h, hs.d2h);
    if (ew == cudaSuccess && any_recon) ew = cudaStreamWaitEvent(s, ev_end_d2h, 0);
  }
  const cudaError_t ef = cudaFreeAsync(block, s);
  for (cudaEvent_t ev : {ev_start, ev_end_d2h, ev_h2d[0], ev_h2d[1], ev_comp[0], ev_comp[1],
                         ev_d2h[0], ev_d2h[1]})
    if (ev) cudaEventDestroy(ev);
  if (rc) return rc;
  if (e != cudaSuccess)
    return fail(TDCT_ECUDA, "tdct_codec_error_batched_host: %s%s%s: %s", what,
                bad_plane >= 0 ? " of plane " : "",
                bad_plane >= 0 ? std::to_string(bad_plane).c_str() : "", cudaGetErrorString(e));
  if (ew != cudaSuccess) return cuda_fail(ew, "tdct_codec_error_batched_host: stream join");
  if (ef != cudaSuccess) return cuda_fail(ef, "cudaFreeAsync");
  return TDCT_OK;
}

int tdct_ssim_batched(const tdct_ssim_plane* planes, int nplanes, double* d_mssim,
                      tdct_stream_t stream) {
  if (!planes || nplanes < 1 || nplanes > (1 << 20))
    return fail(TDCT_EINVAL, "nplanes = %d outside 1..2^20 (or planes is NULL)", nplanes);
  if (!d_mssim || (reinterpret_cast<uintptr_t>(d_mssim) & 7))
    return fail(TDCT_EINVAL, "d_mssim NULL or not 8-byte aligned");
  std::vector<SsimDesc> descs(nplanes);
  int64_t units = 0;
  for (int i = 0; i < nplanes; ++i) {
    const tdct_ssim_plane& p = planes[i];
    if (!p.x || !p.y) return fail(TDCT_EINVAL, "plane %d: NULL plane pointer", i);
    if (p.H < kSsimWin || p.W < kSsimWin || p.H > (1 << 28) || p.W > (1 << 28))
      return fail(TDCT_EINVAL, "plane %d: size %d x %d (SSIM needs at least 11 x 11)", i, p.H,
                  p.W);
    if (p.x_pitch < p.W || p.y_pitch < p.W)
      return fail(TDCT_EINVAL, "plane %d: pitch below W", i);
    SsimDesc& d = descs[i];
    std::memset(&d, 0, sizeof d);
    d.x = static_cast<const uint8_t*>(p.x);
    d.y = static_cast<const uint8_t*>(p.y);
    d.xpitch = p.x_pitch;
    d.ypitch = p.y_pitch;
    d.H = p.H;
    d.W = p.W;
    d.strips = (p.W - (kSsimWin - 1) + kSsimStrip - 1) / kSsimStrip;
    d.bands = (p.H - (kSsimWin - 1) + kSsimBand - 1) / kSsimBand;
    d.unit_begin = units;
    d.slot = i;
    units += (int64_t)d.strips * d.bands;
  }
  // window of Wang et al. (2004): g_j = exp(-(j - 5)^2 / (2 * 1.5^2)), unit sum
  SsimParams sp;
  double g[kSsimWin], gs = 0.0;
  for (int j = 0; j < kSsimWin; ++j) {
    const double t = j - (kSsimWin - 1) / 2;
    g[j] = std::exp(-t * t / (2.0 * 1.5 * 1.5));
    gs += g[j];
  }
  for (int j = 0; j < kSsimWin; ++j) sp.g[j] = (float)(g[j] / gs);
  sp.C1 = (float)((0.01 * 255.0) * (0.01 * 255.0));
  sp.C2 = (float)((0.03 * 255.0) * (0.03 * 255.0));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  void* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, sizeof(SsimDesc) * nplanes, s);
  if (e != cudaSuccess) return fail(TDCT_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e));
  SsimDesc* d_descs = static_cast<SsimDesc*>(scratch);
  e = cudaMemcpyAsync(d_descs, descs.data(), sizeof(SsimDesc) * nplanes, cudaMemcpyHostToDevice,
                      s);
  if (e == cudaSuccess) e = launch_ssim(d_descs, nplanes, units, sp, d_mssim, s);
  const cudaError_t ef = cudaFreeAsync(scratch, s);
  if (e != cudaSuccess) return cuda_fail(e, "tdct_ssim_batched");
  if (ef != cudaSuccess) return cuda_fail(ef, "cudaFreeAsync");
  return TDCT_OK;
}

int tdct_codec_error_jam(const void* d_img, int64_t pitch, int H, int W, int dtype, int B,
                         const int8_t* T, const int32_t* n, int r, void* d_recon,
                         int64_t recon_pitch, uint64_t* d_sse, double* d_psnr,
                         tdct_stream_t stream) {
  if (B != 16 && B != 32) return fail(TDCT_EINVAL, "B = %d is neither 16 nor 32", B);
  if (!T || !n) return fail(TDCT_EINVAL, "T and n must not be NULL");
  if (r < 1 || r > B * B) return fail(TDCT_EINVAL, "r = %d outside 1..%d", r, B * B);
  int rc = check_plane(d_img, pitch, H, W, dtype, "tdct_codec_error_jam");
  if (rc) return rc;
  if (d_recon && (rc = check_plane(d_recon, recon_pitch, H, W, dtype, "recon"))) return rc;
  if (!d_sse || (reinterpret_cast<uintptr_t>(d_sse) & 7))
    return fail(TDCT_EINVAL, "d_sse NULL or not 8-byte aligned");
  if (d_psnr && (reinterpret_cast<uintptr_t>(d_psnr) & 7))
    return fail(TDCT_EINVAL, "d_psnr not 8-byte aligned");
  for (int a = 0; a < B; ++a)
    for (int c = 0; c < B; ++c) {
      int64_t dot = 0;
      for (int l = 0; l < B; ++l) dot += (int64_t)T[a * B + l] * T[c * B + l];
      if (dot != (a == c ? (int64_t)n[a] : 0))
        return fail(TDCT_ENOTORTHO, "(T T^T)[%d][%d] = %lld does not match diag(n)", a, c,
                    (long long)dot);
    }
  // the JAM matrices from T1: row 2i = [t_i, reverse(t_i)], row 2i + 1 =
  // [t_i, -reverse(t_i)] for the rows t_i of the half-size matrix
  std::vector<int> cur(kT1, kT1 + 64);
  for (int h = 8; h < B; h *= 2) {
    std::vector<int> nxt(4 * h * h);
    for (int i = 0; i < h; ++i)
      for (int m = 0; m < h; ++m) {
        const int t = cur[i * h + m];
        nxt[(2 * i) * 2 * h + m] = t;
        nxt[(2 * i) * 2 * h + 2 * h - 1 - m] = t;
        nxt[(2 * i + 1) * 2 * h + m] = t;
        nxt[(2 * i + 1) * 2 * h + 2 * h - 1 - m] = -t;
      }
    cur.swap(nxt);
  }
  for (int e = 0; e < B * B; ++e)
    if (cur[e] != T[e])
      return fail(TDCT_EUNSUPPORTED,
                  "the %d-point kernels implement the JAM transform of T1 (§6.2) only", B);
  JamParams jp;
  std::memset(&jp, 0, sizeof jp);
  int64_t L = 1;
  for (int i = 0; i < B; ++i) L = L / gcd64(L, n[i]) * n[i];
  for (int i = 0; i < B; ++i) jp.q[i] = (int32_t)(L / n[i]);
  jp.L2 = L * L;
  jp.limit = 256 * 2 * jp.L2;
  jp.hiw = (int32_t)(128 * 2 * jp.L2);
  jp.r = r;
  const int64_t d = 2 * jp.L2;
  int k = 32;
  while (k < 62 && (((int64_t)1 << (k + 1)) + d - 1) / d < ((int64_t)1 << 32)) ++k;
  const int64_t magic = (((int64_t)1 << k) + d - 1) / d;
  const int64_t err = magic * d - ((int64_t)1 << k);
  // the 32-bit second inverse stage of 16x16 u8 blocks needs |2N + L^2| < 2^31
  // with |2N| <= 256 B L^2 (centred samples, orthogonal projection)
  if ((B == 16 && dtype == TDCT_U8 && 256 * (int64_t)B * jp.L2 + jp.L2 >= ((int64_t)1 << 31)) ||
      jp.limit >= ((int64_t)1 << 31) ||
      (unsigned __int128)err * (unsigned __int128)jp.limit >= ((unsigned __int128)1 << k))
    return fail(TDCT_EUNSUPPORTED, "no exact 32-bit division constant for L = %lld", (long long)L);
  jp.magic = (uint32_t)magic;
  jp.shift = k - 32;
  {
    // the 16x16 u8 epilogue: x' in the upper half of a signed 32-bit high
    // product, exact for 0 <= a <= limit (and negative for negative a)
    const int64_t m16 = (((int64_t)1 << 48) + d - 1) / d;
    const int64_t err16 = m16 * d - ((int64_t)1 << 48);
    if (B == 16 && dtype == TDCT_U8 &&
        (m16 >= ((int64_t)1 << 31) ||
         (unsigned __int128)err16 * (unsigned __int128)(jp.limit + 1) >= ((unsigned __int128)1 << 48)))
      return fail(TDCT_EUNSUPPORTED, "no exact 16-bit-lane division constant for L = %lld",
                  (long long)L);
    jp.magic16 = (int32_t)m16;
  }
  const auto a16 = [](const void* p, int64_t pitch) {
    return ((reinterpret_cast<uintptr_t>(p) | (uintptr_t)pitch) & 15) == 0;
  };
  jp.aligned = (a16(d_img, pitch) ? 1 : 0) | (d_recon && a16(d_recon, recon_pitch) ? 2 : 0);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned long long* sse = reinterpret_cast<unsigned long long*>(d_sse);
  const int64_t nblocks = (int64_t)((H + B - 1) / B) * ((W + B - 1) / B);
  if (nblocks >= ((int64_t)1 << 30))
    return fail(TDCT_EINVAL, "%lld blocks of %d x %d: at most 2^30 - 1 per plane", (long long)nblocks, B, B);
  cudaError_t e = cudaMemsetAsync(sse, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return cuda_fail(e, "tdct_codec_error_jam memset");
  const PlaneDesc P = make_desc(d_img, pitch, H, W, dtype, 64, d_recon, recon_pitch, 0);
  if ((e = launch_jam_codec(B, P, jp, sse, s)) != cudaSuccess)
    return cuda_fail(e, "tdct_codec_error_jam launch");
  if (d_psnr) {
    psnr_kernel<<<1, 32, 0, s>>>(sse, nullptr, (int64_t)H * W, d_psnr, 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "psnr launch");
  }
  return TDCT_OK;
}

int tdct_search(int N, const int8_t* alphabet, int np, const int32_t* order, int n_order,
                const int32_t* fixed_rows, const int8_t* fixed_vals, int n_fixed, int tie,
                int8_t* T_out, int32_t* complete, tdct_stream_t stream) {
  if (N < 2 || N > kSearchMaxN) return fail(TDCT_EINVAL, "N = %d outside 2..16", N);
  if (!alphabet || np < 2 || np > 9) return fail(TDCT_EINVAL, "alphabet of %d values", np);
  if (!order || n_order < 1 || n_order > N) return fail(TDCT_EINVAL, "n_order = %d", n_order);
  if (n_fixed < 0 || n_fixed + n_order > N || (n_fixed > 0 && (!fixed_rows || !fixed_vals)))
    return fail(TDCT_EINVAL, "n_fixed = %d (or NULL presets)", n_fixed);
  if (tie != 0 && tie != 1) return fail(TDCT_EINVAL, "tie = %d is neither 0 nor 1", tie);
  if (!T_out || !complete) return fail(TDCT_EINVAL, "T_out and complete must not be NULL");
  SearchParams sp;
  std::memset(&sp, 0, sizeof sp);
  std::vector<int> vals(alphabet, alphabet + np);
  std::sort(vals.begin(), vals.end());
  int maxabs = 0;
  for (int a = 0; a < np; ++a) {
    if (vals[a] < -kSearchMaxAbs || vals[a] > kSearchMaxAbs)
      return fail(TDCT_EINVAL, "alphabet value %d outside [-16, 16]", vals[a]);
    maxabs = std::max(maxabs, std::abs(vals[a]));
    if (a > 0 && vals[a] == vals[a - 1]) return fail(TDCT_EINVAL, "alphabet repeats %d", vals[a]);
    sp.alphabet[a] = vals[a];
  }
  uint64_t total = 1;
  for (int k = 0; k < N; ++k) {
    total *= (uint64_t)np;
    if (total > (1ull << 31)) return fail(TDCT_EUNSUPPORTED, "np^N above 2^31 candidates");
  }
  std::vector<int> used(N, 0);
  for (int f = 0; f < n_fixed; ++f) {
    const int r = fixed_rows[f];
    if (r < 0 || r >= N || used[r]) return fail(TDCT_EINVAL, "preset row %d", r);
    used[r] = 1;
    for (int k = 0; k < N; ++k) sp.fixed[f][k] = fixed_vals[f * N + k];
  }
  for (int i = 0; i < n_order; ++i) {
    const int r = order[i];
    if (r < 0 || r >= N || used[r]) return fail(TDCT_EINVAL, "order entry %d (row %d)", i, r);
    used[r] = 1;
  }
  sp.np = np;
  sp.N = N;
  sp.max_n2 = N * maxabs * maxabs;
  sp.total = (uint32_t)total;
  sp.n_fixed = n_fixed;
  sp.tie_large = tie;
  sp.hit_cap = g_search_hit_cap.load();
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  void* block = nullptr;
  const size_t bytes_mask = round_up((size_t)total, 256);
  const size_t bytes_hits = sizeof(SearchHit) * (size_t)kSearchHitCap;
  cudaError_t e = cudaMallocAsync(&block, bytes_mask + bytes_hits + sizeof(SearchState), s);
  if (e != cudaSuccess) return fail(TDCT_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e));
  uint8_t* allowed = static_cast<uint8_t*>(block);
  SearchHit* hits = reinterpret_cast<SearchHit*>(static_cast<char*>(block) + bytes_mask);
  SearchState* st =
      reinterpret_cast<SearchState*>(static_cast<char*>(block) + bytes_mask + bytes_hits);
  SearchState init;
  std::memset(&init, 0, sizeof init);
  init.pick_key = ~0ull;
  e = cudaMemcpyAsync(st, &init, sizeof init, cudaMemcpyHostToDevice, s);
  for (int i = 0; i < n_order && e == cudaSuccess; ++i) {
    // exact row of the orthonormal N-point DCT-II, coordinates reversed
    const int k = order[i];
    for (int j = 0; j < kSearchMaxN; ++j) sp.crow_rev[j] = 0.0;
    for (int j = 0; j < N; ++j) {
      const double ck = k == 0 ? std::sqrt(1.0 / N) : std::sqrt(2.0 / N);
      sp.crow_rev[N - 1 - j] = ck * std::cos(M_PI * (2.0 * j + 1.0) * k / (2.0 * N));
    }
    e = enqueue_search_row(sp, st, allowed, hits, i == 0, i, s);
  }
  SearchState out;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&out, st, sizeof out, cudaMemcpyDeviceToHost, s);
  const cudaError_t ef = cudaFreeAsync(block, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "tdct_search");
  if (ef != cudaSuccess) return cuda_fail(ef, "cudaFreeAsync");
  std::memset(T_out, 0, (size_t)N * N);
  for (int f = 0; f < n_fixed; ++f)
    for (int k = 0; k < N; ++k) T_out[fixed_rows[f] * N + k] = fixed_vals[f * N + k];
  // the rows committed before a dead end (all of them otherwise)
  for (int i = 0; i < out.n_done && i < n_order; ++i) {
    uint32_t idx = out.chosen[i];
    for (int k = N - 1; k >= 0; --k) {
      T_out[order[i] * N + k] = (int8_t)vals[idx % np];
      idx /= np;
    }
  }
  *complete = out.dead ? 0 : 1;
  return TDCT_OK;
}

int tdct_dct_codec_error(const void* d_img, int64_t pitch, int H, int W, int dtype, int r,
                         int precision, float* d_coef, void* d_recon, int64_t recon_pitch,
                         uint64_t* d_sse, double* d_psnr, tdct_stream_t stream) {
  int rc = check_r(r);
  if (rc) return rc;
  if ((rc = check_plane(d_img, pitch, H, W, dtype, "tdct_dct_codec_error"))) return rc;
  if (d_recon && (rc = check_plane(d_recon, recon_pitch, H, W, dtype, "recon"))) return rc;
  if (precision != TDCT_FP32 && precision != TDCT_BF16 && precision != TDCT_BF16X3)
    return fail(TDCT_EINVAL, "precision %d is not a tdct_precision", precision);
  if (precision == TDCT_BF16X3 && dtype != TDCT_U8)
    return fail(TDCT_EUNSUPPORTED, "TDCT_BF16X3 takes u8 planes (use TDCT_FP32 for int16)");
  if (!d_sse || (reinterpret_cast<uintptr_t>(d_sse) & 7))
    return fail(TDCT_EINVAL, "d_sse NULL or not 8-byte aligned");
  if (d_coef && (reinterpret_cast<uintptr_t>(d_coef) & 3))
    return fail(TDCT_EINVAL, "d_coef not 4-byte aligned");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned long long* sse = reinterpret_cast<unsigned long long*>(d_sse);
  cudaError_t e = cudaMemsetAsync(sse, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return cuda_fail(e, "tdct_dct_codec_error memset");
  const PlaneDesc P = make_desc(d_img, pitch, H, W, dtype, r, d_recon, recon_pitch, 0);
  // bf16 operands on u8 planes: the two GEMMs on the tensor cores (one bf16
  // term per weight, or three for FP32-level accuracy); otherwise the CUDA cores
  e = (precision == TDCT_BF16X3 || (precision == TDCT_BF16 && dtype == TDCT_U8))
          ? launch_dct_tc(P, precision == TDCT_BF16X3 ? 3 : 1, d_coef, status_word(), sse, s)
          : launch_dct_codec(P, precision, d_coef, sse, s);
  if (e != cudaSuccess) return cuda_fail(e, "tdct_dct_codec_error launch");
  if (d_psnr) {
    psnr_kernel<<<1, 32, 0, s>>>(sse, nullptr, (int64_t)H * W, d_psnr, 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "psnr launch");
  }
  return TDCT_OK;
}

}  // extern "C"

namespace {

// Shared body of the two sweep entry points: validation, the sweep's unit
// table (32 blocks per unit) in stream-ordered scratch, the kernel, PSNR.
int sweep_batched(const tdct_plane* planes, int nplanes, bool dct, const float* C,
                  uint64_t* d_sse, double* d_psnr, cudaStream_t s, const char* who) {
  if (!planes || nplanes < 1 || nplanes > (1 << 20))
    return fail(TDCT_EINVAL, "%s: nplanes = %d outside 1..2^20 (or planes is NULL)", who, nplanes);
  if (!d_sse || (reinterpret_cast<uintptr_t>(d_sse) & 7))
    return fail(TDCT_EINVAL, "%s: d_sse NULL or not 8-byte aligned", who);
  if (d_psnr && (reinterpret_cast<uintptr_t>(d_psnr) & 7))
    return fail(TDCT_EINVAL, "%s: d_psnr not 8-byte aligned", who);
  std::vector<PlaneDesc> descs(nplanes);
  std::vector<int64_t> npix(nplanes);
  int64_t units = 0;
  for (int i = 0; i < nplanes; ++i) {
    const tdct_plane& p = planes[i];
    char what[64];
    std::snprintf(what, sizeof what, "%s plane %d", who, i);
    int rc = check_plane(p.img, p.pitch, p.H, p.W, p.dtype, what);
    if (rc) return rc;
    if (p.dtype != TDCT_U8)
      return fail(TDCT_EUNSUPPORTED, "%s: the sweep takes u8 planes (plane %d is int16)", who, i);
    if (p.recon) return fail(TDCT_EINVAL, "%s: plane %d: recon must be NULL", who, i);
    PlaneDesc d = make_desc(p.img, p.pitch, p.H, p.W, p.dtype, 64, nullptr, 0, i);
    d.chunks = (d.nbx + kSweepUnitBlocks - 1) / kSweepUnitBlocks;
    d.unit_begin = units;
    units += (int64_t)d.nby * d.chunks;
    descs[i] = d;
    npix[i] = (int64_t)p.H * p.W;
  }
  const size_t bytes_desc = sizeof(PlaneDesc) * descs.size();
  const size_t bytes_npix = sizeof(int64_t) * npix.size();
  void* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, bytes_desc + bytes_npix, s);
  if (e != cudaSuccess) return fail(TDCT_ENOMEM, "%s: cudaMallocAsync: %s", who, cudaGetErrorString(e));
  PlaneDesc* d_descs = static_cast<PlaneDesc*>(scratch);
  int64_t* d_npix = reinterpret_cast<int64_t*>(static_cast<char*>(scratch) + bytes_desc);
  unsigned long long* sse = reinterpret_cast<unsigned long long*>(d_sse);
  if ((e = cudaMemcpyAsync(d_descs, descs.data(), bytes_desc, cudaMemcpyHostToDevice, s)) ==
          cudaSuccess &&
      (e = cudaMemcpyAsync(d_npix, npix.data(), bytes_npix, cudaMemcpyHostToDevice, s)) ==
          cudaSuccess &&
      (e = cudaMemsetAsync(sse, 0, sizeof(unsigned long long) * 64 * (size_t)nplanes, s)) ==
          cudaSuccess) {
    PlaneTable tab;
    std::memset(&tab, 0, sizeof tab);
    tab.d = d_descs;
    tab.n = nplanes;
    tab.total_units = units;
    e = launch_sweep(tab, dct, C, sse, s);
    if (e == cudaSuccess && d_psnr) {
      const int n = 64 * nplanes;
      psnr_sweep_kernel<<<(n + 255) / 256, 256, 0, s>>>(sse, d_npix, d_psnr, n);
      e = cudaGetLastError();
    }
  }
  const cudaError_t ef = cudaFreeAsync(scratch, s);
  if (e != cudaSuccess) return cuda_fail(e, who);
  if (ef != cudaSuccess) return cuda_fail(ef, "cudaFreeAsync");
  return TDCT_OK;
}

}  // namespace

extern "C" {

int tdct_sweep_batched(const tdct_plane* planes, int nplanes, const int8_t T[64],
                       const int32_t n[8], uint64_t* d_sse, double* d_psnr,
                       tdct_stream_t stream) {
  Transform tr;
  int rc = resolve_transform(T, n, &tr);
  if (rc) return rc;
  if (!tr.t1)
    return fail(TDCT_EUNSUPPORTED,
                "tdct_sweep_batched implements T1 (its fast algorithm); use tdct_codec_error_batched "
                "with one plane per r for another T");
  const float C[64] = {};
  return sweep_batched(planes, nplanes, false, C, d_sse, d_psnr,
                       reinterpret_cast<cudaStream_t>(stream), "tdct_sweep_batched");
}

int tdct_dct_sweep_batched(const tdct_plane* planes, int nplanes, int precision,
                           uint64_t* d_sse, double* d_psnr, tdct_stream_t stream) {
  if (precision != TDCT_FP32)
    return fail(TDCT_EUNSUPPORTED, "tdct_dct_sweep_batched: precision must be TDCT_FP32");
  float C[64];
  for (int k = 0; k < 8; ++k)
    for (int j = 0; j < 8; ++j) {
      const double ck = k == 0 ? std::sqrt(1.0 / 8.0) : std::sqrt(2.0 / 8.0);
      C[8 * k + j] = (float)(ck * std::cos(M_PI * (2.0 * j + 1.0) * k / 16.0));
    }
  return sweep_batched(planes, nplanes, true, C, d_sse, d_psnr,
                       reinterpret_cast<cudaStream_t>(stream), "tdct_dct_sweep_batched");
}

int tdct_debug_inject_wait_timeout(int enable) {
  g_inject_timeout.store(enable ? 1 : 0);
  return TDCT_OK;
}

int tdct_debug_search_hit_cap(int cap) {
  g_search_hit_cap.store(cap >= 0 && cap <= kSearchHitCap ? cap : kSearchHitCap);
  return TDCT_OK;
}

int tdct_shutdown(void) {
  int cur = 0;
  const bool have_cur = cudaGetDevice(&cur) == cudaSuccess;
  cudaError_t first = cudaSuccess;
  std::lock_guard<std::mutex> lock(g_host_mu);
  for (int dev = 0; dev < 256; ++dev) {
    HostStreams& hs = g_host_streams[dev];
    if (!hs.h2d && !hs.d2h) continue;
    cudaError_t e = cudaSetDevice(dev);
    for (cudaStream_t* st : {&hs.h2d, &hs.d2h}) {
      if (!*st) continue;
      if (e == cudaSuccess) e = cudaStreamSynchronize(*st);
      const cudaError_t ed = cudaStreamDestroy(*st);
      if (e == cudaSuccess) e = ed;
      *st = nullptr;
    }
    if (first == cudaSuccess) first = e;
  }
  if (have_cur) cudaSetDevice(cur);
  return first == cudaSuccess ? TDCT_OK : cuda_fail(first, "tdct_shutdown");
}

int tdct_sync_status(tdct_stream_t stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  int status = 0;
  e = cudaMemcpyFromSymbol(&status, g_status, sizeof status);
  if (e != cudaSuccess) return cuda_fail(e, "read status word");
  const int zero = 0;
  e = cudaMemcpyToSymbol(g_status, &zero, sizeof zero);
  if (e != cudaSuccess) return cuda_fail(e, "clear status word");
  if (status == TDCT_ETIMEOUT) return fail(TDCT_ETIMEOUT, "a bounded device wait gave up");
  if (status != 0) return fail(TDCT_EDEVICE, "device check failed with code %d", status);
  return TDCT_OK;
}

}  // extern "C"
