/*
 * tdct.h -- C ABI of the GB300 library for the 8x8 approximate-DCT block
 * codec of Oliveira et al., "Low-complexity 8-point DCT approximation based
 * on angle similarity for image and video coding" (arXiv 1808.02950).
 *
 * The path (§6.1 of the paper): every 8x8 block A of a plane is transformed
 * as B = C_hat A C_hat^T with C_hat = S T (Eq. (1)), S = sqrt((T T^T)^-1)
 * (Eq. (2)); the first r coefficients of the zig-zag scan are kept and the
 * rest zeroed; the block is reconstructed as C_hat^T B' C_hat; the
 * reconstruction is compared with the original (SSE / PSNR).
 *
 * Arguments are plain pointers and sizes.  Conventions for every call:
 *   - "d_" pointers are CUDA device pointers owned by the caller; the host
 *     arrays T and n are read before the call returns.
 *   - T is the 8x8 low-complexity matrix, row-major int8 (row k = t_k^T,
 *     §3.1 Eq. (4)); n are the 8 squared row norms, n_k = (T T^T)_kk, i.e.
 *     S = diag(1/sqrt(n_k)) as §4.1 states it for T1.  The library checks
 *     that T T^T == diag(n) with every n_k >= 1 and returns TDCT_ENOTORTHO
 *     otherwise.  The paper's T1 (§4.1) runs on the fused kernels of its
 *     fast algorithm (§5.1), on either engine below.  Any other orthogonal
 *     T (T2 of §4.1, the orthogonal matrices of Table 2, ...) runs on the
 *     generic kernels (direct integer products with T, CUDA cores only)
 *     with the same exact results, provided L = lcm(n) <= 725 (the exact
 *     32-bit range: 4082 L^2 < 2^31); a larger L returns
 *     TDCT_EUNSUPPORTED, and so does a tensor-core path with T != T1.
 *   - Planes are row-major with a row pitch in BYTES.  dtype TDCT_U8 holds
 *     8-bit samples (images), TDCT_I16 holds int16 residual samples in
 *     [-255, 255].  H and W are in samples and need not be multiples of 8:
 *     edge blocks are zero padded and padded samples do not enter the SSE.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *     default stream) and never synchronise it.  Host-side argument errors
 *     are returned before anything is enqueued.  No exception crosses the
 *     ABI and nothing aborts the process.  tdct_last_error() gives a
 *     thread-local message for the last failing call.
 *   - Bit-exactness: coefficients Z = T A T^T are integers; the
 *     reconstruction equals N / L^2 with L = lcm(n) and an integer N, and is
 *     rounded half away from zero, then clamped to [0, 255] (U8) or
 *     [-255, 255] (I16).  Every result is identical to the integer
 *     definition, bit for bit.
 */
#ifndef TDCT_H_
#define TDCT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream handle; identical to cudaStream_t / CUstream. */
typedef struct CUstream_st* tdct_stream_t;

enum tdct_status {
  TDCT_OK = 0,
  TDCT_EINVAL = 1,       /* bad argument: null pointer, size, r, pitch, dtype */
  TDCT_ENOTORTHO = 2,    /* T T^T is not diag(n) */
  TDCT_ECUDA = 3,        /* a CUDA runtime call failed */
  TDCT_ETIMEOUT = 4,     /* a bounded device wait gave up (see tdct_sync_status) */
  TDCT_EDEVICE = 5,      /* the device reported an internal check failure */
  TDCT_ENOMEM = 6,       /* device or host allocation failed */
  TDCT_EUNSUPPORTED = 7  /* valid request the library does not implement */
};

enum tdct_dtype { TDCT_U8 = 0, TDCT_I16 = 1 };

enum tdct_precision { TDCT_FP32 = 0, TDCT_BF16 = 1, TDCT_BF16X3 = 2 };

/*
 * Forward-transform engines of the fused codec.
 *   TDCT_PATH_BUTTERFLY  the fast algorithm of §5.1 on the CUDA cores
 *                        (for T != T1: the generic kernels).
 *   TDCT_PATH_TENSOR     Z = T1 X T1^T as a GEMM on the tensor cores
 *                        (tcgen05.mma; sm_103a has no int8 MMA, so pixels
 *                        enter as exact fp16 values and the FP32 accumulation
 *                        is exact).  Bit-identical results to the butterfly.
 *                        Used for u8 planes with 16-byte aligned rows,
 *                        W % 16 == 0 and H % 8 == 0; other planes of the batch
 *                        take the butterfly.
 *   TDCT_PATH_TENSOR_PIPELINED
 *                        the tensor engine with the GEMM of the next tile
 *                        running while the current tile is computed
 *                        (faster at large r, slower at small r).
 *   TDCT_PATH_AUTO       the library's choice (plans: autotuned).
 */
enum tdct_path {
  TDCT_PATH_AUTO = 0,
  TDCT_PATH_BUTTERFLY = 1,
  TDCT_PATH_TENSOR = 2,
  TDCT_PATH_TENSOR_PIPELINED = 3
};

/*
 * tdct_forward -- forward 2-D transform of every block (§6.1, B = C_hat A
 * C_hat^T), returning the integer part Z = T A T^T.
 *   d_img     plane, H x W samples of `dtype`, row pitch `pitch` bytes
 *   d_coef    output, int32 [ceil(H/8)][ceil(W/8)][8][8]; element (i, j) of a
 *             block is Z_ij (i = vertical, j = horizontal frequency).  The
 *             normalised coefficient is B_ij = Z_ij / sqrt(n_i n_j).
 * Errors: TDCT_EINVAL (null pointer, H or W < 1, pitch too small, dtype),
 *         TDCT_ENOTORTHO, TDCT_EUNSUPPORTED, TDCT_ECUDA.
 */
int tdct_forward(const void* d_img, int64_t pitch, int H, int W, int dtype,
                 const int8_t T[64], const int32_t n[8], int32_t* d_coef,
                 tdct_stream_t stream);

/*
 * tdct_zonal_inverse -- zonal retention of the first r zig-zag coefficients
 * and inverse 2-D transform (§6.1, A = C_hat^T B' C_hat) of every block.
 *   d_coef    int32 Z as written by tdct_forward ([nby][nbx][8][8])
 *   r         retained coefficients, 1..64
 *   d_out     reconstruction, H x W samples of `dtype`, pitch `out_pitch`
 * Errors: as tdct_forward, plus TDCT_EINVAL for r outside 1..64.
 */
int tdct_zonal_inverse(const int32_t* d_coef, int H, int W, int dtype,
                       const int8_t T[64], const int32_t n[8], int r, void* d_out,
                       int64_t out_pitch, tdct_stream_t stream);

/*
 * tdct_codec_error -- the fused codec of one plane: forward, zonal r,
 * inverse, rounding, and the reconstruction error (§6.1).  Each sample is
 * read from HBM once; the reconstruction is written once if requested.
 *   d_recon   reconstruction output or NULL (error only)
 *   d_sse     output, one uint64: sum over valid samples of (a - a')^2
 *   d_psnr    output or NULL, one double: 10 log10(255^2 H W / SSE),
 *             +inf when SSE = 0
 * Errors: as tdct_zonal_inverse.
 */
int tdct_codec_error(const void* d_img, int64_t pitch, int H, int W, int dtype,
                     const int8_t T[64], const int32_t n[8], int r, void* d_recon,
                     int64_t recon_pitch, uint64_t* d_sse, double* d_psnr,
                     tdct_stream_t stream);

/* One plane of a ragged batch (device pointers, per-plane r and dtype). */
typedef struct tdct_plane {
  const void* img;     /* device pointer to sample (0, 0) */
  int64_t pitch;       /* row pitch in bytes */
  int32_t H, W;        /* size in samples, >= 1 */
  int32_t r;           /* retained zig-zag coefficients, 1..64 */
  int32_t dtype;       /* TDCT_U8 or TDCT_I16 */
  void* recon;         /* device pointer or NULL */
  int64_t recon_pitch; /* row pitch in bytes of recon */
} tdct_plane;

/*
 * tdct_codec_error_batched -- tdct_codec_error over a ragged batch of planes
 * (different sizes, r and dtype) in one enqueue: the library builds a
 * block-offset table, stages it in stream-ordered device memory and runs
 * persistent kernels over all planes.
 *   planes    host array of nplanes descriptors (1 <= nplanes <= 2^20)
 *   d_sse     output, uint64 [nplanes]
 *   d_psnr    output or NULL, double [nplanes]
 *   path      a tdct_path.  The first TDCT_PATH_TENSOR call on a device
 *             uploads the tensor-core weight tables synchronously: make it
 *             outside any stream capture.
 * Errors: as tdct_codec_error for any plane, TDCT_ENOMEM.
 */
int tdct_codec_error_batched(const tdct_plane* planes, int nplanes, const int8_t T[64],
                             const int32_t n[8], uint64_t* d_sse, double* d_psnr,
                             int path, tdct_stream_t stream);

/*
 * tdct_codec_error_batched_noalloc -- tdct_codec_error_batched for callers
 * that must not allocate device memory.  The paper has no counterpart: this
 * is a deployment variant.  Some callers cannot call cudaMalloc (or let a
 * library do it): a process whose own allocator has reserved the device
 * memory up front, a real-time pipeline that forbids allocation after start
 * (an allocation can synchronise the device and has unbounded latency), or
 * code running where a stream-ordered pool is not available.  Here the
 * block-offset table lives in a fixed array inside the library's device
 * image, sized for TDCT_NOALLOC_MAX_PLANES planes (about 176 KB, held by
 * every GPU that loads the library until the process exits).
 *   Arguments, outputs and results are those of tdct_codec_error_batched
 *   (the same kernels run), except that nplanes above TDCT_NOALLOC_MAX_PLANES
 *   returns TDCT_EINVAL.  No device memory is allocated or freed.
 *   The first call on a device looks up the array's device address (once
 *   per device, with that device current).  Every call rewrites the shared
 *   array: calls whose work overlaps on the GPU (for example on two streams)
 *   race on it and must be serialised by the caller.  Calls from several
 *   host threads enqueue their table copy and kernels under one library
 *   lock, so their enqueues never interleave; the GPU-side rule above still
 *   applies.
 */
#define TDCT_NOALLOC_MAX_PLANES 2048
int tdct_codec_error_batched_noalloc(const tdct_plane* planes, int nplanes, const int8_t T[64],
                                     const int32_t n[8], uint64_t* d_sse, double* d_psnr,
                                     tdct_stream_t stream);

/*
 * tdct_codec_error_batched_host -- tdct_codec_error_batched on planes that
 * live in HOST memory, with the results returned to host memory (§6.1 per
 * plane; same kernels, same bit-exact results).  The copies to the device
 * are pipelined with the codec: consecutive planes are grouped into chunks
 * of about `chunk_bytes` (0 = 64 MiB; a larger plane forms its own chunk),
 * staged in two device buffers, and chunk c + 1 is copied while chunk c is
 * coded (and, when reconstructions are requested, chunk c - 1's are copied
 * back).  The transfers use two library-owned non-blocking streams per
 * device (created on first use, kept until exit); device memory comes from
 * the stream-ordered pool and is released on `stream`.
 *   planes    host array of nplanes descriptors whose img / recon are HOST
 *             pointers (recon may be NULL: no reconstruction is copied back).
 *             Page-locked memory lets the copies run at the link's rate and
 *             asynchronously; pageable memory works through the CUDA
 *             driver's staging.
 *   h_sse     host output, uint64 [nplanes]
 *   h_psnr    host output or NULL, double [nplanes]
 * Asynchronous on `stream`: outputs and reconstructions are complete when
 * `stream` has completed the call's work (with pageable h_sse / h_psnr the
 * call returns only after they are written).  The host buffers must stay
 * valid until then.  Errors: as tdct_codec_error_batched (the engine is the
 * CUDA-core one).
 */
int tdct_codec_error_batched_host(const tdct_plane* planes, int nplanes, const int8_t T[64],
                                  const int32_t n[8], uint64_t* h_sse, double* h_psnr,
                                  size_t chunk_bytes, tdct_stream_t stream);

/*
 * tdct_sweep_batched -- the zonal sweep of §6.1: for every plane, the SSE of
 * the codec with each retention r = 1, 2, ..., 64, from one read of the
 * plane.  Each block is transformed once (Z = T1 A T1^T) and reconstructed
 * incrementally, one zig-zag basis image per r; every r's reconstruction
 * is rounded and clamped exactly as tdct_codec_error does, so entry r is bit
 * for bit the SSE that tdct_codec_error returns for that r.
 *   planes    host array of nplanes u8 planes (1 <= nplanes <= 2^20); their
 *             r fields are not used; recon must be NULL (reconstructions are
 *             not written)
 *   T, n      T1 and its squared row norms (TDCT_EUNSUPPORTED for any other
 *             orthogonal T; TDCT_ENOTORTHO as usual)
 *   d_sse     output, uint64 [nplanes][64]: d_sse[64 p + r - 1]
 *   d_psnr    output or NULL, double [nplanes][64], +inf where SSE = 0
 * Device scratch for the plane table comes from the stream-ordered pool.
 * Errors: TDCT_EINVAL (arguments, as tdct_codec_error_batched),
 *         TDCT_EUNSUPPORTED (int16 planes, T != T1), TDCT_ENOMEM, TDCT_ECUDA.
 */
int tdct_sweep_batched(const tdct_plane* planes, int nplanes, const int8_t T[64],
                       const int32_t n[8], uint64_t* d_sse, double* d_psnr,
                       tdct_stream_t stream);

/*
 * tdct_dct_sweep_batched -- the same sweep with the exact orthonormal
 * DCT-II of §2 (the comparison transform of §6.1) in FP32:
 * x_r = 1/2 + sum_{s < r} Y_s (C_i[k] C_j[l]) accumulated one basis image
 * per r, floored and clamped to [0, 255].  Close to, not identical with,
 * the FP64 definition (PSNR within 0.01 dB).
 *   precision TDCT_FP32 (TDCT_BF16 returns TDCT_EUNSUPPORTED)
 *   other arguments as tdct_sweep_batched
 */
int tdct_dct_sweep_batched(const tdct_plane* planes, int nplanes, int precision,
                           uint64_t* d_sse, double* d_psnr, tdct_stream_t stream);

/*
 * tdct_codec_error_jam -- the codec of §6.1 with B x B blocks, B = 16 or 32,
 * and the B-point transforms that §6.2 derives from T1 with the JAM
 * recursion (T_(16) and T_(32) as printed there; Ĉ = S T with S from
 * T T^T = diag(n), the 1/sqrt(2) of the recursion included in S).  Zonal
 * retention keeps the first r positions of the B x B zig-zag scan (the 8x8
 * rule extended: anti-diagonals, odd ones from (0, s) downwards, even ones
 * from (s, 0) upwards); reconstruction, rounding and clamping as for 8x8
 * blocks, bit-exact.
 *   T, n      the B x B matrix (row-major int8) and its B squared row norms;
 *             T must be T_(16) or T_(32) (TDCT_EUNSUPPORTED otherwise: the
 *             kernels implement the JAM fast algorithm)
 *   r         1..B^2
 *   other arguments as tdct_codec_error; edge blocks are zero padded.
 * Errors: as tdct_codec_error, and TDCT_EINVAL for a plane of 2^30 or more
 * B x B blocks.
 */
int tdct_codec_error_jam(const void* d_img, int64_t pitch, int H, int W, int dtype, int B,
                         const int8_t* T, const int32_t* n, int r, void* d_recon,
                         int64_t recon_pitch, uint64_t* d_sse, double* d_psnr,
                         tdct_stream_t stream);

/*
 * tdct_ssim_batched -- mean structural similarity (MSSIM) of pairs of u8
 * planes, the third figure of merit of §6.1, with the index as defined by
 * Wang, Bovik, Sheikh and Simoncelli (2004), which §6.1 cites: an 11x11
 * Gaussian window (standard deviation 1.5 samples, normalised to unit sum),
 * K1 = 0.01, K2 = 0.03, L = 255, evaluated at every position where the window
 * lies inside the plane (no padding) and averaged:
 *   SSIM = ((2 mx my + C1)(2 sxy + C2)) / ((mx^2 + my^2 + C1)(sx^2 + sy^2 + C2)).
 * Typical use: x = an original plane, y = its reconstruction from the codec.
 * Computed in FP32 (centred samples, separable window), accumulated in FP64;
 * agrees with an FP64 evaluation of the definition to about 1e-6.
 *   planes    host array of nplanes pairs (1 <= nplanes <= 2^20); x and y
 *             are device pointers with row pitches in bytes; H, W >= 11
 *   d_mssim   output, double [nplanes]
 * Errors: TDCT_EINVAL (NULL pointer, H or W below 11, pitch below W,
 * misaligned output), TDCT_ENOMEM, TDCT_ECUDA.
 */
typedef struct tdct_ssim_plane {
  const void* x;   /* device pointer to sample (0, 0) of the reference plane */
  int64_t x_pitch; /* row pitch in bytes */
  const void* y;   /* device pointer to sample (0, 0) of the compared plane */
  int64_t y_pitch; /* row pitch in bytes */
  int32_t H, W;    /* size in samples, >= 11 */
} tdct_ssim_plane;

int tdct_ssim_batched(const tdct_ssim_plane* planes, int nplanes, double* d_mssim,
                      tdct_stream_t stream);

/*
 * tdct_search -- the greedy angle search of §3 (Eq. (6); §6.2 poses it for
 * N = 16) on the GPU, for one row order.  Candidates are the vectors of
 * P^N (P = `alphabet`), enumerated as base-|P| numbers over the sorted
 * alphabet with the first coordinate most significant; the zero vector is
 * not a candidate.  For each row k of `order` in turn, the candidate with the
 * largest cos(c_k, d) = <c_k, d> / ||d|| (c_k = row k of the orthonormal
 * N-point DCT-II, FP64) among those orthogonal to every preset and every
 * row already chosen becomes row k.  Cosines within 1e-12 of the maximum
 * tie; `tie` 0 keeps the smaller-norm vector, 1 the larger, then the first
 * in the enumeration.  Candidates are screened with FP32 cosines and those
 * within 1e-5 of the FP32 maximum are resolved in FP64 (the FP32 error is
 * below 5.4e-7, so the result is that of the FP64 rule).
 *   N           blocklength, 2..16
 *   alphabet    np distinct values in [-16, 16], 2 <= np <= 9,
 *               np^N <= 2^31
 *   order       n_order distinct rows (0-based), searched in this order
 *   fixed_rows  n_fixed distinct preset rows (0-based; not in `order`),
 *               fixed_vals their n_fixed x N entries (row-major); both may be
 *               NULL when n_fixed = 0
 *   T_out       host output, int8 [N][N]: searched and preset rows; rows not
 *               reached stay 0
 *   complete    host output: 1, or 0 when some row had no orthogonal
 *               candidate left (the rows before it are in T_out)
 * Synchronous: the call waits for its work on `stream`.  Device scratch of
 * np^N bytes (one per candidate) plus 1 MiB comes from the stream-ordered
 * pool.
 * Errors: TDCT_EINVAL (arguments), TDCT_EUNSUPPORTED (np^N > 2^31),
 * TDCT_ENOMEM, TDCT_ECUDA.
 */
int tdct_search(int N, const int8_t* alphabet, int np, const int32_t* order, int n_order,
                const int32_t* fixed_rows, const int8_t* fixed_vals, int n_fixed, int tie,
                int8_t* T_out, int32_t* complete, tdct_stream_t stream);

/*
 * Batch plans: the same work as tdct_codec_error_batched, prepared once
 * (validation, block-offset table in device memory, launch configuration)
 * and replayed as one CUDA graph per launch.  The plan owns its device
 * memory until tdct_plan_destroy.  Planes' pointers are fixed at creation.
 */
typedef struct tdct_plan tdct_plan;

/*
 * path: a tdct_path.  TDCT_PATH_AUTO autotunes: every candidate engine and
 * launch shape (CTAs per SM) runs on the plan's own planes (their inputs
 * must hold valid data; reconstructions are written) and the fastest is
 * kept.  Creation synchronises the device work it enqueues; call it outside
 * stream capture.
 */
int tdct_plan_create(const tdct_plane* planes, int nplanes, const int8_t T[64],
                     const int32_t n[8], int path, tdct_plan** out_plan);
/* The configuration a plan uses: engine (tdct_path), CTAs per SM (0 = the
 * library default) and, for autotuned plans, the tuned step time in ms. */
int tdct_plan_config(const tdct_plan* plan, int* path, int* ctas_per_sm, float* tuned_ms);
/* Enqueue one run of the plan on `stream`: SSE (and PSNR) for every plane.
 * When every group of the plan runs the u8 bulk-copy ring kernel (T1, u8
 * planes with 16-byte aligned rows, the butterfly engine), the graph holds
 * only the codec launches: the warp that finishes a plane's last units
 * writes its SSE and PSNR from per-plane accumulators the plan owns and
 * leaves them at zero.  Launches of one plan therefore must not overlap on
 * the GPU (launches on one stream never do).  Otherwise the graph resets
 * d_sse, runs the codec launches and a PSNR kernel. */
int tdct_plan_launch(tdct_plan* plan, uint64_t* d_sse, double* d_psnr, tdct_stream_t stream);
/* Kernel launches one tdct_plan_launch performs (for launch accounting):
 * one per group, plus the PSNR kernel unless the launches close themselves. */
int tdct_plan_kernel_count(const tdct_plan* plan);

/*
 * How a plan's planes are grouped into codec launches (no counterpart in the
 * paper; introspection for callers and tests).  One entry per launch: the
 * sample type, r, the number of planes and how the samples reach the kernel:
 *   TDCT_LOAD_BULK    per-warp shared-memory ring filled by bulk copies
 *                     (u8, 16-byte aligned rows, W % 16 == 0, H % 8 == 0);
 *   TDCT_LOAD_STAGED  per-warp shared-memory ring filled by 8-byte cp.async
 *                     copies (8-byte aligned rows, W % 8 == 0, any H);
 *   TDCT_LOAD_PLAIN   plain global loads (all other planes; every plane when
 *                     T != T1, whose generic kernels load directly).
 * Writes min(max, groups) entries to `out` and the number of groups to
 * *count.  Errors: TDCT_EINVAL (NULL plan or count, max < 0).
 */
enum tdct_load { TDCT_LOAD_PLAIN = 0, TDCT_LOAD_BULK = 1, TDCT_LOAD_STAGED = 2 };
typedef struct {
  int32_t dtype;   /* tdct_dtype */
  int32_t r;
  int32_t load;    /* tdct_load */
  int32_t planes;
} tdct_plan_group;
int tdct_plan_groups(const tdct_plan* plan, tdct_plan_group* out, int max, int* count);
void tdct_plan_destroy(tdct_plan* plan);

/*
 * tdct_dct_codec_error -- the exact-DCT comparison codec (§6.1 with C the
 * orthonormal 8-point DCT-II of §2, C[k][j] = c_k cos(pi (2j+1) k / 16)).
 *   precision TDCT_FP32: FP32 constants, FP32 arithmetic (CUDA cores).
 *             TDCT_BF16: bf16 operands, FP32 accumulation.  u8 planes run
 *             as two GEMMs per 128 blocks on the tensor cores: Y = X (C kron
 *             C)^T over the kept coefficients (samples exact in bf16, each
 *             weight C_i[k] C_j[l] rounded once to bf16), then the
 *             reconstruction from Y rounded to bf16.  int16 planes run on the
 *             CUDA cores with the separable form (constants, inputs and the
 *             inter-stage values rounded to bf16, FP32 accumulation).
 *             Coefficient error stated, not targeted: within 2^-6 of max |Y|.
 *             TDCT_BF16X3: u8 planes only, the tensor-core GEMMs with three
 *             bf16 terms per weight and two per coefficient: FP32-level
 *             accuracy (within 1e-5 of max |Y|, PSNR within 0.01 dB of FP64).
 *   d_coef    output or NULL: float [nby][nbx][8][8], Y = C A C^T
 *   Rounding and clamping as the integer path.  Results are close to, not
 *   identical with, the FP64 definition.
 */
int tdct_dct_codec_error(const void* d_img, int64_t pitch, int H, int W, int dtype, int r,
                         int precision, float* d_coef, void* d_recon, int64_t recon_pitch,
                         uint64_t* d_sse, double* d_psnr, tdct_stream_t stream);

/*
 * Device status word: a bounded device-side wait that gives up, or an
 * internal consistency check, records a code instead of trapping.  This
 * synchronises `stream`, returns TDCT_OK, TDCT_ETIMEOUT or TDCT_EDEVICE and
 * clears the word.
 */
int tdct_sync_status(tdct_stream_t stream);

/*
 * Test hook for the bounded waits (no counterpart in the paper).  With
 * enable != 0, the next fused-codec launch that uses the bulk-copy ring
 * withholds one copy, so its mbarrier wait gives up after about 10 ms and
 * records TDCT_ETIMEOUT in the status word instead of waiting for ever; the
 * launch's results are then incomplete.  The hook disarms itself after one
 * launch.  Used by the test suite to check that a stuck copy is reported and
 * leaves the context usable.
 */
int tdct_debug_inject_wait_timeout(int enable);

/*
 * Test hook for tdct_search (no counterpart in the paper).  Sets the capacity
 * of the per-row list of candidates that pass the FP32 screen; a row with more
 * such candidates falls back to a second full scan.  cap outside [0, 65536]
 * restores the default (65536).  The result of tdct_search does not depend on
 * it; the test suite uses a small cap to run the fallback scan.
 */
int tdct_debug_search_hit_cap(int cap);

/*
 * tdct_shutdown -- release what the library owns (the workspace convention
 * of the boundary: caller-owned buffers everywhere, library-owned resources
 * released here).  Waits for and destroys the per-device transfer streams of
 * tdct_codec_error_batched_host.  The fixed device arrays (status word,
 * tensor-core weight tables, the table of tdct_codec_error_batched_noalloc)
 * are part of the library's device image and go with the CUDA context; plans
 * belong to the caller (tdct_plan_destroy).  Call it when no call of the
 * library is in flight; afterwards the library stays usable and re-creates
 * the streams on demand.  Calling it again is harmless.  The current device
 * is restored.  Errors: TDCT_ECUDA (the first failing CUDA call; the streams
 * are released regardless).
 */
int tdct_shutdown(void);

/* Thread-local description of the last error returned on this thread. */
const char* tdct_last_error(void);

/* Library version string. */
const char* tdct_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TDCT_H_ */
