/*
 * tdct_oracle.c -- plain CPU oracle of the 8x8 blockwise codec of §6.1.
 *
 * TEST INFRASTRUCTURE.  This file is the reference that the CUDA library is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * legs of the benchmark load it; the product path never does.  It shares no
 * code, header, table or constant with the CUDA sources.
 *
 * What it computes, per 8x8 block X (rows k = vertical, columns l):
 *   forward (§6.1, Eq. (1)):  B = C_hat X C_hat^T with C_hat = S T and
 *       S = sqrt((T T^T)^-1) = diag(1/sqrt(n)), n = diag(T T^T) (Eq. (2),
 *       T T^T diagonal).  The integer part Z = T X T^T is computed by the
 *       definition (two 8x8 integer matrix products), B = S Z S.
 *   zonal retention (§6.1): keep the first r coefficients of the zig-zag scan
 *       (generated by rule below), zero the rest.
 *   inverse (§6.1): A' = C_hat^T B' C_hat.  With L = lcm(n) and q = L/n this
 *       is exactly N / L^2 where N = T^T (M o Z o q q^T) T (int64), because
 *       S (M o S Z S) S = M o Z / (n n^T) = M o Z o q q^T / L^2.
 *   rounding: the paper is silent; the experiments ran in MATLAB, whose
 *       double -> integer conversion rounds half away from zero and
 *       saturates.  x' = sign(N) * floor((|N| + L^2/2) / L^2), done exactly in
 *       integers, then clamped to [0,255] (u8 planes) or [-255,255] (int16
 *       residual planes).
 *   error (§6.1): SSE = sum (x - x')^2 over the valid pixels of the plane.
 *
 * Edge blocks of planes whose sides are not multiples of 8 are zero padded;
 * padded samples take part in the transform but not in the SSE.
 *
 * The exact-DCT comparison path does the same in FP64 with the orthonormal
 * DCT-II C[k][j] = c_k cos(pi (2j+1) k / 16), c_0 = sqrt(1/8), c_k = 1/2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ENOTORTHO 2
#define ORC_EINVAL 1

/* ---- zig-zag scan by rule (JPEG / Pao convention) -----------------------
 * Anti-diagonals s = i + j = 0..14 in order.  On odd s the scan runs from
 * (0, s) towards increasing i; on even s from (s, 0) towards decreasing i;
 * positions outside 0..7 are skipped.  First steps: (0,0) (0,1) (1,0) (2,0).
 */
void orc_zigzag(int32_t pos_of_index[64], int32_t index_of_pos[64]) {
  int idx = 0;
  for (int s = 0; s <= 14; ++s) {
    if (s % 2 == 1) {
      for (int i = 0; i <= s; ++i) {
        int j = s - i;
        if (i < 8 && j < 8) {
          pos_of_index[idx] = i * 8 + j;
          index_of_pos[i * 8 + j] = idx;
          ++idx;
        }
      }
    } else {
      for (int i = s; i >= 0; --i) {
        int j = s - i;
        if (i < 8 && j < 8) {
          pos_of_index[idx] = i * 8 + j;
          index_of_pos[i * 8 + j] = idx;
          ++idx;
        }
      }
    }
  }
}

static int64_t gcd64(int64_t a, int64_t b) {
  while (b) {
    int64_t t = a % b;
    a = b;
    b = t;
  }
  return a < 0 ? -a : a;
}

/* n = diag(T T^T); fails if T T^T is not diagonal (Eq. (2) then has no
 * diagonal square root and the inverse is not a transpose). */
int orc_row_norms(const int32_t T[64], int64_t n[8]) {
  for (int a = 0; a < 8; ++a) {
    for (int b = 0; b < 8; ++b) {
      int64_t dot = 0;
      for (int l = 0; l < 8; ++l) dot += (int64_t)T[a * 8 + l] * T[b * 8 + l];
      if (a == b) {
        if (dot <= 0) return ORC_ENOTORTHO;
        n[a] = dot;
      } else if (dot != 0) {
        return ORC_ENOTORTHO;
      }
    }
  }
  return ORC_OK;
}

/* Z = T X T^T by the definition (two integer matrix products). */
void orc_forward_block(const int64_t X[64], const int32_t T[64], int64_t Z[64]) {
  int64_t Y[64];
  for (int i = 0; i < 8; ++i)
    for (int l = 0; l < 8; ++l) {
      int64_t acc = 0;
      for (int k = 0; k < 8; ++k) acc += (int64_t)T[i * 8 + k] * X[k * 8 + l];
      Y[i * 8 + l] = acc;
    }
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j) {
      int64_t acc = 0;
      for (int l = 0; l < 8; ++l) acc += Y[i * 8 + l] * (int64_t)T[j * 8 + l];
      Z[i * 8 + j] = acc;
    }
}

/* Second, independent method: vec(Z) = (T kron T) vec(X), row-major vec. */
void orc_forward_block_kron(const int64_t X[64], const int32_t T[64], int64_t Z[64]) {
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j) {
      int64_t acc = 0;
      for (int k = 0; k < 8; ++k)
        for (int l = 0; l < 8; ++l)
          acc += (int64_t)T[i * 8 + k] * (int64_t)T[j * 8 + l] * X[k * 8 + l];
      Z[i * 8 + j] = acc;
    }
}

/* Rounded reconstruction of one block from its integer coefficients Z.
 * keep[p] = 1 for retained positions p = 8 i + j. */
static void inverse_block(const int64_t Z[64], const int32_t T[64], const int64_t q[8],
                          int64_t L2, const int32_t keep[64], int64_t lo, int64_t hi,
                          int64_t out[64]) {
  int64_t W[64], V[64];
  for (int p = 0; p < 64; ++p) W[p] = keep[p] ? Z[p] * q[p / 8] * q[p % 8] : 0;
  /* V = T^T W */
  for (int k = 0; k < 8; ++k)
    for (int j = 0; j < 8; ++j) {
      int64_t acc = 0;
      for (int i = 0; i < 8; ++i) acc += (int64_t)T[i * 8 + k] * W[i * 8 + j];
      V[k * 8 + j] = acc;
    }
  /* N = V T */
  for (int k = 0; k < 8; ++k)
    for (int l = 0; l < 8; ++l) {
      int64_t N = 0;
      for (int j = 0; j < 8; ++j) N += V[k * 8 + j] * (int64_t)T[j * 8 + l];
      int64_t a = N < 0 ? -N : N;
      int64_t m = a / L2;
      int64_t rem = a - m * L2;
      if (2 * rem >= L2) m += 1; /* half away from zero */
      int64_t x = N < 0 ? -m : m;
      if (x < lo) x = lo;
      if (x > hi) x = hi;
      out[k * 8 + l] = x;
    }
}

static int64_t load_sample(const uint8_t* base, int64_t pitch, int dtype, int y, int x) {
  const uint8_t* row = base + (int64_t)y * pitch;
  if (dtype == 0) return row[x];
  int16_t v;
  memcpy(&v, row + 2 * (int64_t)x, 2);
  return v;
}

static void store_sample(uint8_t* base, int64_t pitch, int dtype, int y, int x, int64_t v) {
  uint8_t* row = base + (int64_t)y * pitch;
  if (dtype == 0) {
    row[x] = (uint8_t)v;
  } else {
    int16_t s = (int16_t)v;
    memcpy(row + 2 * (int64_t)x, &s, 2);
  }
}

/*
 * Codec of one plane with an integer matrix T (orthogonal rows).
 *   img, pitch (bytes), H, W, dtype (0 = u8, 1 = int16 residual)
 *   r in [1, 64]
 *   recon (nullable, same dtype, recon_pitch bytes)
 *   coef (nullable): Z for every block, [ceil(H/8)][ceil(W/8)][64], row-major
 *   sse: sum of squared errors over valid pixels
 */
int orc_codec_plane(const uint8_t* img, int64_t pitch, int H, int W, int dtype,
                    const int32_t T[64], int r, uint8_t* recon, int64_t recon_pitch,
                    int64_t* coef, int64_t* sse) {
  if (!img || !sse || H <= 0 || W <= 0 || r < 1 || r > 64 || (dtype != 0 && dtype != 1))
    return ORC_EINVAL;
  int64_t n[8];
  if (orc_row_norms(T, n) != ORC_OK) return ORC_ENOTORTHO;
  int64_t L = n[0];
  for (int i = 1; i < 8; ++i) L = L / gcd64(L, n[i]) * n[i];
  int64_t q[8];
  for (int i = 0; i < 8; ++i) q[i] = L / n[i];
  int64_t L2 = L * L;
  int32_t pos_of[64], idx_of[64], keep[64];
  orc_zigzag(pos_of, idx_of);
  for (int p = 0; p < 64; ++p) keep[p] = idx_of[p] < r;
  int64_t lo = dtype == 0 ? 0 : -255, hi = 255;

  int nby = (H + 7) / 8, nbx = (W + 7) / 8;
  int64_t total = 0;
  for (int by = 0; by < nby; ++by)
    for (int bx = 0; bx < nbx; ++bx) {
      int64_t X[64], Z[64], R[64];
      for (int k = 0; k < 8; ++k)
        for (int l = 0; l < 8; ++l) {
          int y = by * 8 + k, x = bx * 8 + l;
          X[k * 8 + l] = (y < H && x < W) ? load_sample(img, pitch, dtype, y, x) : 0;
        }
      orc_forward_block(X, T, Z);
      if (coef) {
        int64_t* dst = coef + ((int64_t)by * nbx + bx) * 64;
        for (int p = 0; p < 64; ++p) dst[p] = Z[p];
      }
      inverse_block(Z, T, q, L2, keep, lo, hi, R);
      for (int k = 0; k < 8; ++k)
        for (int l = 0; l < 8; ++l) {
          int y = by * 8 + k, x = bx * 8 + l;
          if (y < H && x < W) {
            int64_t d = X[k * 8 + l] - R[k * 8 + l];
            total += d * d;
            if (recon) store_sample(recon, recon_pitch, dtype, y, x, R[k * 8 + l]);
          }
        }
    }
  *sse = total;
  return ORC_OK;
}

/* Reconstruction from given coefficients Z (the inverse half of the codec). */
int orc_zonal_inverse_plane(const int64_t* coef, int H, int W, int dtype, const int32_t T[64],
                            int r, uint8_t* recon, int64_t recon_pitch) {
  if (!coef || !recon || H <= 0 || W <= 0 || r < 1 || r > 64) return ORC_EINVAL;
  int64_t n[8];
  if (orc_row_norms(T, n) != ORC_OK) return ORC_ENOTORTHO;
  int64_t L = n[0];
  for (int i = 1; i < 8; ++i) L = L / gcd64(L, n[i]) * n[i];
  int64_t q[8];
  for (int i = 0; i < 8; ++i) q[i] = L / n[i];
  int32_t pos_of[64], idx_of[64], keep[64];
  orc_zigzag(pos_of, idx_of);
  for (int p = 0; p < 64; ++p) keep[p] = idx_of[p] < r;
  int64_t lo = dtype == 0 ? 0 : -255, hi = 255;
  int nby = (H + 7) / 8, nbx = (W + 7) / 8;
  for (int by = 0; by < nby; ++by)
    for (int bx = 0; bx < nbx; ++bx) {
      int64_t R[64];
      inverse_block(coef + ((int64_t)by * nbx + bx) * 64, T, q, L * L, keep, lo, hi, R);
      for (int k = 0; k < 8; ++k)
        for (int l = 0; l < 8; ++l) {
          int y = by * 8 + k, x = bx * 8 + l;
          if (y < H && x < W) store_sample(recon, recon_pitch, dtype, y, x, R[k * 8 + l]);
        }
    }
  return ORC_OK;
}

/* ---- exact DCT in FP64 ------------------------------------------------- */

void orc_dct_matrix(double C[64]) {
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < 8; ++k)
    for (int j = 0; j < 8; ++j) {
      double ck = k == 0 ? sqrt(1.0 / 8.0) : sqrt(2.0 / 8.0);
      C[k * 8 + j] = ck * cos(pi * (2.0 * j + 1.0) * k / 16.0);
    }
}

/*
 * Exact-DCT codec of one plane in FP64: Y = C X C^T, keep the first r zig-zag
 * coefficients, X' = C^T Y' C, round half away from zero, clamp.
 *   coef (nullable): Y in FP64, [ceil(H/8)][ceil(W/8)][64].
 */
int orc_dct_codec_plane(const uint8_t* img, int64_t pitch, int H, int W, int dtype, int r,
                        uint8_t* recon, int64_t recon_pitch, double* coef, int64_t* sse) {
  if (!img || !sse || H <= 0 || W <= 0 || r < 1 || r > 64 || (dtype != 0 && dtype != 1))
    return ORC_EINVAL;
  double C[64];
  orc_dct_matrix(C);
  int32_t pos_of[64], idx_of[64];
  orc_zigzag(pos_of, idx_of);
  double lo = dtype == 0 ? 0.0 : -255.0, hi = 255.0;
  int nby = (H + 7) / 8, nbx = (W + 7) / 8;
  int64_t total = 0;
  for (int by = 0; by < nby; ++by)
    for (int bx = 0; bx < nbx; ++bx) {
      double X[64], T1[64], Y[64], V[64];
      for (int k = 0; k < 8; ++k)
        for (int l = 0; l < 8; ++l) {
          int y = by * 8 + k, x = bx * 8 + l;
          X[k * 8 + l] = (y < H && x < W) ? (double)load_sample(img, pitch, dtype, y, x) : 0.0;
        }
      for (int i = 0; i < 8; ++i)
        for (int l = 0; l < 8; ++l) {
          double acc = 0;
          for (int k = 0; k < 8; ++k) acc += C[i * 8 + k] * X[k * 8 + l];
          T1[i * 8 + l] = acc;
        }
      for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) {
          double acc = 0;
          for (int l = 0; l < 8; ++l) acc += T1[i * 8 + l] * C[j * 8 + l];
          Y[i * 8 + j] = acc;
        }
      if (coef) {
        double* dst = coef + ((int64_t)by * nbx + bx) * 64;
        for (int p = 0; p < 64; ++p) dst[p] = Y[p];
      }
      for (int p = 0; p < 64; ++p)
        if (idx_of[p] >= r) Y[p] = 0.0;
      for (int k = 0; k < 8; ++k)
        for (int j = 0; j < 8; ++j) {
          double acc = 0;
          for (int i = 0; i < 8; ++i) acc += C[i * 8 + k] * Y[i * 8 + j];
          V[k * 8 + j] = acc;
        }
      for (int k = 0; k < 8; ++k)
        for (int l = 0; l < 8; ++l) {
          double acc = 0;
          for (int j = 0; j < 8; ++j) acc += V[k * 8 + j] * C[j * 8 + l];
          double x = round(acc); /* C round(): half away from zero */
          if (x < lo) x = lo;
          if (x > hi) x = hi;
          int y = by * 8 + k, xx = bx * 8 + l;
          if (y < H && xx < W) {
            int64_t d = (int64_t)X[k * 8 + l] - (int64_t)x;
            total += d * d;
            if (recon) store_sample(recon, recon_pitch, dtype, y, xx, (int64_t)x);
          }
        }
    }
  *sse = total;
  return ORC_OK;
}

/* PSNR = 10 log10(255^2 / MSE), MSE = SSE / npix; +inf when SSE = 0. */
double orc_psnr(int64_t sse, int64_t npix) {
  if (sse == 0) return INFINITY;
  double mse = (double)sse / (double)npix;
  return 10.0 * log10(255.0 * 255.0 / mse);
}

/*
 * Mean structural similarity (MSSIM) of two u8 planes.  §6.1 evaluates the
 * reconstructions with SSIM as defined by Wang, Bovik, Sheikh and Simoncelli
 * (2004); the parameters are that paper's: an 11x11 circular-symmetric
 * Gaussian weighting window w (standard deviation 1.5 samples, normalised to
 * unit sum), K1 = 0.01, K2 = 0.03, dynamic range L = 255.  At every position
 * where the window lies entirely inside the plane (no padding):
 *   mx = sum w x,  sx^2 = sum w (x - mx)^2,  sxy = sum w (x - mx)(y - my),
 *   SSIM = ((2 mx my + C1)(2 sxy + C2)) / ((mx^2 + my^2 + C1)(sx^2 + sy^2 + C2))
 * with C1 = (K1 L)^2, C2 = (K2 L)^2; MSSIM = the mean of SSIM over those
 * positions.  Everything by the definition (two passes over each window),
 * in double.  Returns ORC_EINVAL when the plane is smaller than the window.
 */
int orc_ssim_plane(const uint8_t* x, int64_t xpitch, const uint8_t* y, int64_t ypitch, int H,
                   int W, double* mssim) {
  enum { WIN = 11, HALF = 5 };
  if (H < WIN || W < WIN) return ORC_EINVAL;
  double w[WIN][WIN], wsum = 0.0;
  for (int i = 0; i < WIN; ++i)
    for (int j = 0; j < WIN; ++j) {
      const double di = i - HALF, dj = j - HALF;
      w[i][j] = exp(-(di * di + dj * dj) / (2.0 * 1.5 * 1.5));
      wsum += w[i][j];
    }
  for (int i = 0; i < WIN; ++i)
    for (int j = 0; j < WIN; ++j) w[i][j] /= wsum;
  const double C1 = (0.01 * 255.0) * (0.01 * 255.0), C2 = (0.03 * 255.0) * (0.03 * 255.0);
  double total = 0.0;
  for (int r0 = 0; r0 + WIN <= H; ++r0)
    for (int c0 = 0; c0 + WIN <= W; ++c0) {
      double mx = 0.0, my = 0.0;
      for (int i = 0; i < WIN; ++i)
        for (int j = 0; j < WIN; ++j) {
          mx += w[i][j] * x[(int64_t)(r0 + i) * xpitch + c0 + j];
          my += w[i][j] * y[(int64_t)(r0 + i) * ypitch + c0 + j];
        }
      double sxx = 0.0, syy = 0.0, sxy = 0.0;
      for (int i = 0; i < WIN; ++i)
        for (int j = 0; j < WIN; ++j) {
          const double dx = x[(int64_t)(r0 + i) * xpitch + c0 + j] - mx;
          const double dy = y[(int64_t)(r0 + i) * ypitch + c0 + j] - my;
          sxx += w[i][j] * dx * dx;
          syy += w[i][j] * dy * dy;
          sxy += w[i][j] * dx * dy;
        }
      total += ((2.0 * mx * my + C1) * (2.0 * sxy + C2)) /
               ((mx * mx + my * my + C1) * (sxx + syy + C2));
    }
  *mssim = total / ((double)(H - WIN + 1) * (double)(W - WIN + 1));
  return ORC_OK;
}

/*
 * The codec of §6.1 for B x B blocks (B = 8, 16 or 32; §6.2 builds the 16-
 * and 32-point matrices with the JAM recursion), for any integer T with
 * orthogonal rows, by the definitions above written for B:
 *   Z = T X T^T (int64), keep the first r positions of the B x B zig-zag
 *   scan (anti-diagonals, odd ones from (0, s) with i increasing, even ones
 *   from (s, 0) with i decreasing), N = T^T (M o Z o q q^T) T with q = L / n,
 *   L = lcm(n), x' = sign(N) floor((|N| + L^2/2) / L^2), clamped.
 * Magnitudes stay in int64: |Z| < 2^20 and |N| < 2^43 for B = 32.
 */
static void zigzag_b(int B, int32_t* index_of_pos) {
  int idx = 0;
  for (int s = 0; s <= 2 * B - 2; ++s) {
    if (s % 2 == 1) {
      for (int i = 0; i <= s; ++i) {
        const int j = s - i;
        if (i < B && j < B) index_of_pos[i * B + j] = idx++;
      }
    } else {
      for (int i = s; i >= 0; --i) {
        const int j = s - i;
        if (i < B && j < B) index_of_pos[i * B + j] = idx++;
      }
    }
  }
}

int orc_zigzag_b(int B, int32_t* index_of_pos) {
  if (B < 1 || B > 64) return ORC_EINVAL;
  zigzag_b(B, index_of_pos);
  return ORC_OK;
}

int orc_codec_plane_b(const uint8_t* img, int64_t pitch, int H, int W, int dtype, int B,
                      const int32_t* T, int r, uint8_t* recon, int64_t recon_pitch,
                      int64_t* sse) {
  if (!img || !sse || !T || H <= 0 || W <= 0 || (B != 8 && B != 16 && B != 32) || r < 1 ||
      r > B * B || (dtype != 0 && dtype != 1))
    return ORC_EINVAL;
  const int BB = B * B;
  int64_t* n = (int64_t*)malloc(sizeof(int64_t) * B);
  int64_t* q = (int64_t*)malloc(sizeof(int64_t) * B);
  int32_t* zz = (int32_t*)malloc(sizeof(int32_t) * BB);
  int64_t* X = (int64_t*)malloc(sizeof(int64_t) * BB);
  int64_t* Y = (int64_t*)malloc(sizeof(int64_t) * BB);
  int64_t* Z = (int64_t*)malloc(sizeof(int64_t) * BB);
  int rc = ORC_OK;
  for (int a = 0; a < B && rc == ORC_OK; ++a)
    for (int b = 0; b < B; ++b) {
      int64_t dot = 0;
      for (int l = 0; l < B; ++l) dot += (int64_t)T[a * B + l] * T[b * B + l];
      if (a == b) {
        if (dot <= 0) rc = ORC_ENOTORTHO;
        n[a] = dot;
      } else if (dot != 0) {
        rc = ORC_ENOTORTHO;
      }
    }
  if (rc == ORC_OK) {
    int64_t L = n[0];
    for (int i = 1; i < B; ++i) L = L / gcd64(L, n[i]) * n[i];
    for (int i = 0; i < B; ++i) q[i] = L / n[i];
    const int64_t L2 = L * L;
    zigzag_b(B, zz);
    const int64_t lo = dtype == 0 ? 0 : -255, hi = 255;
    const int nby = (H + B - 1) / B, nbx = (W + B - 1) / B;
    int64_t total = 0;
    for (int by = 0; by < nby; ++by)
      for (int bx = 0; bx < nbx; ++bx) {
        for (int k = 0; k < B; ++k)
          for (int l = 0; l < B; ++l) {
            const int y = by * B + k, x = bx * B + l;
            X[k * B + l] = (y < H && x < W) ? load_sample(img, pitch, dtype, y, x) : 0;
          }
        /* Y = T X, Z = Y T^T */
        for (int i = 0; i < B; ++i)
          for (int l = 0; l < B; ++l) {
            int64_t acc = 0;
            for (int k = 0; k < B; ++k) acc += (int64_t)T[i * B + k] * X[k * B + l];
            Y[i * B + l] = acc;
          }
        for (int i = 0; i < B; ++i)
          for (int j = 0; j < B; ++j) {
            int64_t acc = 0;
            for (int l = 0; l < B; ++l) acc += Y[i * B + l] * (int64_t)T[j * B + l];
            Z[i * B + j] = zz[i * B + j] < r ? acc * q[i] * q[j] : 0;
          }
        /* V = T^T W (into Y), N = V T */
        for (int k = 0; k < B; ++k)
          for (int j = 0; j < B; ++j) {
            int64_t acc = 0;
            for (int i = 0; i < B; ++i) acc += (int64_t)T[i * B + k] * Z[i * B + j];
            Y[k * B + j] = acc;
          }
        for (int k = 0; k < B; ++k)
          for (int l = 0; l < B; ++l) {
            int64_t N = 0;
            for (int j = 0; j < B; ++j) N += Y[k * B + j] * (int64_t)T[j * B + l];
            const int64_t a = N < 0 ? -N : N;
            int64_t m = a / L2;
            if (2 * (a - m * L2) >= L2) m += 1; /* half away from zero */
            int64_t xr = N < 0 ? -m : m;
            if (xr < lo) xr = lo;
            if (xr > hi) xr = hi;
            const int y = by * B + k, x = bx * B + l;
            if (y < H && x < W) {
              const int64_t d = X[k * B + l] - xr;
              total += d * d;
              if (recon) store_sample(recon, recon_pitch, dtype, y, x, xr);
            }
          }
      }
    *sse = total;
  }
  free(n);
  free(q);
  free(zz);
  free(X);
  free(Y);
  free(Z);
  return rc;
}
