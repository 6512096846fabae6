/*
 * Oracle for the 14-addition approximate DCT codec of Bayer & Cintra,
 * "DCT-like Transform for Image Compression Requires 14 Additions Only".
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously correct CPU
 * restatement of what the codec computes.  Only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or constant with the CUDA library; the two meet only through
 * the seeded synthetic inputs, which hold none of the codec's arithmetic.
 *
 * Everything here uses the dense matrix T of Section 2 (no fast algorithm, no
 * blocking, no fusion), 64-bit integers for the codec and double precision for
 * the float variant:
 *
 *   forward      Z = T x T^T, x = X - 128 per 8x8 block       (Sec. 2 matrix T; Sec. 3 blockwise 2D)
 *   quantise     q = round-half-away(Z / Q)  and/or  zonal zig-zag mask (Sec. 2 "D^2 merged"; Sec. 3 zig-zag r)
 *   dequantise   S_ij = q_ij * Q_ij * 2^(6 - a_i - a_j), D^2 = diag(2^-a_i)   (Sec. 2, D and D^2)
 *   inverse      R = T^T S T                                    (Sec. 2 orthogonality: T^-1 = T^T D^2)
 *   reconstruct  pixel = clamp(floor((R + 32) / 64) + 128, 0, 255)
 *
 *   float        y = D T x T^T D; z = y - (Q / 2 pi) sin(2 pi y / Q)   (Sec. 2 C^ = D T)
 *   adjoint      g_x = T^T D (g_z * (1 - cos(2 pi y / Q))) D T
 *
 * Parity: every function below is pinned by tests against facts the paper and
 * mathematics fix (factorisation, orthogonality, identity round trip, brute-force
 * rounding, finite differences).  None is "parity unpinned".
 */
#define _USE_MATH_DEFINES
#include <math.h>
#include <stdint.h>
#include <string.h>

/* Section 2: the 8x8 transform matrix T with entries in {0, +1, -1}. */
static const int64_t T[8][8] = {
    {1,  1,  1,  1,  1,  1,  1,  1},
    {1,  0,  0,  0,  0,  0,  0, -1},
    {1,  0,  0, -1, -1,  0,  0,  1},
    {0,  0, -1,  0,  0,  1,  0,  0},
    {1, -1, -1,  1,  1, -1, -1,  1},
    {0, -1,  0,  0,  0,  0,  1,  0},
    {0, -1,  1,  0,  0,  1, -1,  0},
    {0,  0,  0, -1,  1,  0,  0,  0},
};

/* Section 2: D = diag(1/sqrt8, 1/sqrt2, 1/2, 1/sqrt2, 1/sqrt8, 1/sqrt2, 1/2, 1/sqrt2),
 * so D^2 = diag(2^-a_i) with these exponents. */
static const int A_EXP[8] = {3, 1, 2, 1, 3, 1, 2, 1};

enum { MODE_NONE = 0, MODE_STEP = 1, MODE_ZONAL = 2, MODE_STEP_ZONAL = 3 };

void oracle_matrix_T(int64_t out[64]) {
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j) out[i * 8 + j] = T[i][j];
}

void oracle_scale_exponents(int32_t out[8]) {
  for (int i = 0; i < 8; ++i) out[i] = A_EXP[i];
}

/* Section 3: the standard (JPEG) zig-zag sequence over an 8x8 block.  Walk the
 * anti-diagonals s = i + j in increasing order; on even s move up-right (row i
 * decreasing), on odd s move down-left (row i increasing).  rank[i*8+j] is the
 * position of (i, j) in that sequence. */
void oracle_zigzag_rank(int32_t rank[64]) {
  int k = 0;
  for (int s = 0; s <= 14; ++s) {
    if (s % 2 == 0) {
      for (int i = (s < 8 ? s : 7); i >= 0 && s - i <= 7; --i) rank[i * 8 + (s - i)] = k++;
    } else {
      for (int i = (s < 8 ? 0 : s - 7); i <= 7 && i <= s; ++i) rank[i * 8 + (s - i)] = k++;
    }
  }
}

static int64_t floor_div(int64_t a, int64_t b) { /* b > 0 */
  int64_t q = a / b;
  if ((a % b) != 0 && a < 0) q -= 1;
  return q;
}

/* Z = T x T^T for one block, x already level-shifted. */
static void forward_block(const int64_t x[64], int64_t Z[64]) {
  int64_t Y[64]; /* Y = T x */
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j) {
      int64_t acc = 0;
      for (int k = 0; k < 8; ++k) acc += T[i][k] * x[k * 8 + j];
      Y[i * 8 + j] = acc;
    }
  for (int i = 0; i < 8; ++i) /* Z = Y T^T */
    for (int j = 0; j < 8; ++j) {
      int64_t acc = 0;
      for (int k = 0; k < 8; ++k) acc += Y[i * 8 + k] * T[j][k];
      Z[i * 8 + j] = acc;
    }
}

/* R = T^T S T for one block. */
static void inverse_block(const int64_t S[64], int64_t R[64]) {
  int64_t V[64]; /* V = T^T S */
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j) {
      int64_t acc = 0;
      for (int k = 0; k < 8; ++k) acc += T[k][i] * S[k * 8 + j];
      V[i * 8 + j] = acc;
    }
  for (int i = 0; i < 8; ++i) /* R = V T */
    for (int j = 0; j < 8; ++j) {
      int64_t acc = 0;
      for (int k = 0; k < 8; ++k) acc += V[i * 8 + k] * T[k][j];
      R[i * 8 + j] = acc;
    }
}

static int check_plane(int32_t width, int32_t height, int64_t pitch) {
  if (width <= 0 || height <= 0 || width % 8 || height % 8 || pitch < width) return -1;
  return 0;
}

/* Forward transform of one uint8 plane.  Z: int64 block-major
 * [height/8][width/8][8][8].  Returns 0, or -1 on a bad shape. */
int oracle_forward(const uint8_t* src, int64_t pitch, int32_t width, int32_t height, int64_t* Z) {
  if (check_plane(width, height, pitch)) return -1;
  const int wb = width / 8, hb = height / 8;
  for (int by = 0; by < hb; ++by)
    for (int bx = 0; bx < wb; ++bx) {
      int64_t x[64];
      for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j)
          x[i * 8 + j] = (int64_t)src[(int64_t)(8 * by + i) * pitch + 8 * bx + j] - 128;
      forward_block(x, Z + ((int64_t)by * wb + bx) * 64);
    }
  return 0;
}

/* Quantise nblocks blocks of coefficients (block-major, 64 per block).
 * STEP: q = round half away from zero of Z/Q, i.e. sgn(Z) * floor((2|Z| + Q) / (2Q)).
 * ZONAL: keep Z where zig-zag rank < r, zero elsewhere (Sec. 3).
 * STEP_ZONAL: the step quantiser, then the zonal mask.  NONE: q = Z.
 * Returns 0, or -1 on bad parameters. */
int oracle_quantise(const int64_t* Z, int64_t nblocks, int32_t mode, const uint16_t* Q, int32_t r,
                    int64_t* q) {
  if (mode < MODE_NONE || mode > MODE_STEP_ZONAL || r < 0 || r > 64) return -1;
  int32_t rank[64];
  oracle_zigzag_rank(rank);
  const int step = (mode == MODE_STEP || mode == MODE_STEP_ZONAL);
  const int zonal = (mode == MODE_ZONAL || mode == MODE_STEP_ZONAL);
  if (step)
    for (int k = 0; k < 64; ++k)
      if (Q[k] < 1) return -1;
  for (int64_t b = 0; b < nblocks; ++b)
    for (int k = 0; k < 64; ++k) {
      int64_t z = Z[b * 64 + k], v = z;
      if (step) {
        int64_t mag = z < 0 ? -z : z;
        int64_t Qk = Q[k];
        int64_t m = (2 * mag + Qk) / (2 * Qk); /* both non-negative: plain floor */
        v = z < 0 ? -m : m;
      }
      if (zonal && rank[k] >= r) v = 0;
      q[b * 64 + k] = v;
    }
  return 0;
}

/* Dequantise with D^2 merged (S_ij = q_ij * Q_ij * 2^(6 - a_i - a_j); Q = 1 in the
 * NONE and ZONAL modes), invert R = T^T S T, and reconstruct one uint8 plane:
 * pixel = clamp(floor((R + 32) / 64) + 128, 0, 255).  Returns 0 or -1. */
int oracle_inverse(const int64_t* q, int32_t mode, const uint16_t* Q, uint8_t* dst, int64_t pitch,
                   int32_t width, int32_t height) {
  if (check_plane(width, height, pitch) || mode < MODE_NONE || mode > MODE_STEP_ZONAL) return -1;
  const int step = (mode == MODE_STEP || mode == MODE_STEP_ZONAL);
  if (step)
    for (int k = 0; k < 64; ++k)
      if (Q[k] < 1) return -1;
  const int wb = width / 8, hb = height / 8;
  for (int by = 0; by < hb; ++by)
    for (int bx = 0; bx < wb; ++bx) {
      const int64_t* qb = q + ((int64_t)by * wb + bx) * 64;
      int64_t S[64], R[64];
      for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) {
          int64_t Qij = step ? (int64_t)Q[i * 8 + j] : 1;
          int64_t scale = (int64_t)1 << (6 - A_EXP[i] - A_EXP[j]);
          S[i * 8 + j] = qb[i * 8 + j] * Qij * scale;
        }
      inverse_block(S, R);
      for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) {
          int64_t p = floor_div(R[i * 8 + j] + 32, 64) + 128;
          if (p < 0) p = 0;
          if (p > 255) p = 255;
          dst[(int64_t)(8 * by + i) * pitch + 8 * bx + j] = (uint8_t)p;
        }
    }
  return 0;
}

/* Whole round trip of one plane: forward, quantise, inverse.  Scratch is
 * 2 * nblocks * 64 int64 provided by the caller; q_out (nullable) receives the
 * quantised coefficients.  Returns 0 or -1. */
int oracle_roundtrip(const uint8_t* src, int64_t src_pitch, uint8_t* dst, int64_t dst_pitch,
                     int32_t width, int32_t height, int32_t mode, const uint16_t* Q, int32_t r,
                     int64_t* scratch, int64_t* q_out) {
  if (check_plane(width, height, src_pitch) || check_plane(width, height, dst_pitch)) return -1;
  const int64_t nb = (int64_t)(width / 8) * (height / 8);
  int64_t* Z = scratch;
  int64_t* q = q_out ? q_out : scratch + nb * 64;
  if (oracle_forward(src, src_pitch, width, height, Z)) return -1;
  if (oracle_quantise(Z, nb, mode, Q, r, q)) return -1;
  return oracle_inverse(q, mode, Q, dst, dst_pitch, width, height);
}

/* ---------------- float variant (double precision) ---------------- */

static void d_diag(double d[8]) {
  for (int i = 0; i < 8; ++i) d[i] = 1.0 / sqrt((double)(1 << A_EXP[i])); /* Sec. 2 D */
}

/* y = D T x T^T D for one block, x row-major 8x8. */
static void fwd_block_f64(const double x[64], double y[64]) {
  double d[8], Y[64];
  d_diag(d);
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j) {
      double acc = 0;
      for (int k = 0; k < 8; ++k) acc += (double)T[i][k] * x[k * 8 + j];
      Y[i * 8 + j] = acc;
    }
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j) {
      double acc = 0;
      for (int k = 0; k < 8; ++k) acc += Y[i * 8 + k] * (double)T[j][k];
      y[i * 8 + j] = d[i] * acc * d[j];
    }
}

/* g = T^T D G D T for one block. */
static void adj_block_f64(const double G[64], double g[64]) {
  double d[8], S[64], V[64];
  d_diag(d);
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j) S[i * 8 + j] = d[i] * G[i * 8 + j] * d[j];
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j) {
      double acc = 0;
      for (int k = 0; k < 8; ++k) acc += (double)T[k][i] * S[k * 8 + j];
      V[i * 8 + j] = acc;
    }
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j) {
      double acc = 0;
      for (int k = 0; k < 8; ++k) acc += V[i * 8 + k] * (double)T[k][j];
      g[i * 8 + j] = acc;
    }
}

static int check_f64(int64_t planes, int32_t H, int32_t W) {
  return (planes < 0 || H <= 0 || W <= 0 || H % 8 || W % 8) ? -1 : 0;
}

/* Float forward over planes x [planes][H][W] (row-major).  y_out (nullable)
 * receives D T x T^T D per block in place of the pixels; z_out receives the
 * soft-quantised y - (Q/2pi) sin(2pi y / Q), or y itself when Qsoft is NULL. */
int oracle_forward_f64(const double* x, int64_t planes, int32_t H, int32_t W, const double* Qsoft,
                       double* y_out, double* z_out) {
  if (check_f64(planes, H, W)) return -1;
  const double two_pi = 2.0 * M_PI;
  for (int64_t p = 0; p < planes; ++p)
    for (int by = 0; by < H / 8; ++by)
      for (int bx = 0; bx < W / 8; ++bx) {
        double xb[64], yb[64];
        const int64_t base = p * (int64_t)H * W + (int64_t)(8 * by) * W + 8 * bx;
        for (int i = 0; i < 8; ++i)
          for (int j = 0; j < 8; ++j) xb[i * 8 + j] = x[base + (int64_t)i * W + j];
        fwd_block_f64(xb, yb);
        for (int i = 0; i < 8; ++i)
          for (int j = 0; j < 8; ++j) {
            const double yv = yb[i * 8 + j];
            double zv = yv;
            if (Qsoft) {
              const double Qk = Qsoft[i * 8 + j];
              zv = yv - (Qk / two_pi) * sin(two_pi * yv / Qk);
            }
            if (y_out) y_out[base + (int64_t)i * W + j] = yv;
            z_out[base + (int64_t)i * W + j] = zv;
          }
      }
  return 0;
}

/* Adjoint of oracle_forward_f64 with respect to x:
 * g_x = T^T D (g_z * dz/dy) D T, dz/dy = 1 - cos(2 pi y / Q) (1 when Qsoft is NULL). */
int oracle_backward_f64(const double* x, const double* gz, int64_t planes, int32_t H, int32_t W,
                        const double* Qsoft, double* gx) {
  if (check_f64(planes, H, W)) return -1;
  const double two_pi = 2.0 * M_PI;
  for (int64_t p = 0; p < planes; ++p)
    for (int by = 0; by < H / 8; ++by)
      for (int bx = 0; bx < W / 8; ++bx) {
        double xb[64], yb[64], G[64], g[64];
        const int64_t base = p * (int64_t)H * W + (int64_t)(8 * by) * W + 8 * bx;
        for (int i = 0; i < 8; ++i)
          for (int j = 0; j < 8; ++j) xb[i * 8 + j] = x[base + (int64_t)i * W + j];
        fwd_block_f64(xb, yb);
        for (int i = 0; i < 8; ++i)
          for (int j = 0; j < 8; ++j) {
            double dzdy = 1.0;
            if (Qsoft) dzdy = 1.0 - cos(two_pi * yb[i * 8 + j] / Qsoft[i * 8 + j]);
            G[i * 8 + j] = gz[base + (int64_t)i * W + j] * dzdy;
          }
        adj_block_f64(G, g);
        for (int i = 0; i < 8; ++i)
          for (int j = 0; j < 8; ++j) gx[base + (int64_t)i * W + j] = g[i * 8 + j];
      }
  return 0;
}

/* ---------------- exact-DCT comparator (double precision) ---------------- */

/* Sec. 3 compares the approximation against the exact DCT: the orthonormal 8x8
 * DCT-II, C[k][j] = alpha_k cos(pi (2j + 1) k / 16), alpha_0 = 1/sqrt(8),
 * alpha_k = 1/2.  Keep the first r zig-zag coefficients of C (X - 128) C^T,
 * invert with C^T Y C, add 128, round to nearest (ties to even) and clamp to
 * 0..255.  Returns 0, or -1 on a bad shape or r. */
void oracle_dct_matrix(double out[64]) {
  for (int k = 0; k < 8; ++k)
    for (int j = 0; j < 8; ++j)
      out[k * 8 + j] = (k == 0 ? sqrt(0.125) : 0.5) * cos(M_PI * (2 * j + 1) * k / 16.0);
}

int oracle_dct_zonal(const uint8_t* src, int64_t pitch, int32_t width, int32_t height, int32_t r, uint8_t* dst,
                     int64_t dst_pitch) {
  if (check_plane(width, height, pitch) || check_plane(width, height, dst_pitch) || r < 0 || r > 64) return -1;
  double C[64];
  int32_t rank[64];
  oracle_dct_matrix(C);
  oracle_zigzag_rank(rank);
  for (int by = 0; by < height / 8; ++by)
    for (int bx = 0; bx < width / 8; ++bx) {
      double x[64], Y[64], T1[64];
      for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) x[i * 8 + j] = (double)src[(int64_t)(8 * by + i) * pitch + 8 * bx + j] - 128.0;
      for (int k = 0; k < 8; ++k) /* T1 = C x */
        for (int j = 0; j < 8; ++j) {
          double acc = 0;
          for (int i = 0; i < 8; ++i) acc += C[k * 8 + i] * x[i * 8 + j];
          T1[k * 8 + j] = acc;
        }
      for (int k = 0; k < 8; ++k) /* Y = T1 C^T, zonal mask */
        for (int l = 0; l < 8; ++l) {
          double acc = 0;
          for (int j = 0; j < 8; ++j) acc += T1[k * 8 + j] * C[l * 8 + j];
          Y[k * 8 + l] = rank[k * 8 + l] < r ? acc : 0.0;
        }
      for (int i = 0; i < 8; ++i) /* T1 = C^T Y */
        for (int l = 0; l < 8; ++l) {
          double acc = 0;
          for (int k = 0; k < 8; ++k) acc += C[k * 8 + i] * Y[k * 8 + l];
          T1[i * 8 + l] = acc;
        }
      for (int i = 0; i < 8; ++i) /* X^ = T1 C, rounded and clamped */
        for (int j = 0; j < 8; ++j) {
          double acc = 0;
          for (int l = 0; l < 8; ++l) acc += T1[i * 8 + l] * C[l * 8 + j];
          double p = rint(acc + 128.0);
          if (p < 0) p = 0;
          if (p > 255) p = 255;
          dst[(int64_t)(8 * by + i) * dst_pitch + 8 * bx + j] = (uint8_t)p;
        }
    }
  return 0;
}
