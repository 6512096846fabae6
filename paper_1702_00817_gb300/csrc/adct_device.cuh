// Device-side building blocks of the codec: the 14-addition butterfly of
// Bayer & Cintra (Sec. 2, T = P A3 A2 A1), its transpose for the inverse, the
// D^2-merged quantiser, and the descriptor/parameter structures the kernels
// read.  Everything here is templated on the value type so that the host-side
// diagnostic (adct_butterfly_host) instantiates exactly the code the kernels run.
#pragma once

#include <stdint.h>

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace adct {

// D^2 = diag(2^-a_i) with a = (3, 1, 2, 1, 3, 1, 2, 1): Sec. 2, matrix D.
__host__ __device__ constexpr int scale_exp(int i) {
  return (i == 0 || i == 4) ? 3 : ((i == 2 || i == 6) ? 2 : 1);
}

// Forward 8-point transform X = T x on v[0], v[S], ..., v[7S], in place.
// Sec. 2 factorisation T = P A3 A2 A1:
//   A1: the four sums x_k + x_{7-k} and four differences x_k - x_{7-k} (8 adds);
//   A2: sums/differences of the first four (4 adds) and -1 on rows 4..6, which
//       is absorbed by subtracting in the opposite order;
//   A3: sum/difference of the first two (2 adds) and -1 on row 2 (absorbed);
//   P : the output permutation (register renaming only).
// 14 additions, no multiplications, no shifts (Table 1).
template <int S, class V>
__host__ __device__ __forceinline__ void fwd8(V* v) {
  const V x0 = v[0], x1 = v[S], x2 = v[2 * S], x3 = v[3 * S];
  const V x4 = v[4 * S], x5 = v[5 * S], x6 = v[6 * S], x7 = v[7 * S];
  const V b0 = x0 + x7, b1 = x1 + x6, b2 = x2 + x5, b3 = x3 + x4;  // A1, upper half
  v[1 * S] = x0 - x7;                                               // A1 row 7 -> X1
  v[3 * S] = x5 - x2;                                               // -(A1 row 5) -> X3
  v[5 * S] = x6 - x1;                                               // -(A1 row 6) -> X5
  v[7 * S] = x4 - x3;                                               // -(A1 row 4) -> X7
  const V c0 = b0 + b3, c1 = b1 + b2;                               // A2 rows 0, 1
  v[2 * S] = b0 - b3;                                               // A2 row 3 -> X2
  v[6 * S] = b2 - b1;                                               // -(A2 row 2) -> X6
  v[0] = c0 + c1;                                                   // A3 row 0 -> X0
  v[4 * S] = c0 - c1;                                               // A3 row 1 -> X4
}

// Inverse 8-point transform x = T^T X from in[0], in[S], ..., in[7S] into
// out[0], out[S], ..., out[7S] (in and out may alias): the transposed flow
// graph T^T = A1^T A2^T A3^T P^T = A1 A2 A3 P^T (A1, A2, A3 are symmetric),
// again 14 additions.  The input type may differ from the output type: the
// codec passes unevaluated dequantised coefficients (q, w) whose + and - are
// multiply-adds, which merges the D^2 scaling into the first inverse pass.
template <int S, class VI, class VO>
__host__ __device__ __forceinline__ void inv8(const VI* in, VO* out) {
  const VI X0 = in[0], X1 = in[S], X2 = in[2 * S], X3 = in[3 * S];
  const VI X4 = in[4 * S], X5 = in[5 * S], X6 = in[6 * S], X7 = in[7 * S];
  const auto c0 = X0 + X4, c1 = X0 - X4;  // A3 after P^T
  const auto b0 = c0 + X2, b3 = c0 - X2;  // A2 rows 0, 3
  const auto b1 = c1 - X6, b2 = c1 + X6;  // A2 rows 1, 2 (A3's sign on row 2 absorbed)
  out[0] = b0 + X1;                       // A1 (its -1 entries absorbed)
  out[7 * S] = b0 - X1;
  out[1 * S] = b1 - X5;
  out[6 * S] = b1 + X5;
  out[2 * S] = b2 - X3;
  out[5 * S] = b2 + X3;
  out[3 * S] = b3 - X7;
  out[4 * S] = b3 + X7;
}

template <int S, class V>
__host__ __device__ __forceinline__ void inv8(V* v) {
  inv8<S, V, V>(v, v);
}

// Separable 2D forward transform of a row-major 8x8 block: rows, then columns.
template <class V>
__host__ __device__ __forceinline__ void fwd2d(V* v) {
#pragma unroll
  for (int i = 0; i < 8; ++i) fwd8<1>(v + 8 * i);
#pragma unroll
  for (int j = 0; j < 8; ++j) fwd8<8>(v + j);
}

// Separable 2D inverse R = T^T S T: columns (V = T^T S), then rows (R = V T).
template <class V>
__host__ __device__ __forceinline__ void inv2d(V* v) {
#pragma unroll
  for (int j = 0; j < 8; ++j) inv8<8>(v + j);
#pragma unroll
  for (int i = 0; i < 8; ++i) inv8<1>(v + 8 * i);
}

// Same, reading the column pass's input from `in` (another type).
template <class VI, class V>
__host__ __device__ __forceinline__ void inv2d(const VI* in, V* v) {
#pragma unroll
  for (int j = 0; j < 8; ++j) inv8<8, VI, V>(in + j, v + j);
#pragma unroll
  for (int i = 0; i < 8; ++i) inv8<1>(v + 8 * i);
}

// One unit of the flat work index: a planar uint8 plane (the flat index counts
// its 8x8 blocks), or an interleaved image of nch = 3 or 4 channels (the flat
// index counts its 8x8 pixel positions, each carrying nch blocks).  Images
// whose sides are not multiples of 8 are covered by ceil(side / 8) blocks;
// the last block column holds ew valid pixel columns and the last block row
// eh valid rows (1..8), the rest is the edge replicated.  A descriptor may
// cover a rectangle of an image's blocks (its interior, its last block column
// or its last block row): src, dst and coef then point at the rectangle's
// first block, wb x hb are its blocks, cwb is the image's blocks per row (the
// coefficient row stride) and bx0 the rectangle's first block column.
// Block (by, bx) of the descriptor sits at src + (8 by) pitch + 8 nch bx; its
// coefficients at coef + (by cwb + bx) c, c = 64 (or r, packed zonal).
struct PlaneDesc {
  const uint8_t* src;
  uint8_t* dst;
  int16_t* coef;    // channel 0's coefficients
  int64_t pitch;    // bytes between pixel rows
  int64_t cstride;  // int16 between the coefficient planes of consecutive channels
  int32_t wb;       // blocks per row of this descriptor
  int32_t hb;       // block rows of this descriptor
  int32_t cwb;      // blocks per coefficient row (the whole image's blocks per row)
  int32_t plane_id; // plane number of channel 0 in the call (per-plane outputs)
  int16_t ew;       // valid pixel columns of the descriptor's last block column (0: that column
                    // belongs to another launch and is skipped: the interior of a split image)
  int16_t eh;       // valid pixel rows of its last block row
  int16_t nch;      // 1: planar plane; 3, 4: interleaved channels
  int16_t bx0;      // first block column within the image
};
static_assert(sizeof(PlaneDesc) == 64, "descriptor layout");

// Per-call quantiser constants, passed by value: they live in the kernel
// parameter bank, so the fully unrolled per-position accesses are free
// instruction operands.  For position k = 8i + j with step Q:
//   STEP (Q <= 16384): n = Z + c with c = floor(Q/2) + K*Q (+1 when Q = 1), where
//     K = ceil(8193 / Q) keeps n in [0, 2^16); when Q is even and Z < 0 the
//     bias drops by one so that ties round away from zero: ssel is the byte
//     selector 0xBBBB (every byte the sign of byte 3: -1 for Z < 0, else 0)
//     for even Q and 0x4444 (a zero byte: no correction) otherwise.
//     m = umulhi(n, magic) = floor(n / Q) exactly (magic = ceil(2^32 / Q), or
//     2^32 - 1 with the +1 above for Q = 1; exact for n < 2^16, Q <= 2^16),
//     q = m - K = sgn(Z) floor((|Z| + floor(Q/2)) / Q) = round half away from zero of Z / Q.
//   STEP (Q > 16384): |Z| <= 8192 < Q/2, so q = 0: magic = c = K = 0.
//   When Z is computed from raw pixels, Z_00 carries +8192 (the level shift
//   T (X - 128) T^T = T X T^T - 8192 e0 e0^T); c at (0, 0) then includes -8192.
//   w  : dequantisation weight 4 * Q * 2^(6 - a_i - a_j) (D^2 merged; the factor 4
//        puts the pixel in the high byte of a 16-bit value), Q = 1 unless STEP;
//   kw : -K * w, plus 4 * 8224 (8224 = 32 + 128 * 64) at (0, 0), so that S = m * w + kw
//        (8224: rounding of R / 64 and level shift of every pixel, T^T e0 = 1).
//   keep: -1 where the zig-zag rank is below r, 0 elsewhere (ZONAL modes).
struct QuantParams {
  int32_t c[64];
  uint32_t magic[64];
  int32_t K[64];
  uint32_t ssel[64];
  int32_t w[64];
  int32_t kw[64];
  int32_t keep[64];
  int32_t r;  // zonal: number of zig-zag coefficients kept (the packed layout stores r per block)
};

// QM_ZONAL_ZZ: the zonal quantiser with coefficients stored packed, the first
// r zig-zag coefficients of each block (r int16 per block) instead of 64.
enum QMode { QM_NONE = 0, QM_STEP = 1, QM_ZONAL = 2, QM_STEP_ZONAL = 3, QM_ZONAL_ZZ = 4 };

// The standard zig-zag sequence over an 8x8 block (Sec. 3): pos[t] = 8 i + j of
// the t-th coefficient; anti-diagonals s = i + j in order, even s walked with i
// decreasing, odd s with i increasing.
struct ZigZag {
  int pos[64];
};
__host__ __device__ constexpr ZigZag make_zigzag() {
  ZigZag z{};
  int t = 0;
  for (int s = 0; s < 15; ++s) {
    const int lo = s < 8 ? 0 : s - 7, hi = s < 8 ? s : 7;
    if (s % 2 == 0) {
      for (int i = hi; i >= lo; --i) z.pos[t++] = 8 * i + (s - i);
    } else {
      for (int i = lo; i <= hi; ++i) z.pos[t++] = 8 * i + (s - i);
    }
  }
  return z;
}

// Zones of the zonal quantiser: zone s holds the coefficients on anti-diagonals
// 0..s (i + j <= s); zone_count(s) of them.  The first r zig-zag positions lie
// in zone zone_for(r); zones above kZoneHiMax are served by the full zone 14.
__host__ __device__ constexpr int zone_count(int s) {
  int n = 0;
  for (int d = 0; d <= s; ++d) n += d < 8 ? d + 1 : 15 - d;
  return n;
}
constexpr int kZoneLoMax = 4;  // zones 0..4: r <= 15
constexpr int kZoneHiMax = 8;  // zones 5..8: r <= 43
inline int zone_for(int r) {
  for (int s = 0; s <= kZoneHiMax; ++s)
    if (r <= zone_count(s)) return s;
  return 14;
}

}  // namespace adct
