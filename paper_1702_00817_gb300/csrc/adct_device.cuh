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

// Inverse 8-point transform x = T^T X on v[0], v[S], ..., v[7S], in place:
// the transposed flow graph T^T = A1^T A2^T A3^T P^T = A1 A2 A3 P^T (A1, A2, A3
// are symmetric), again 14 additions.
template <int S, class V>
__host__ __device__ __forceinline__ void inv8(V* v) {
  const V X0 = v[0], X1 = v[S], X2 = v[2 * S], X3 = v[3 * S];
  const V X4 = v[4 * S], X5 = v[5 * S], X6 = v[6 * S], X7 = v[7 * S];
  const V c0 = X0 + X4, c1 = X0 - X4;  // A3 after P^T
  const V b0 = c0 + X2, b3 = c0 - X2;  // A2 rows 0, 3
  const V b1 = c1 - X6, b2 = c1 + X6;  // A2 rows 1, 2 (A3's sign on row 2 absorbed)
  v[0] = b0 + X1;                      // A1 (its -1 entries absorbed)
  v[7 * S] = b0 - X1;
  v[1 * S] = b1 - X5;
  v[6 * S] = b1 + X5;
  v[2 * S] = b2 - X3;
  v[5 * S] = b2 + X3;
  v[3 * S] = b3 - X7;
  v[4 * S] = b3 + X7;
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

// One plane of the flattened block index.  Planes of a multi-channel image
// are separate entries.  Block f of the plane (row-major over blocks) sits at
// src + (8 * (f / wb)) * pitch + 8 * (f % wb); its coefficients at coef + 64 f.
struct PlaneDesc {
  const uint8_t* src;
  uint8_t* dst;
  int16_t* coef;
  int64_t pitch;
  int64_t first;  // flat index of the plane's block 0
  int32_t wb;     // blocks per row
  int32_t hb;     // block rows
};
static_assert(sizeof(PlaneDesc) == 48, "descriptor layout");

// Per-call quantiser constants, passed by value (they live in the kernel
// parameter bank, so the unrolled per-position accesses are free operands).
//   magic/bias: floor((|Z| + bias) / Q) == umulhi(|Z| + bias, magic) with
//               magic = ceil(2^32 / Q), bias = floor(Q / 2) for Q >= 2, and
//               magic = 2^32 - 1, bias = 1 for Q = 1 (exact for |Z| + bias < 2^16).
//   w:          dequantisation weight Q_ij * 2^(6 - a_i - a_j) (D^2 merged).
//   keep:       -1 where the zig-zag rank is below r, 0 elsewhere.
struct QuantParams {
  uint32_t magic[64];
  uint32_t bias[64];
  int32_t w[64];
  int32_t keep[64];
};

enum QMode { QM_NONE = 0, QM_STEP = 1, QM_ZONAL = 2, QM_STEP_ZONAL = 3 };

// Round half away from zero of z / Q for |z| <= 8192:
// sgn(z) * floor((|z| + floor(Q/2)) / Q), the division by the magic multiply.
__device__ __forceinline__ int32_t quant_step(int32_t z, uint32_t magic, uint32_t bias) {
  const uint32_t mag = (uint32_t)(z < 0 ? -z : z) + bias;
  const int32_t q = (int32_t)__umulhi(mag, magic);
  return z < 0 ? -q : q;
}

template <int QMODE>
__device__ __forceinline__ int32_t quantise1(int32_t z, const QuantParams& qp, int k) {
  int32_t q = z;
  if (QMODE == QM_STEP || QMODE == QM_STEP_ZONAL) q = quant_step(z, qp.magic[k], qp.bias[k]);
  if (QMODE == QM_ZONAL || QMODE == QM_STEP_ZONAL) q &= qp.keep[k];
  return q;
}

}  // namespace adct
