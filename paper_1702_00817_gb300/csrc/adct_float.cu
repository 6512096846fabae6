// Differentiable float32 variant of the transform (Sec. 2: C^ = D T is
// orthogonal) for sm_103a.  Forward: y = D T x T^T D per 8x8 block, then the
// optional soft quantiser y - (Q/2pi) sin(2pi y/Q).  Backward (adjoint):
// gx = T^T D (gy * (1 - cos(2pi y/Q))) D T, with y recomputed from x so the
// forward saves nothing but x.  T and T^T are applied with the same
// 14-addition butterflies as the integer codec (fadd only); D enters as one
// multiply per coefficient.  One thread per block, rows then columns.
#include <cuda_runtime.h>

#include "adct_internal.h"

namespace adct {
namespace {

constexpr int kFloatThreads = 128;  // with 3 CTAs per SM: up to 168 registers (sinpif/cospif unrolled 64 times)

// d_i = 2^(-a_i / 2): 1/sqrt8, 1/sqrt2, 1/2 (Sec. 2, matrix D)
__host__ __device__ constexpr float d_of(int i) {
  return scale_exp(i) == 3 ? 0.35355339059327373f : (scale_exp(i) == 2 ? 0.5f : 0.70710678118654752f);
}

__device__ __forceinline__ void load_block(const float* __restrict__ p, int32_t W, float* v) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float4 a = __ldcs((const float4*)(p + (int64_t)i * W));
    const float4 b = __ldcs((const float4*)(p + (int64_t)i * W) + 1);
    v[8 * i + 0] = a.x; v[8 * i + 1] = a.y; v[8 * i + 2] = a.z; v[8 * i + 3] = a.w;
    v[8 * i + 4] = b.x; v[8 * i + 5] = b.y; v[8 * i + 6] = b.z; v[8 * i + 7] = b.w;
  }
}

__device__ __forceinline__ void store_block(float* __restrict__ p, int32_t W, const float* v) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    __stcs((float4*)(p + (int64_t)i * W), make_float4(v[8 * i + 0], v[8 * i + 1], v[8 * i + 2], v[8 * i + 3]));
    __stcs((float4*)(p + (int64_t)i * W) + 1, make_float4(v[8 * i + 4], v[8 * i + 5], v[8 * i + 6], v[8 * i + 7]));
  }
}

__device__ __forceinline__ int64_t block_offset(int64_t g, int64_t nb, int32_t wb, int32_t H, int32_t W) {
  const int64_t plane = g / nb;
  const int64_t f = g - plane * nb;
  const int64_t by = f / wb, bx = f - by * wb;
  return plane * (int64_t)H * W + 8 * by * (int64_t)W + 8 * bx;
}

template <bool SOFT>
__global__ void __launch_bounds__(kFloatThreads, 3) k_float_fwd(const float* __restrict__ x, float* __restrict__ y, int64_t total,
                                                   int64_t nb, int32_t wb, int32_t H, int32_t W, const FloatParams fp) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t off = block_offset(g, nb, wb, H, W);
    float v[64];
    load_block(x + off, W, v);
    fwd2d(v);
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int k = 8 * i + j;
        float t = v[k] * (d_of(i) * d_of(j));
        if (SOFT) t = t - fp.c2pi[k] * sinpif(t * fp.r2[k]);
        v[k] = t;
      }
    store_block(y + off, W, v);
  }
}

template <bool SOFT>
__global__ void __launch_bounds__(kFloatThreads, 3) k_float_bwd(const float* __restrict__ x, const float* __restrict__ gy,
                                                      float* __restrict__ gx, int64_t total, int64_t nb, int32_t wb,
                                                      int32_t H, int32_t W, const FloatParams fp) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t off = block_offset(g, nb, wb, H, W);
    // v <- dz/dy * d_i d_j per coefficient (y recomputed from x), then v <- gy * v
    float v[64];
    if (SOFT) {
      load_block(x + off, W, v);
      fwd2d(v);
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int k = 8 * i + j;
          const float dd = d_of(i) * d_of(j);
          v[k] = (1.0f - cospif(v[k] * dd * fp.r2[k])) * dd;
        }
    }
    const float* gp = gy + off;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float4 a = __ldcs((const float4*)(gp + (int64_t)i * W));
      const float4 b = __ldcs((const float4*)(gp + (int64_t)i * W) + 1);
      const float r[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
      for (int j = 0; j < 8; ++j) v[8 * i + j] = SOFT ? r[j] * v[8 * i + j] : r[j] * (d_of(i) * d_of(j));
    }
    inv2d(v);
    store_block(gx + off, W, v);
  }
}

int float_grid(int64_t total, int sm_count) {
  int64_t want = (total + kFloatThreads - 1) / kFloatThreads;
  const int64_t cap = (int64_t)sm_count * 3;
  if (want > cap) want = cap;
  return (int)(want < 1 ? 1 : want);
}

}  // namespace

cudaError_t launch_float_forward(const float* x, float* y, int64_t planes, int32_t H, int32_t W,
                                 const FloatParams* fp, int sm_count, cudaStream_t stream) {
  const int32_t wb = W / 8;
  const int64_t nb = (int64_t)(H / 8) * wb;
  const int64_t total = planes * nb;
  if (total <= 0) return cudaSuccess;
  FloatParams none{};
  const int grid = float_grid(total, sm_count);
  if (fp) k_float_fwd<true><<<grid, kFloatThreads, 0, stream>>>(x, y, total, nb, wb, H, W, *fp);
  else k_float_fwd<false><<<grid, kFloatThreads, 0, stream>>>(x, y, total, nb, wb, H, W, none);
  return cudaGetLastError();
}

cudaError_t launch_float_backward(const float* x, const float* gy, float* gx, int64_t planes, int32_t H,
                                  int32_t W, const FloatParams* fp, int sm_count, cudaStream_t stream) {
  const int32_t wb = W / 8;
  const int64_t nb = (int64_t)(H / 8) * wb;
  const int64_t total = planes * nb;
  if (total <= 0) return cudaSuccess;
  FloatParams none{};
  const int grid = float_grid(total, sm_count);
  if (fp) k_float_bwd<true><<<grid, kFloatThreads, 0, stream>>>(x, gy, gx, total, nb, wb, H, W, *fp);
  else k_float_bwd<false><<<grid, kFloatThreads, 0, stream>>>(x, gy, gx, total, nb, wb, H, W, none);
  return cudaGetLastError();
}

}  // namespace adct
