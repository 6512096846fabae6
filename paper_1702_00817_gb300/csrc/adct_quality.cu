// Exact-DCT comparator for the quality sweep (the protocol of Sec. 3 / Fig. 2:
// PSNR and the MSE percentage error of the approximation relative to the DCT
// as functions of the number r of retained zig-zag coefficients).  Every 8x8
// block goes through the orthonormal 8x8 DCT-II in float32, keeps the first r
// zig-zag coefficients, is inverted, rounded to 8 bits and compared with the
// input; per-plane squared errors accumulate in 64-bit counters.  One thread
// per block over the flattened block index of the plane descriptor table.
#include <cuda_runtime.h>

#include "adct_internal.h"

namespace adct {
namespace {

struct DctParams {
  float c[64];         // C[k][j] = alpha_k cos(pi (2j + 1) k / 16), row-major
  uint64_t keep_mask;  // bit 8i + j set when coefficient (i, j) is kept
};

__global__ void __launch_bounds__(128) k_dct_quality(const PlaneDesc* __restrict__ planes,
                                                     const int64_t* __restrict__ starts, int32_t nplanes,
                                                     int64_t total, const DctParams p,
                                                     unsigned long long* __restrict__ sse) {
  unsigned long long acc = 0;
  int acc_plane = -1;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nplanes;  // plane of block g
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(starts + mid) <= g) lo = mid; else hi = mid;
    }
    const PlaneDesc* d = planes + lo;
    const uint32_t wb = (uint32_t)__ldg(&d->wb);
    const uint32_t f = (uint32_t)(g - __ldg(starts + lo));
    const uint32_t by = f / wb, bx = f - by * wb;
    const int64_t pitch = __ldg(&d->pitch);
    const uint8_t* src = (const uint8_t*)__ldg((const unsigned long long*)&d->src) + (int64_t)(8 * by) * pitch + 8 * bx;
    float x[64], t[64];
    uint2 raw[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      raw[i] = *(const uint2*)(src + i * pitch);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        x[8 * i + j] = (float)((raw[i].x >> (8 * j)) & 0xFF) - 128.0f;
        x[8 * i + 4 + j] = (float)((raw[i].y >> (8 * j)) & 0xFF) - 128.0f;
      }
    }
    // Y = C X C^T (rows, then columns), zonal mask
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int l = 0; l < 8; ++l) {
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) s = fmaf(x[8 * i + j], p.c[8 * l + j], s);
        t[8 * i + l] = s;
      }
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int l = 0; l < 8; ++l) {
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) s = fmaf(p.c[8 * k + i], t[8 * i + l], s);
        x[8 * k + l] = ((p.keep_mask >> (8 * k + l)) & 1ull) ? s : 0.f;
      }
    // X^ = C^T Y C
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int l = 0; l < 8; ++l) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) s = fmaf(p.c[8 * k + i], x[8 * k + l], s);
        t[8 * i + l] = s;
      }
    uint32_t err = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float s = 0.f;
#pragma unroll
        for (int l = 0; l < 8; ++l) s = fmaf(t[8 * i + l], p.c[8 * l + j], s);
        const int rec = (int)fminf(fmaxf(rintf(s + 128.0f), 0.0f), 255.0f);
        const int org = (int)(((j < 4 ? raw[i].x : raw[i].y) >> (8 * (j & 3))) & 0xFF);
        err += (uint32_t)((rec - org) * (rec - org));
      }
    if (lo != acc_plane) {
      if (acc_plane >= 0) atomicAdd(sse + acc_plane, acc);
      acc_plane = lo;
      acc = 0;
    }
    acc += err;
  }
  if (acc_plane >= 0) atomicAdd(sse + acc_plane, acc);
}

}  // namespace

cudaError_t launch_dct_quality(const PlaneDesc* planes, const int64_t* starts, int32_t nplanes, int64_t total,
                               const float* dct64, uint64_t keep_mask, unsigned long long* sse, int sm_count,
                               cudaStream_t stream) {
  if (total <= 0) return cudaSuccess;
  DctParams p;
  for (int k = 0; k < 64; ++k) p.c[k] = dct64[k];
  p.keep_mask = keep_mask;
  int64_t grid = (total + 127) / 128;
  if (grid > (int64_t)sm_count * 8) grid = (int64_t)sm_count * 8;
  k_dct_quality<<<(int)grid, 128, 0, stream>>>(planes, starts, nplanes, total, p, sse);
  return cudaGetLastError();
}

}  // namespace adct
