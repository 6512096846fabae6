// Integer codec kernels for sm_103a: the blockwise 2D 14-addition transform
// (Sec. 2 fast algorithm; Sec. 3 8x8 blocks), the D^2-merged quantiser and
// the inverse, as one persistent kernel over a flattened block index.
//
// Work split: the grid is sized to the SMs (persistent); each warp owns a
// contiguous chunk of the flat block index and walks it 32 blocks at a time,
// one 8x8 block per lane, so every row load of a warp reads 32 adjacent
// blocks = 256 contiguous bytes of an image row.  The 8x8 block lives in 64
// registers; both passes of the separable transform and the transpose
// between them are register renaming.  The path is add-only and bound by
// HBM bytes, so no tensor cores are involved.
#include <cuda_runtime.h>

#include "adct_internal.h"

namespace adct {
namespace {

constexpr int kMaxThreads = 256;

__device__ __forceinline__ int32_t sext_lo16(uint32_t w) { return (int32_t)(int16_t)(w & 0xFFFFu); }
__device__ __forceinline__ int32_t sext_hi16(uint32_t w) { return ((int32_t)w) >> 16; }
__device__ __forceinline__ uint32_t pack16(int32_t lo, int32_t hi) {
  return __byte_perm((uint32_t)lo, (uint32_t)hi, 0x5410);
}
__device__ __forceinline__ uint32_t clamp_u8(int32_t r) { return (uint32_t)min(max(r >> 6, 0), 255); }
__device__ __forceinline__ uint32_t pack_u8x4(uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  return __byte_perm(__byte_perm(a, b, 0x0040), __byte_perm(c, d, 0x0040), 0x5410);
}

template <int KIND>
struct KindTraits {
  static constexpr bool in_pix = (KIND == K_FORWARD || KIND == K_RT_FULL || KIND == K_RT_PIX || KIND == K_RT_COEF);
  static constexpr bool quant = (KIND == K_QUANTISE || KIND == K_RT_FULL || KIND == K_RT_PIX || KIND == K_RT_COEF);
  static constexpr bool write_coef = (KIND == K_FORWARD || KIND == K_QUANTISE || KIND == K_RT_FULL || KIND == K_RT_COEF);
  static constexpr bool inv = (KIND == K_INVERSE || KIND == K_RT_FULL || KIND == K_RT_PIX);
};

template <int KIND, int QMODE>
__global__ void __launch_bounds__(kMaxThreads, 2)
k_codec(const PlaneDesc* __restrict__ planes, const int64_t* __restrict__ starts, int32_t nplanes, int64_t total,
        int64_t chunk, const QuantParams qp) {
  using KT = KindTraits<KIND>;
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t begin = gwarp * chunk;
  if (begin >= total) return;
  const int64_t end = min(total, begin + chunk);

  // plane holding `begin`: largest p with starts[p] <= begin
  int lo = 0, hi = nplanes;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(starts + mid) <= begin) lo = mid; else hi = mid;
  }
  int p = lo;
  int64_t next_start = __ldg(starts + p + 1);

  for (int64_t g = begin + lane; g < end; g += 32) {
    while (g >= next_start) {
      ++p;
      next_start = __ldg(starts + p + 1);
    }
    const PlaneDesc* d = planes + p;
    const int64_t first = __ldg(&d->first);
    const int32_t wb = __ldg(&d->wb);
    const uint32_t f = (uint32_t)(g - first);
    const uint32_t by = f / (uint32_t)wb;
    const uint32_t bx = f - by * (uint32_t)wb;
    const int64_t pitch = __ldg(&d->pitch);
    const int64_t pix_off = (int64_t)(8 * by) * pitch + 8 * bx;

    int32_t v[64];
    if (KT::in_pix) {
      const uint8_t* s = (const uint8_t*)__ldg((const unsigned long long*)&d->src) + pix_off;
      uint2 w[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) w[i] = __ldcs((const uint2*)(s + i * pitch));
#pragma unroll
      for (int i = 0; i < 8; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          v[8 * i + j] = (int32_t)__byte_perm(w[i].x, 0u, 0x4440 | j);
          v[8 * i + 4 + j] = (int32_t)__byte_perm(w[i].y, 0u, 0x4440 | j);
        }
      }
      fwd2d(v);
      v[0] -= 8192;  // level shift: T (X - 128) T^T = T X T^T - 8192 e0 e0^T (T 1 = 8 e0)
    } else {
      const int16_t* c = (const int16_t*)__ldg((const unsigned long long*)&d->coef) + (int64_t)f * 64;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int4 u = __ldcs((const int4*)c + t);
        v[8 * t + 0] = sext_lo16(u.x); v[8 * t + 1] = sext_hi16(u.x);
        v[8 * t + 2] = sext_lo16(u.y); v[8 * t + 3] = sext_hi16(u.y);
        v[8 * t + 4] = sext_lo16(u.z); v[8 * t + 5] = sext_hi16(u.z);
        v[8 * t + 6] = sext_lo16(u.w); v[8 * t + 7] = sext_hi16(u.w);
      }
    }

    if (KT::quant) {
#pragma unroll
      for (int k = 0; k < 64; ++k) v[k] = quantise1<QMODE>(v[k], qp, k);
    }

    if (KT::write_coef) {
      int16_t* c = (int16_t*)__ldg((const unsigned long long*)&d->coef) + (int64_t)f * 64;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        int4 u;
        u.x = (int)pack16(v[8 * t + 0], v[8 * t + 1]);
        u.y = (int)pack16(v[8 * t + 2], v[8 * t + 3]);
        u.z = (int)pack16(v[8 * t + 4], v[8 * t + 5]);
        u.w = (int)pack16(v[8 * t + 6], v[8 * t + 7]);
        __stcs((int4*)c + t, u);
      }
    }

    if (KT::inv) {
#pragma unroll
      for (int k = 0; k < 64; ++k) v[k] *= qp.w[k];
      // +32 rounding and +128 level shift on every pixel: T^T e0 = 1, so
      // adding 32 + 128 * 64 to S_00 adds it to all of R.
      v[0] += 8224;
      inv2d(v);
      uint8_t* o = (uint8_t*)__ldg((const unsigned long long*)&d->dst) + pix_off;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        uint2 w;
        w.x = pack_u8x4(clamp_u8(v[8 * i + 0]), clamp_u8(v[8 * i + 1]), clamp_u8(v[8 * i + 2]), clamp_u8(v[8 * i + 3]));
        w.y = pack_u8x4(clamp_u8(v[8 * i + 4]), clamp_u8(v[8 * i + 5]), clamp_u8(v[8 * i + 6]), clamp_u8(v[8 * i + 7]));
        __stcs((uint2*)(o + i * pitch), w);
      }
    }
  }
}

using KernelFn = void (*)(const PlaneDesc*, const int64_t*, int32_t, int64_t, int64_t, const QuantParams);

template <int KIND>
KernelFn pick_mode(int qmode) {
  switch (qmode) {
    case QM_STEP: return k_codec<KIND, QM_STEP>;
    case QM_ZONAL: return k_codec<KIND, QM_ZONAL>;
    case QM_STEP_ZONAL: return k_codec<KIND, QM_STEP_ZONAL>;
    default: return k_codec<KIND, QM_NONE>;
  }
}

KernelFn pick_kernel(int kind, int qmode) {
  switch (kind) {
    case K_FORWARD: return k_codec<K_FORWARD, QM_NONE>;
    case K_QUANTISE:
      switch (qmode) {
        case QM_STEP: return k_codec<K_QUANTISE, QM_STEP>;
        case QM_ZONAL: return k_codec<K_QUANTISE, QM_ZONAL>;
        case QM_STEP_ZONAL: return k_codec<K_QUANTISE, QM_STEP_ZONAL>;
        default: return nullptr;
      }
    case K_INVERSE: return k_codec<K_INVERSE, QM_NONE>;
    case K_RT_FULL: return pick_mode<K_RT_FULL>(qmode);
    case K_RT_PIX: return pick_mode<K_RT_PIX>(qmode);
    case K_RT_COEF: return pick_mode<K_RT_COEF>(qmode);
    default: return nullptr;
  }
}

}  // namespace

int codec_grid(const LaunchShape& shape, int sm_count, int64_t total) {
  const int64_t per_cta = shape.threads;  // one block per lane per pass
  int64_t want = (total + per_cta - 1) / per_cta;
  int64_t cap = (int64_t)sm_count * shape.ctas_per_sm;
  if (want > cap) want = cap;
  return (int)(want < 1 ? 1 : want);
}

cudaError_t launch_codec(const CodecLaunch& c, const LaunchShape& shape, int sm_count, cudaStream_t stream) {
  if (c.total <= 0) return cudaSuccess;
  KernelFn fn = pick_kernel(c.kind, c.qmode);
  if (!fn) return cudaErrorInvalidValue;
  if (shape.threads < 32 || shape.threads > kMaxThreads || shape.threads % 32) return cudaErrorInvalidValue;
  const int grid = codec_grid(shape, sm_count, c.total);
  const int64_t warps = (int64_t)grid * (shape.threads / 32);
  int64_t chunk = (c.total + warps - 1) / warps;
  chunk = (chunk + 31) / 32 * 32;
  fn<<<grid, shape.threads, 0, stream>>>(c.planes, c.starts, c.nplanes, c.total, chunk, c.qp);
  return cudaGetLastError();
}

}  // namespace adct
