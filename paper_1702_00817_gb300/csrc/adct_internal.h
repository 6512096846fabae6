// Internal interface between the C-ABI layer (adct_api.cu) and the kernel
// translation units (adct_codec.cu, adct_float.cu).  Not installed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "adct_device.cuh"

namespace adct {

// What one launch of the integer codec kernel does per block.
enum Kind {
  K_FORWARD = 0,  // src -> coef (Z)
  K_QUANTISE = 1, // coef -> coef (q), in place
  K_INVERSE = 2,  // coef (q) -> dst
  K_RT_FULL = 3,  // src -> coef (q) and dst
  K_RT_PIX = 4,   // src -> dst (q not stored)
  K_RT_COEF = 5,  // src -> coef (q), no reconstruction (encode)
};

struct LaunchShape {
  int threads;            // per CTA, multiple of 32
  int ctas_per_sm;
  int blocks_per_thread;  // 1 or 2
  int stage_coef;         // 0 or 1
};

struct CodecLaunch {
  const PlaneDesc* planes;  // device
  const int64_t* starts;    // device, nplanes + 1 entries
  int32_t nplanes;
  int64_t total;            // blocks over all planes
  int kind;                 // Kind
  int qmode;                // QMode (quantiser applied by QUANTISE / RT kinds)
  bool pitch16;             // every plane's src/dst and pitch are 16-byte aligned, wb even
  QuantParams qp;
};

// Launches the integer codec kernel.  Returns cudaSuccess or the launch error.
cudaError_t launch_codec(const CodecLaunch& c, const LaunchShape& shape, int sm_count, cudaStream_t stream);

// Largest grid the persistent kernel uses for this shape (CTAs).
int codec_grid(const LaunchShape& shape, int sm_count, int64_t total);

// Float variant (Sec. 2 C^ = D T): forward (optionally soft-quantised) and adjoint.
struct FloatParams {
  float c2pi[64];  // Q / (2 pi)
  float r2[64];    // 2 / Q  (sin(2 pi y / Q) = sinpi(y * 2 / Q))
};
cudaError_t launch_float_forward(const float* x, float* y, int64_t planes, int32_t H, int32_t W,
                                 const FloatParams* fp, int sm_count, cudaStream_t stream);
cudaError_t launch_float_backward(const float* x, const float* gy, float* gx, int64_t planes, int32_t H,
                                  int32_t W, const FloatParams* fp, int sm_count, cudaStream_t stream);

}  // namespace adct
