// Internal interface between the C-ABI layer (adct_api.cu) and the kernel
// translation units (adct_codec*.cu, adct_float.cu, adct_quality.cu).  Not installed.
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
  K_RT_SSE = 6,   // src -> round trip -> squared error against src per plane (nothing stored)
};

// Edge class of a launch (the codec kernel's EDGE parameter): images whose
// sides are multiples of 8; images with edge blocks (right or bottom edge);
// the interiors of split edge images, whose flat rows include a masked last
// block column (descriptor ew = 0) so that their tiles stay aligned.
enum EdgeClass { kEdgeNone = 0, kEdgeBlocks = 1, kEdgeMasked = 2 };

struct LaunchShape {
  int threads;      // per CTA, multiple of 32, at most 256
  int ctas_per_sm;  // persistent grid = SMs x ctas_per_sm (at most)
  int stage_coef;   // 0: direct 16-byte coefficient stores, 1: staged 512-byte warp stores, -1: per kernel
};

struct CodecLaunch {
  const PlaneDesc* planes;  // device
  const int64_t* starts;    // device, nplanes + 1 entries
  int32_t nplanes;
  int64_t total;            // blocks over all planes
  int kind;                 // Kind
  int qmode;                // QMode (quantiser applied by QUANTISE / RT kinds)
  bool evenq;               // the step table has an even step <= 16384 (tie correction needed)
  unsigned long long* sse;  // K_RT_SSE: per-plane sums of squared reconstruction error (device)
  unsigned int* fault;      // checked builds: bits set by the kernels' bounds checks (device; may be NULL)
  int nch;                  // 1: planar planes; 3 or 4: interleaved images
  int edge;                 // edge class: 0 none, 1 edge blocks, 2 interiors with a masked last column
  bool after_interior;      // edge class 1 right after a masked-interior launch on the same stream:
                            // launched as its programmatic dependent (overlaps its tail)
  QuantParams qp;
};

// One instantiation of the integer codec kernel.
using KernelFn = void (*)(const PlaneDesc*, const int64_t*, int32_t, int64_t, int64_t, int, unsigned long long*,
                          unsigned int*, const QuantParams);

// Bits of the fault word of a checked build (ADCT_CHECKED): a tile position
// outside its plane's blocks, a pixel copy past the row pitch.
enum CheckedFault : unsigned int { FAULT_POSITION = 1u, FAULT_ROW_BYTES = 2u };

// Zonal kernels specialised on the zone (adct_codec_zonal_lo.cu: zones
// 0..kZoneLoMax; adct_codec_zonal_hi.cu: up to kZoneHiMax); nullptr when the
// kind / mode pair has no specialisation.
KernelFn pick_zonal_kernel_lo(int kind, int qmode, int zs);
KernelFn pick_zonal_kernel_hi(int kind, int qmode, int zs);
// Kernels for interleaved images of nch = 3 or 4 channels, without and with
// edge blocks (adct_codec_interleaved.cu, adct_codec_interleaved_edge.cu);
// nullptr for kinds without one.
KernelFn pick_interleaved_kernel(int kind, int qmode, bool evenq, int nch);
KernelFn pick_interleaved_edge_kernel(int kind, int qmode, bool evenq, int nch);
// Kernels for planar images with edge blocks (adct_codec_edge.cu).
KernelFn pick_edge_kernel(int kind, int qmode, bool evenq);
// Kernels for the interiors of split edge images, whose descriptors mask
// their last block column (adct_codec_masked.cu: planar;
// adct_codec_interleaved_masked.cu: nch = 3 or 4).
KernelFn pick_masked_kernel(int kind, int qmode, bool evenq);
KernelFn pick_interleaved_masked_kernel(int kind, int qmode, bool evenq, int nch);

// Device allocation of the library (cudaMalloc), with failure injection for
// tests: the environment variable ADCT_FAULT_INJECT=alloc:K makes the K-th
// call of the process (counted from 1) fail with cudaErrorMemoryAllocation
// without allocating, as if the device were out of memory.
cudaError_t device_alloc(void** ptr, size_t bytes);

// Launches the integer codec kernel.  Returns cudaSuccess or the launch error.
cudaError_t launch_codec(const CodecLaunch& c, const LaunchShape& shape, int sm_count, cudaStream_t stream);

// Largest grid the persistent kernel uses for this shape (CTAs), and its dynamic shared memory.
int codec_grid(const LaunchShape& shape, int sm_count, int64_t total);
size_t codec_smem_bytes(const LaunchShape& shape, int kind, int nch = 1, int zs = 14);

// Exact-DCT comparator of the quality sweep: zonal round trip of every block
// with the orthonormal 8x8 DCT-II in float32; per-plane squared error.
cudaError_t launch_dct_quality(const PlaneDesc* planes, const int64_t* starts, int32_t nplanes, int64_t total,
                               const float* dct64, uint64_t keep_mask, unsigned long long* sse, int sm_count,
                               cudaStream_t stream);

// Float variant (Sec. 2 C^ = D T): forward (optionally soft-quantised) and adjoint.
// Per position k = 8 i + j with soft step Q_k: the soft quantiser's phase is
// 2 pi h with h = y / Q_k = v d_i d_j / Q_k (v the unscaled coefficient
// T x T^T): the forward forms it as y rq, the adjoint as v g.
struct FloatParams {
  float c2pi[64];  // Q / (2 pi)
  float rq[64];    // 1 / Q
  float g[64];     // d_i d_j / Q
};
cudaError_t launch_float_forward(const float* x, float* y, int64_t planes, int32_t H, int32_t W,
                                 const FloatParams* fp, int sm_count, cudaStream_t stream);
cudaError_t launch_float_backward(const float* x, const float* gy, float* gx, int64_t planes, int32_t H,
                                  int32_t W, const FloatParams* fp, int sm_count, cudaStream_t stream);

}  // namespace adct
