// Instantiation and launch of the integer codec kernel (the kernel itself is
// in adct_codec_kernel.cuh): every kind and quantiser mode with the full zone,
// plus the dispatch to the zone-specialised zonal kernels.
#include "adct_codec_kernel.cuh"

namespace adct {
namespace {

constexpr int kZoneAll = 14;  // anti-diagonals 0..14: every coefficient

template <int KIND, bool EVENQ>
KernelFn pick_mode(int qmode) {
  switch (qmode) {
    case QM_ZONAL_ZZ: return (KIND == K_RT_FULL || KIND == K_RT_COEF) ? k_codec<KIND, QM_ZONAL_ZZ, false, kZoneAll>
                                                                     : k_codec<KIND, QM_ZONAL, false, kZoneAll>;
    case QM_STEP: return k_codec<KIND, QM_STEP, EVENQ, kZoneAll>;
    case QM_ZONAL: return k_codec<KIND, QM_ZONAL, false, kZoneAll>;
    case QM_STEP_ZONAL: return k_codec<KIND, QM_STEP_ZONAL, EVENQ, kZoneAll>;
    default: return k_codec<KIND, QM_NONE, false, kZoneAll>;
  }
}

template <bool EVENQ>
KernelFn pick_kernel_q(int kind, int qmode) {
  switch (kind) {
    case K_FORWARD: return k_codec<K_FORWARD, QM_NONE, false, kZoneAll>;
    case K_QUANTISE:
      switch (qmode) {
        case QM_STEP: return k_codec<K_QUANTISE, QM_STEP, EVENQ, kZoneAll>;
        case QM_ZONAL: return k_codec<K_QUANTISE, QM_ZONAL, false, kZoneAll>;
        case QM_STEP_ZONAL: return k_codec<K_QUANTISE, QM_STEP_ZONAL, EVENQ, kZoneAll>;
        default: return nullptr;
      }
    case K_INVERSE:
      return qmode == QM_ZONAL_ZZ ? k_codec<K_INVERSE, QM_ZONAL_ZZ, false, kZoneAll>
                                  : k_codec<K_INVERSE, QM_NONE, false, kZoneAll>;
    case K_RT_FULL: return pick_mode<K_RT_FULL, EVENQ>(qmode);
    case K_RT_PIX: return pick_mode<K_RT_PIX, EVENQ>(qmode);
    case K_RT_COEF: return pick_mode<K_RT_COEF, EVENQ>(qmode);
    case K_RT_SSE: return pick_mode<K_RT_SSE, EVENQ>(qmode);
    default: return nullptr;
  }
}

KernelFn pick_kernel(int kind, int qmode, bool evenq) {
  return evenq ? pick_kernel_q<true>(kind, qmode) : pick_kernel_q<false>(kind, qmode);
}

}  // namespace

namespace {
template <int NCH>
int warp_smem_n(int kind) {
  switch (kind) {
    case K_FORWARD: return SmemPlan<K_FORWARD, NCH>::warp;
    case K_QUANTISE: return SmemPlan<K_QUANTISE, NCH>::warp;
    case K_INVERSE: return SmemPlan<K_INVERSE, NCH>::warp;
    case K_RT_FULL: return SmemPlan<K_RT_FULL, NCH>::warp;
    case K_RT_PIX: return SmemPlan<K_RT_PIX, NCH>::warp;
    case K_RT_SSE: return SmemPlan<K_RT_SSE, NCH>::warp;
    default: return SmemPlan<K_RT_COEF, NCH>::warp;
  }
}
int warp_smem(int kind, int nch) {
  return nch == 3 ? warp_smem_n<3>(kind) : nch == 4 ? warp_smem_n<4>(kind) : warp_smem_n<1>(kind);
}
}  // namespace

// CTAs per SM when the caller leaves the choice to the library (measured on
// 256 x 1080x1920 batches): four, except three for the encode with dense
// coefficient output, whose 192 bytes of traffic per block run best with
// fewer requests in flight.  Capped at the resident count, which is three for
// the kernels that use more than 128 registers.
int default_ctas_per_sm(int kind, int qmode) { return (kind == K_RT_COEF && qmode != QM_ZONAL_ZZ) ? 3 : 4; }

size_t codec_smem_bytes(const LaunchShape& shape, int kind, int nch) {
  return (size_t)(shape.threads / 32) * warp_smem(kind, nch);
}

int codec_grid(const LaunchShape& shape, int sm_count, int64_t total) {
  int64_t want = (total + shape.threads - 1) / shape.threads;
  const int64_t cap = (int64_t)sm_count * (shape.ctas_per_sm > 0 ? shape.ctas_per_sm : 4);
  if (want > cap) want = cap;
  return (int)(want < 1 ? 1 : want);
}

cudaError_t launch_codec(const CodecLaunch& c, const LaunchShape& shape, int sm_count, cudaStream_t stream) {
  if (c.total <= 0) return cudaSuccess;
  KernelFn fn = nullptr;
  if (c.nch == 3 || c.nch == 4) {
    fn = c.edge ? pick_interleaved_edge_kernel(c.kind, c.qmode, c.evenq, c.nch)
                : pick_interleaved_kernel(c.kind, c.qmode, c.evenq, c.nch);
    if (!fn) return cudaErrorInvalidValue;
  } else if (c.edge) {
    fn = pick_edge_kernel(c.kind, c.qmode, c.evenq);
    if (!fn) return cudaErrorInvalidValue;
  } else if (c.qmode == QM_ZONAL || c.qmode == QM_ZONAL_ZZ) {
    const int zs = zone_for(c.qp.r);
    if (zs <= kZoneLoMax) fn = pick_zonal_kernel_lo(c.kind, c.qmode, zs);
    else if (zs <= kZoneHiMax) fn = pick_zonal_kernel_hi(c.kind, c.qmode, zs);
  }
  if (!fn) fn = pick_kernel(c.kind, c.qmode, c.evenq);
  if (!fn) return cudaErrorInvalidValue;
  if (shape.threads < 32 || shape.threads > kMaxThreads || shape.threads % 32) return cudaErrorInvalidValue;
  const size_t smem = codec_smem_bytes(shape, c.kind, c.nch);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  // never size the persistent grid beyond what can be resident at once
  int resident = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, fn, shape.threads, smem) != cudaSuccess || resident < 1)
    resident = 1;
  LaunchShape sh = shape;
  if (sh.ctas_per_sm == 0) sh.ctas_per_sm = default_ctas_per_sm(c.kind, c.qmode);
  if (sh.ctas_per_sm > resident) sh.ctas_per_sm = resident;
  const int grid = codec_grid(sh, sm_count, c.total);
  const int64_t warps = (int64_t)grid * (shape.threads / 32);
  int64_t chunk = (c.total + warps - 1) / warps;
  chunk = (chunk + kTile - 1) / kTile * kTile;
  fn<<<grid, shape.threads, smem, stream>>>(c.planes, c.starts, c.nplanes, c.total, chunk, shape.stage_coef, c.sse,
                                            c.fault, c.qp);
  return cudaGetLastError();
}

}  // namespace adct
