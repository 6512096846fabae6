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

// Packed zonal layout with r = 64 (the dense layout in zig-zag order).
KernelFn pick_zz64(int kind) {
  switch (kind) {
    case K_RT_FULL: return k_codec<K_RT_FULL, QM_ZONAL_ZZ, false, kZoneZZ64>;
    case K_RT_COEF: return k_codec<K_RT_COEF, QM_ZONAL_ZZ, false, kZoneZZ64>;
    case K_INVERSE: return k_codec<K_INVERSE, QM_ZONAL_ZZ, false, kZoneZZ64>;
    default: return nullptr;
  }
}

}  // namespace

namespace {
template <int NCH, int ZS>
int warp_smem_z(int kind) {
  switch (kind) {
    case K_FORWARD: return SmemPlan<K_FORWARD, NCH, ZS>::warp;
    case K_QUANTISE: return SmemPlan<K_QUANTISE, NCH, ZS>::warp;
    case K_INVERSE: return SmemPlan<K_INVERSE, NCH, ZS>::warp;
    case K_RT_FULL: return SmemPlan<K_RT_FULL, NCH, ZS>::warp;
    case K_RT_PIX: return SmemPlan<K_RT_PIX, NCH, ZS>::warp;
    case K_RT_SSE: return SmemPlan<K_RT_SSE, NCH, ZS>::warp;
    default: return SmemPlan<K_RT_COEF, NCH, ZS>::warp;
  }
}
static_assert(ADCT_DEEP_ZONE <= 4, "warp_smem tells zones 0..4 apart only");
// Shared memory per warp of the kernel for this kind, channel count and zone.
int warp_smem(int kind, int nch, int zs) {
  if (nch == 3) return warp_smem_z<3, 14>(kind);
  if (nch == 4) return warp_smem_z<4, 14>(kind);
  switch (zs) {
    case 0: return warp_smem_z<1, 0>(kind);
    case 1: return warp_smem_z<1, 1>(kind);
    case 2: return warp_smem_z<1, 2>(kind);
    case 3: return warp_smem_z<1, 3>(kind);
    case 4: return warp_smem_z<1, 4>(kind);
    default: return warp_smem_z<1, 14>(kind);
  }
}
}  // namespace

// CTAs per SM when the caller leaves the choice to the library (measured on
// 256 x 1080x1920 batches): four, except three for the encode with dense
// coefficient output, whose 192 bytes of traffic per block run best with
// fewer requests in flight.  Capped at the resident count, which is three for
// the kernels that use more than 128 registers.
int default_ctas_per_sm(int kind, int qmode) { return (kind == K_RT_COEF && qmode != QM_ZONAL_ZZ) ? 3 : 4; }

size_t codec_smem_bytes(const LaunchShape& shape, int kind, int nch, int zs) {
  return (size_t)(shape.threads / 32) * warp_smem(kind, nch, zs);
}

int codec_grid(const LaunchShape& shape, int sm_count, int64_t total) {
  int64_t want = (total + shape.threads - 1) / shape.threads;
  const int64_t cap = (int64_t)sm_count * (shape.ctas_per_sm > 0 ? shape.ctas_per_sm : 4);
  if (want > cap) want = cap;
  return (int)(want < 1 ? 1 : want);
}

namespace {
// One launch of the persistent kernel, resolved: the instantiation, its
// resident grid and shared memory, and the coefficient staging.
struct Prepared {
  KernelFn fn = nullptr;
  int grid = 0;     // CTAs (never more than can be resident at once)
  int cap = 0;      // CTAs that can be resident at once
  int threads = 0;
  size_t smem = 0;
  int stage = 1;
};

cudaError_t prepare_codec(const CodecLaunch& c, const LaunchShape& shape, int sm_count, Prepared& p) {
  KernelFn fn = nullptr;
  int zs = 14;  // zone of the kernel picked (its shared-memory plan)
  if (c.nch == 3 || c.nch == 4) {
    fn = c.edge == kEdgeBlocks   ? pick_interleaved_edge_kernel(c.kind, c.qmode, c.evenq, c.nch)
         : c.edge == kEdgeMasked ? pick_interleaved_masked_kernel(c.kind, c.qmode, c.evenq, c.nch)
                                 : pick_interleaved_kernel(c.kind, c.qmode, c.evenq, c.nch);
    if (!fn) return cudaErrorInvalidValue;
  } else if (c.edge == kEdgeBlocks) {
    fn = pick_edge_kernel(c.kind, c.qmode, c.evenq);
    if (!fn) return cudaErrorInvalidValue;
  } else if (c.edge == kEdgeMasked) {
    fn = pick_masked_kernel(c.kind, c.qmode, c.evenq);
    if (!fn) return cudaErrorInvalidValue;
  } else if (c.qmode == QM_ZONAL_ZZ && c.qp.r == 64) {
    fn = pick_zz64(c.kind);
  } else if (c.qmode == QM_ZONAL || c.qmode == QM_ZONAL_ZZ) {
    // The packed round trip takes at least the zone-3 kernel: the lighter
    // zone 0-2 kernels ran slower on full-size batches although they execute
    // fewer instructions (r = 1: 231 us against 196 us with the zone-3 kernel,
    // 256 x 1080x1920), their warps waiting on memory twice as often per issue.
    int z = zone_for(c.qp.r);
    if (c.qmode == QM_ZONAL_ZZ && c.kind == K_RT_FULL && z < 3) z = 3;
    if (z <= kZoneLoMax) fn = pick_zonal_kernel_lo(c.kind, c.qmode, z);
    else if (z <= kZoneHiMax) fn = pick_zonal_kernel_hi(c.kind, c.qmode, z);
    if (fn) zs = z;  // a kernel specialised on zone z
  }
  if (!fn) fn = pick_kernel(c.kind, c.qmode, c.evenq);
  if (!fn) return cudaErrorInvalidValue;
  if (shape.threads < 32 || shape.threads > kMaxThreads || shape.threads % 32) return cudaErrorInvalidValue;
  LaunchShape sh = shape;
  // Interleaved images with the CTA count left to the library: one warp per
  // CTA, 12 per SM (measured on 64 RGB 1080x1920 images: 359 us against 385 us
  // with 3 CTAs of 4 warps; planar images gain nothing from it).
  if (sh.ctas_per_sm == 0 && c.nch > 1) {
    sh.threads = 32;
    sh.ctas_per_sm = 12;
  }
  const size_t smem = codec_smem_bytes(sh, c.kind, c.nch, zs);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  // never size the persistent grid beyond what can be resident at once
  int resident = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, fn, sh.threads, smem) != cudaSuccess || resident < 1)
    resident = 1;
  if (sh.ctas_per_sm == 0) sh.ctas_per_sm = default_ctas_per_sm(c.kind, c.qmode);
  if (sh.ctas_per_sm > resident) sh.ctas_per_sm = resident;
  p.fn = fn;
  p.grid = codec_grid(sh, sm_count, c.total);
  p.cap = sh.ctas_per_sm * sm_count;
  p.threads = sh.threads;
  p.smem = smem;
  // staging of the coefficients: the caller's choice, else staged except for
  // the packed round trip with r <= 8, whose direct stores measured faster
  // (r = 1: 185 us against 196 us staged; r = 10: 225 us against 211 us)
  p.stage = shape.stage_coef >= 0 ? shape.stage_coef
                                  : (c.qmode == QM_ZONAL_ZZ && c.kind == K_RT_FULL && c.qp.r <= 8) ? 0 : 1;
  return cudaSuccess;
}

// Launches a prepared kernel on `grid` CTAs: each warp takes a contiguous
// chunk of the flat block index, a whole number of 32-block tiles.
cudaError_t fire(const CodecLaunch& c, const Prepared& p, int grid, cudaStream_t stream) {
  const int64_t warps = (int64_t)grid * (p.threads / 32);
  int64_t chunk = (c.total + warps - 1) / warps;
  chunk = (chunk + kTile - 1) / kTile * kTile;
  if (c.edge == kEdgeBlocks && c.after_interior) {
    // programmatic dependent of the masked-interior launch just before it
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(p.threads);
    cfg.dynamicSmemBytes = p.smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, p.fn, c.planes, c.starts, c.nplanes, c.total, chunk, p.stage, c.sse, c.fault,
                              c.qp);
  }
  p.fn<<<grid, p.threads, p.smem, stream>>>(c.planes, c.starts, c.nplanes, c.total, chunk, p.stage, c.sse, c.fault,
                                            c.qp);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_codec(const CodecLaunch& c, const LaunchShape& shape, int sm_count, cudaStream_t stream) {
  if (c.total <= 0) return cudaSuccess;
  Prepared p;
  const cudaError_t e = prepare_codec(c, shape, sm_count, p);
  return e != cudaSuccess ? e : fire(c, p, p.grid, stream);
}

}  // namespace adct
