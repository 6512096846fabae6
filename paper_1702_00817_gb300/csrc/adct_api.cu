// C ABI of the codec (include/adct.h): argument validation, per-call
// descriptor tables (one launch per pixel layout class), the workspace ring,
// the CUDA-graph cache, the autotuner, the host-buffer pipeline, the
// allocation-free entry point and the multi-GPU sharding plan.  Kernels live
// in adct_codec*.cu, adct_float.cu and adct_quality.cu; this file only
// prepares their parameters and launches them.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "adct.h"
#include "adct_internal.h"

using namespace adct;

namespace {

constexpr int kSlots = 4;       // descriptor workspace ring
constexpr int kPipeSlots = 3;   // host pipeline stages in flight

struct Slot {
  void* dev = nullptr;
  void* host = nullptr;   // pinned staging; after an upload it mirrors the device copy
  size_t cap = 0;
  size_t bytes = 0;       // size of the table the device copy holds (0: none)
  cudaEvent_t done = nullptr;      // last kernel that read the slot
  cudaEvent_t uploaded = nullptr;  // the upload of the current table
  cudaStream_t stream = nullptr;   // stream of the last kernel that read the slot
  bool pending = false;
};

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  void* dev = nullptr;            // the descriptor table the captured launches read
  void* host = nullptr;           // pinned staging of that table
  size_t bytes = 0;
  std::vector<uint8_t> uploaded;  // the table now in dev (empty before the first upload)
  cudaEvent_t done = nullptr;
  bool pending = false;
};

struct PipeSlot {
  cudaStream_t stream = nullptr;
  uint8_t* src = nullptr;
  uint8_t* dst = nullptr;
  int16_t* coef = nullptr;
  size_t pix_cap = 0, coef_cap = 0;
};

}  // namespace

struct adct_context {
  int device = 0;
  int sm_count = 0;
  LaunchShape shape{128, 0, -1};  // ctas_per_sm 0, stage_coef -1: chosen per kernel kind
  std::string last_error;
  Slot slots[kSlots];
  int next_slot = 0;
  cudaStream_t capture_stream = nullptr;
  std::unordered_map<std::string, GraphEntry> graphs;
  PipeSlot pipe[kPipeSlots];
  // kernel timing (benchmarks): event pairs around each launch while enabled
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> tev;
  size_t tev_used = 0;
  int64_t launches = 0;
  unsigned int* fault = nullptr;  // device word for the bounds checks of a checked build
};

namespace adct {
cudaError_t device_alloc(void** ptr, size_t bytes) {
  static const long long fail_at = [] {
    const char* e = std::getenv("ADCT_FAULT_INJECT");
    return (e && std::strncmp(e, "alloc:", 6) == 0) ? std::atoll(e + 6) : 0ll;
  }();
  static std::atomic<long long> calls{0};
  if (fail_at > 0 && ++calls == fail_at) return cudaErrorMemoryAllocation;
  return cudaMalloc(ptr, bytes);
}
}  // namespace adct

namespace {

// NVTX range around one entry point, visible to Nsight tools (free when no
// tool is attached).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
      changed = (cudaSetDevice(dev) == cudaSuccess);
    }
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

adct_status fail(adct_context* ctx, adct_status st, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return st;
}

adct_status cuda_fail(adct_context* ctx, cudaError_t e, const char* where) {
  return fail(ctx, ADCT_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define ADCT_CUDA(ctx, call)                                  \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);  \
  } while (0)

// Brackets one launch with timing events when the context's timing is on.
struct TimedLaunch {
  adct_context* ctx;
  cudaStream_t stream;
  cudaEvent_t stop = nullptr;
  // timed = false (under stream capture): neither counted nor timed
  TimedLaunch(adct_context* c, cudaStream_t s, bool timed = true) : ctx(c), stream(s) {
    if (!timed) return;
    ++ctx->launches;
    if (!ctx->timing) return;
    if (ctx->tev_used == ctx->tev.size()) {
      cudaEvent_t a = nullptr, b = nullptr;
      if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        cudaGetLastError();
        return;
      }
      ctx->tev.emplace_back(a, b);
    }
    auto& pr = ctx->tev[ctx->tev_used++];
    cudaEventRecord(pr.first, stream);
    stop = pr.second;
  }
  void done() {
    if (stop) cudaEventRecord(stop, stream);
    stop = nullptr;
  }
};

// Zig-zag rank of each position (Sec. 3 "standard zigzag sequence"):
// positions ordered by anti-diagonal s = i + j; within a diagonal, even s runs
// from the bottom-left up (i descending), odd s from the top-right down.
void zigzag_rank(int rank[64]) {
  int order[64];
  for (int k = 0; k < 64; ++k) order[k] = k;
  std::sort(order, order + 64, [](int a, int b) {
    const int ia = a / 8, ja = a % 8, ib = b / 8, jb = b % 8;
    const int sa = ia + ja, sb = ib + jb;
    if (sa != sb) return sa < sb;
    return (sa % 2 == 0) ? (ia > ib) : (ia < ib);
  });
  for (int k = 0; k < 64; ++k) rank[order[k]] = k;
}

bool uses_step(int mode) { return mode == ADCT_Q_STEP || mode == ADCT_Q_STEP_ZONAL; }
bool uses_zonal(int mode) { return mode == ADCT_Q_ZONAL || mode == ADCT_Q_STEP_ZONAL || mode == ADCT_Q_ZONAL_ZZ; }

// int16 coefficients stored per 8x8 block: r for the packed zonal layout, else 64.
int32_t coef_per_block(const adct_quant* q) {
  return (q && q->mode == ADCT_Q_ZONAL_ZZ && q->r >= 0 && q->r <= 64) ? q->r : 64;
}

// Per-position quantiser constants (see QuantParams).  pixel_input: Z is
// computed from raw pixels, so Z_00 carries +8192 that the constants remove.
adct_status build_quant(adct_context* ctx, const adct_quant* q, bool pixel_input, QuantParams& qp, bool& evenq) {
  adct_quant none{};
  none.mode = ADCT_Q_NONE;
  if (!q) q = &none;
  if (q->mode < ADCT_Q_NONE || q->mode > ADCT_Q_ZONAL_ZZ) return fail(ctx, ADCT_ERR_INVALID_ARG, "bad quant mode");
  if (uses_zonal(q->mode) && (q->r < 0 || q->r > 64)) return fail(ctx, ADCT_ERR_INVALID_ARG, "r outside 0..64");
  int rank[64];
  zigzag_rank(rank);
  evenq = false;
  qp.r = uses_zonal(q->mode) ? q->r : 64;
  for (int k = 0; k < 64; ++k) {
    const int i = k / 8, j = k % 8;
    // weights carry a factor 4 (2 extra shift bits): the kernels' pixel is the
    // high byte of the saturated 16-bit 4 (R + 8224)
    const int shift = 8 - scale_exp(i) - scale_exp(j);
    const int32_t zoff = (pixel_input && k == 0) ? -8192 : 0;
    qp.keep[k] = (!uses_zonal(q->mode) || rank[k] < q->r) ? -1 : 0;
    qp.c[k] = 0;
    qp.magic[k] = 0;
    qp.K[k] = 0;
    qp.ssel[k] = 0x4444u;
    const int32_t bias = (k == 0) ? 4 * 8224 : 0;  // 4 (32 + 128 * 64)
    if (!uses_step(q->mode)) {
      qp.w[k] = 1 << shift;
      qp.kw[k] = bias;
      continue;
    }
    const uint32_t Q = q->Q[k];
    if (Q < 1) return fail(ctx, ADCT_ERR_INVALID_ARG, "Q entry below 1");
    qp.w[k] = (int32_t)(Q << shift);
    qp.kw[k] = bias;
    if (Q > 16384) continue;  // |Z| <= 8192 < Q / 2: every coefficient rounds to 0
    const int32_t K = (int32_t)((8193 + Q - 1) / Q);
    qp.K[k] = K;
    qp.c[k] = zoff + (int32_t)(Q / 2) + K * (int32_t)Q + (Q == 1 ? 1 : 0);
    qp.magic[k] = (Q == 1) ? 0xFFFFFFFFu : (uint32_t)(((1ull << 32) + Q - 1) / Q);
    qp.ssel[k] = (Q % 2 == 0) ? 0xBBBBu : 0x4444u;
    if (Q % 2 == 0) evenq = true;
    qp.kw[k] = (int32_t)((uint32_t)bias - (uint32_t)K * (uint32_t)qp.w[k]);
  }
  return ADCT_OK;
}

enum Need { NEED_SRC = 1, NEED_DST = 2, NEED_COEF = 4 };

// Checks one image; on error returns the status and sets *why.  coef_only:
// the call reads and writes coefficients only, so the pixel layout is
// irrelevant.
adct_status check_image(const adct_image& im, int need, bool coef_only, const char** why) {
  if (im.width <= 0 || im.height <= 0 || im.width > 65536 || im.height > 65536)
    return *why = "width/height must be in 1..65536", ADCT_ERR_SHAPE;
  if (im.layout != ADCT_LAYOUT_PLANAR && im.layout != ADCT_LAYOUT_INTERLEAVED)
    return *why = "unknown layout", ADCT_ERR_INVALID_ARG;
  if (im.channels < 1) return *why = "channels must be at least 1", ADCT_ERR_INVALID_ARG;
  const bool inter = im.layout == ADCT_LAYOUT_INTERLEAVED && !coef_only;
  if (inter && im.channels != 3 && im.channels != 4)
    return *why = "interleaved images have 3 or 4 channels", ADCT_ERR_UNSUPPORTED;
  if ((need & NEED_SRC) && !im.src) return *why = "src is NULL", ADCT_ERR_INVALID_ARG;
  if ((need & NEED_DST) && !im.dst) return *why = "dst is NULL", ADCT_ERR_INVALID_ARG;
  if ((need & NEED_COEF) && !im.coef) return *why = "coef is NULL", ADCT_ERR_INVALID_ARG;
  if ((uintptr_t)im.coef % 16) return *why = "coef needs 16-byte alignment", ADCT_ERR_ALIGN;
  if (need & (NEED_SRC | NEED_DST)) {
    if (im.pitch < (int64_t)im.width * (inter ? im.channels : 1)) return *why = "pitch too small", ADCT_ERR_SHAPE;
    if (!inter && im.channels > 1 && im.plane_stride < im.pitch * im.height)
      return *why = "plane_stride < pitch * height", ADCT_ERR_SHAPE;
    if ((uintptr_t)im.src % 8 || (uintptr_t)im.dst % 8 || im.pitch % 8 ||
        (!inter && im.channels > 1 && im.plane_stride % 8))
      return *why = "src/dst/pitch/plane_stride need 8-byte alignment", ADCT_ERR_ALIGN;
  }
  return ADCT_OK;
}

// Launch groups of a call without split images: planar, 3-channel and
// 4-channel interleaved, each without and with edge blocks (group_of).
constexpr int kGroups = 6;

// Appends image im's descriptors (one per planar plane, or one for an
// interleaved image) to out[*count..]; cpb is the number of int16
// coefficients stored per block (64, or r when packed); plane_id numbers
// channel 0 of the image among all planes of the call.  Returns the group
// (group_of): 0 planar, 2 interleaved 3 channels, 4 interleaved 4 channels,
// each plus 1 when the image has edge blocks.
int group_of(const adct_image& im, bool coef_only) {
  if (coef_only) return 0;
  const int edge = (im.width % 8 || im.height % 8) ? 1 : 0;
  if (im.layout == ADCT_LAYOUT_INTERLEAVED) return (im.channels == 3 ? 2 : 4) + edge;
  return edge;
}

int describe_image(const adct_image& im, int32_t cpb, bool coef_only, int32_t plane_id, PlaneDesc* out,
                   int32_t* count) {
  const int32_t wb = (im.width + 7) / 8, hb = (im.height + 7) / 8;
  const int64_t nb = (int64_t)wb * hb;
  const bool inter = group_of(im, coef_only) >= 2;  // interleaved
  PlaneDesc d{};
  d.pitch = im.pitch;
  d.cstride = nb * cpb;
  d.wb = wb;
  d.hb = hb;
  d.cwb = wb;
  d.ew = (int16_t)(im.width - 8 * (wb - 1));
  d.eh = (int16_t)(im.height - 8 * (hb - 1));
  d.bx0 = 0;
  if (inter) {
    d.src = im.src;
    d.dst = im.dst;
    d.coef = im.coef;
    d.plane_id = plane_id;
    d.nch = (int16_t)im.channels;
    out[(*count)++] = d;
    return group_of(im, coef_only);
  }
  for (int32_t c = 0; c < im.channels; ++c) {
    d.src = im.src ? im.src + (int64_t)c * im.plane_stride : nullptr;
    d.dst = im.dst ? im.dst + (int64_t)c * im.plane_stride : nullptr;
    d.coef = im.coef ? im.coef + (int64_t)c * nb * cpb : nullptr;
    d.plane_id = plane_id + c;
    d.nch = 1;
    out[(*count)++] = d;
  }
  return group_of(im, coef_only);
}

// Descriptors of one planar plane or one interleaved image (`one`: channels
// 1, or an interleaved image), split when it has edge blocks and at least
// kSplitMin interior blocks: the interior (every block with 8 x 8 valid
// pixels; its flat rows include the masked last column) goes to the group
// without edge handling, the last block column and the rest of the last block
// row to the edge group; otherwise one descriptor.
// Returns the count (1..3); part k belongs to group groups[k].
constexpr int64_t kSplitMin = 64;
int describe_parts(const adct_image& one, int32_t cpb, bool coef_only, int32_t plane_id, PlaneDesc parts[3],
                   int groups[3]) {
  int32_t cnt = 0;
  const int g = describe_image(one, cpb, coef_only, plane_id, parts, &cnt);
  groups[0] = g;
  const PlaneDesc whole = parts[0];
  const bool right = whole.ew < 8, bottom = whole.eh < 8;
  const int32_t wi = whole.wb - (right ? 1 : 0), hi = whole.hb - (bottom ? 1 : 0);
  if ((g & 1) == 0 || (int64_t)wi * hi < kSplitMin) return 1;
  const int64_t bpx = 8 * (int64_t)whole.nch;  // pixel bytes of a block row segment
  const int64_t cpb64 = cpb;
  int n = 0;
  // The interior.  With a right edge column its flat rows still span the
  // whole coefficient row, so that the 32-block tiles stay aligned with the
  // image's rows; the last column is masked (ew = 0: the kernels without edge
  // handling skip it) and goes to the edge launch.
  PlaneDesc d = whole;
  d.wb = whole.wb;
  d.hb = hi;
  d.ew = right ? 0 : 8;
  d.eh = 8;
  parts[n] = d;
  groups[n++] = right ? kGroups + (g >> 1) : (g & ~1);  // masked interior, or the group without edges
  if (right) {  // the last block column, every block row
    d = whole;
    d.src = whole.src ? whole.src + bpx * (whole.wb - 1) : nullptr;
    d.dst = whole.dst ? whole.dst + bpx * (whole.wb - 1) : nullptr;
    d.coef = whole.coef ? whole.coef + cpb64 * (whole.wb - 1) : nullptr;
    d.wb = 1;
    d.bx0 = (int16_t)(whole.wb - 1);
    parts[n] = d;
    groups[n++] = g;
  }
  if (bottom) {  // the last block row without its last block when that is in the column
    d = whole;
    d.src = whole.src ? whole.src + 8 * whole.pitch * (whole.hb - 1) : nullptr;
    d.dst = whole.dst ? whole.dst + 8 * whole.pitch * (whole.hb - 1) : nullptr;
    d.coef = whole.coef ? whole.coef + cpb64 * whole.cwb * (whole.hb - 1) : nullptr;
    d.wb = wi;
    d.hb = 1;
    d.ew = 8;
    parts[n] = d;
    groups[n++] = g;
  }
  return n;
}

// Work units of one call: one group (one launch) per pixel layout class;
// images with edge blocks get their own launch so that the others run kernels
// with the edge handling compiled out.  After the kGroups groups come three
// more for the interiors of split images with a right edge column (planar, 3
// and 4 channels), whose last block column is masked (kernel edge class
// kEdgeMasked).
constexpr int kGroupsAll = kGroups + 3;
constexpr int kGroupNch[kGroupsAll] = {1, 1, 3, 3, 4, 4, 1, 3, 4};
constexpr bool kGroupEdge[kGroupsAll] = {false, true, false, true, false, true, false, false, false};
constexpr int kGroupClass[kGroupsAll] = {kEdgeNone, kEdgeBlocks, kEdgeNone,   kEdgeBlocks, kEdgeNone,
                                         kEdgeBlocks, kEdgeMasked, kEdgeMasked, kEdgeMasked};

int64_t blocks_of(const adct_image& im) { return (int64_t)((im.width + 7) / 8) * ((im.height + 7) / 8); }

struct Tables {
  std::vector<PlaneDesc> planes[kGroupsAll];
  std::vector<int64_t> starts[kGroupsAll];  // flat-index prefix per group (nplanes + 1)
  int32_t nplanes = 0;                   // planes of the call (per-plane outputs)
  int64_t blocks = 0;                    // 8x8 blocks of the call, all channels
  std::vector<uint8_t> blob;             // the groups' tables back to back, as uploaded
  size_t off_planes[kGroupsAll], off_starts[kGroupsAll];

  int64_t total(int g) const { return starts[g].empty() ? 0 : starts[g].back(); }
  void serialise() {
    size_t off = 0;
    for (int g = 0; g < kGroupsAll; ++g) {
      off_planes[g] = off;
      off += planes[g].size() * sizeof(PlaneDesc);
      off_starts[g] = off;
      off += starts[g].size() * sizeof(int64_t);
    }
    blob.resize(off);
    for (int g = 0; g < kGroupsAll; ++g) {
      if (!planes[g].empty()) std::memcpy(blob.data() + off_planes[g], planes[g].data(), planes[g].size() * sizeof(PlaneDesc));
      if (!starts[g].empty()) std::memcpy(blob.data() + off_starts[g], starts[g].data(), starts[g].size() * sizeof(int64_t));
    }
  }
};

// Per-thread table storage, reused call after call so that a steady stream of
// calls (the serving loop) allocates no host memory for its descriptors.
Tables& scratch_tables() {
  static thread_local Tables t;
  return t;
}

// Validates the images and builds the descriptor tables of every group.
adct_status build_tables(adct_context* ctx, const adct_image* imgs, int32_t n, int need, bool coef_only, int32_t cpb,
                         Tables& t) {
  if (n < 0) return fail(ctx, ADCT_ERR_INVALID_ARG, "negative image count");
  if (n > 0 && !imgs) return fail(ctx, ADCT_ERR_INVALID_ARG, "imgs is NULL");
  for (int g = 0; g < kGroupsAll; ++g) {
    t.planes[g].clear();
    t.starts[g].assign(1, 0);
  }
  t.nplanes = 0;
  t.blocks = 0;
  PlaneDesc pieces[3];
  int piece_group[3];
  for (int32_t m = 0; m < n; ++m) {
    const adct_image& im = imgs[m];
    const char* why = "";
    const adct_status st = check_image(im, need, coef_only, &why);
    if (st != ADCT_OK) return fail(ctx, st, std::string(why) + " (image " + std::to_string(m) + ")");
    const int64_t nb = blocks_of(im);
    const bool inter = im.layout == ADCT_LAYOUT_INTERLEAVED && !coef_only;
    const int32_t parts = inter ? 1 : im.channels;
    for (int32_t c = 0; c < parts; ++c) {
      adct_image one = im;
      if (!inter) {  // one planar plane at a time
        one.channels = 1;
        one.src = im.src ? im.src + (int64_t)c * im.plane_stride : nullptr;
        one.dst = im.dst ? im.dst + (int64_t)c * im.plane_stride : nullptr;
        one.coef = im.coef ? im.coef + (int64_t)c * nb * cpb : nullptr;
      }
      const int np = describe_parts(one, cpb, coef_only, t.nplanes + c, pieces, piece_group);
      for (int k = 0; k < np; ++k) {
        const int g = piece_group[k];
        t.planes[g].push_back(pieces[k]);
        t.starts[g].push_back(t.starts[g].back() + (int64_t)pieces[k].wb * pieces[k].hb);
      }
    }
    t.nplanes += im.channels;
    t.blocks += nb * im.channels;
  }
  t.serialise();
  return ADCT_OK;
}

// Finds a slot whose device copy already holds exactly this table (a batch
// repeated call after call) and was last read on the same stream: it is reused
// as is, with no upload.  Only same-stream reuse is allowed, so that the slot's
// `done` event, recorded after the new kernel, still covers every earlier
// reader before the slot is ever overwritten.
Slot* find_cached_slot(adct_context* ctx, const std::vector<uint8_t>& blob, cudaStream_t stream) {
  for (Slot& s : ctx->slots) {
    if (s.bytes != blob.size() || !s.host || s.stream != stream) continue;
    if (std::memcmp(s.host, blob.data(), blob.size()) == 0) return &s;
  }
  return nullptr;
}

// Takes the next workspace slot, waiting for the work that last used it.
adct_status acquire_slot(adct_context* ctx, size_t bytes, Slot** out) {
  Slot& s = ctx->slots[ctx->next_slot];
  ctx->next_slot = (ctx->next_slot + 1) % kSlots;
  if (s.pending) {
    ADCT_CUDA(ctx, cudaEventSynchronize(s.done));
    s.pending = false;
  }
  s.bytes = 0;
  if (s.cap < bytes) {
    size_t cap = std::max<size_t>(bytes, 4096);
    cap = (cap + 4095) / 4096 * 4096;
    if (s.dev) cudaFree(s.dev);
    if (s.host) cudaFreeHost(s.host);
    s.dev = s.host = nullptr;
    s.cap = 0;
    if (device_alloc(&s.dev, cap) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, ADCT_ERR_OOM, "workspace cudaMalloc failed");
    }
    if (cudaMallocHost(&s.host, cap) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(s.dev);
      s.dev = nullptr;
      return fail(ctx, ADCT_ERR_OOM, "workspace cudaMallocHost failed");
    }
    s.cap = cap;
  }
  *out = &s;
  return ADCT_OK;
}

adct_status check_shape(adct_context* ctx, const LaunchShape& sh) {
  if (sh.threads < 32 || sh.threads > 128 || sh.threads % 32 || sh.ctas_per_sm < 0 || sh.ctas_per_sm > 32 ||
      sh.stage_coef < -1 || sh.stage_coef > 1)
    return fail(ctx, ADCT_ERR_INVALID_ARG, "launch shape out of range");
  return ADCT_OK;
}

int kind_for_roundtrip(const adct_image* imgs, int32_t n, bool& ok) {
  bool any_coef = n > 0 && imgs[0].coef, any_dst = n > 0 && imgs[0].dst;
  ok = true;
  for (int32_t m = 0; m < n; ++m)
    if ((imgs[m].coef != nullptr) != any_coef || (imgs[m].dst != nullptr) != any_dst) ok = false;
  if (any_coef && any_dst) return K_RT_FULL;
  if (any_dst) return K_RT_PIX;
  return K_RT_COEF;
}

int need_for_kind(int kind) {
  switch (kind) {
    case K_FORWARD: return NEED_SRC | NEED_COEF;
    case K_QUANTISE: return NEED_COEF;
    case K_INVERSE: return NEED_COEF | NEED_DST;
    case K_RT_FULL: return NEED_SRC | NEED_COEF | NEED_DST;
    case K_RT_PIX: return NEED_SRC | NEED_DST;
    case K_RT_SSE: return NEED_SRC;
    default: return NEED_SRC | NEED_COEF;
  }
}

// Launch order of the groups: per layout class the group without edge
// blocks, the masked interiors of its split images, then its edge group,
// which runs as the programmatic dependent of the masked interiors when
// there are any (its CTAs start in their tail instead of after them).
constexpr int kLaunchOrder[kGroupsAll] = {0, 6, 1, 2, 7, 3, 4, 8, 5};

// One launch per non-empty group of t, whose tables are at dev (t.blob's
// layout), in kLaunchOrder on `stream`.  Under stream capture (timed = false)
// no timing events are recorded; a masked-interior launch and the edge
// launch that depends on it are timed as one.
adct_status launch_groups(adct_context* ctx, CodecLaunch cl, const Tables& t, const char* dev, const LaunchShape& shape,
                          cudaStream_t stream, bool timed = true) {
  auto group = [&](int g) {
    CodecLaunch c = cl;
    c.planes = (const PlaneDesc*)(dev + t.off_planes[g]);
    c.starts = (const int64_t*)(dev + t.off_starts[g]);
    c.nplanes = (int32_t)t.planes[g].size();
    c.total = t.total(g);
    c.nch = kGroupNch[g];
    c.edge = kGroupClass[g];
    c.after_interior = false;
    return c;
  };
  for (int k = 0; k < kGroupsAll; ++k) {
    const int g = kLaunchOrder[k];
    if (t.total(g) == 0) continue;
    const int ge = (kGroupClass[g] == kEdgeMasked && k + 1 < kGroupsAll) ? kLaunchOrder[k + 1] : -1;
    const bool pair = ge >= 0 && t.total(ge) > 0;
    cudaError_t e;
    {
      TimedLaunch tl(ctx, stream, timed);
      e = launch_codec(group(g), shape, ctx->sm_count, stream);
      if (e == cudaSuccess && pair) {
        if (timed) ++ctx->launches;  // two kernels
        CodecLaunch c = group(ge);
        c.after_interior = true;
        e = launch_codec(c, shape, ctx->sm_count, stream);
      }
      tl.done();
    }
    if (pair) ++k;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "codec kernel launch");
  }
  return ADCT_OK;
}

// Validates, uploads the descriptor tables through a workspace slot and launches.
adct_status run_codec(adct_context* ctx, const adct_image* imgs, int32_t n, const adct_quant* quant, int kind,
                      cudaStream_t stream, const LaunchShape& shape, unsigned long long* sse = nullptr) {
  if (!ctx) return ADCT_ERR_INVALID_ARG;
  ctx->last_error.clear();
  adct_status st = check_shape(ctx, shape);
  if (st != ADCT_OK) return st;
  CodecLaunch cl{};
  cl.kind = kind;
  cl.qmode = QM_NONE;
  cl.fault = ctx->fault;
  if (kind != K_FORWARD && !quant) return fail(ctx, ADCT_ERR_INVALID_ARG, "quant is NULL");
  const bool pixel_input = (kind != K_QUANTISE && kind != K_INVERSE);
  st = build_quant(ctx, kind == K_FORWARD ? nullptr : quant, pixel_input, cl.qp, cl.evenq);
  if (st != ADCT_OK) return st;
  if (kind != K_FORWARD && kind != K_INVERSE) cl.qmode = quant->mode;
  const bool packed = kind != K_FORWARD && quant->mode == ADCT_Q_ZONAL_ZZ;
  if (packed && kind == K_QUANTISE)
    return fail(ctx, ADCT_ERR_UNSUPPORTED, "the packed zonal layout is written by adct_roundtrip, not adct_quantise");
  if (packed && kind == K_INVERSE) cl.qmode = QM_ZONAL_ZZ;
  Tables& t = scratch_tables();
  st = build_tables(ctx, imgs, n, need_for_kind(kind), kind == K_QUANTISE, packed ? quant->r : 64, t);
  if (st != ADCT_OK) return st;
  if (t.blocks == 0) return ADCT_OK;
  if (kind == K_QUANTISE && quant->mode == ADCT_Q_NONE) return ADCT_OK;  // identity
  DeviceGuard guard(ctx->device);
  const size_t bytes = t.blob.size();
  Slot* slot = find_cached_slot(ctx, t.blob, stream);
  if (!slot) {
    st = acquire_slot(ctx, bytes, &slot);
    if (st != ADCT_OK) return st;
    std::memcpy(slot->host, t.blob.data(), bytes);
    ADCT_CUDA(ctx, cudaMemcpyAsync(slot->dev, slot->host, bytes, cudaMemcpyHostToDevice, stream));
    ADCT_CUDA(ctx, cudaEventRecord(slot->uploaded, stream));
    slot->bytes = bytes;
  }
  if (kind == K_RT_SSE) {
    cl.sse = sse;
    ADCT_CUDA(ctx, cudaMemsetAsync(sse, 0, (size_t)t.nplanes * sizeof(unsigned long long), stream));
  }
  st = launch_groups(ctx, cl, t, (const char*)slot->dev, shape, stream);
  if (st != ADCT_OK) return st;
  ADCT_CUDA(ctx, cudaEventRecord(slot->done, stream));
  slot->pending = true;
  slot->stream = stream;
  return ADCT_OK;
}

adct_status float_params(adct_context* ctx, const float* Qsoft, FloatParams& fp) {
  for (int k = 0; k < 64; ++k) {
    const float Q = Qsoft[k];
    if (!(Q > 0.0f) || !std::isfinite(Q)) return fail(ctx, ADCT_ERR_INVALID_ARG, "Qsoft entries must be positive");
    fp.c2pi[k] = (float)((double)Q / (2.0 * M_PI));
    fp.rq[k] = (float)(1.0 / (double)Q);
    // d_i d_j = 2^-((a_i + a_j) / 2), Sec. 2 matrix D
    fp.g[k] = (float)(std::pow(2.0, -0.5 * (scale_exp(k / 8) + scale_exp(k % 8))) / (double)Q);
  }
  return ADCT_OK;
}

adct_status check_float(adct_context* ctx, const void* a, const void* b, const void* c, int64_t planes, int32_t H,
                        int32_t W) {
  if (!ctx) return ADCT_ERR_INVALID_ARG;
  ctx->last_error.clear();
  if (planes < 0) return fail(ctx, ADCT_ERR_INVALID_ARG, "negative plane count");
  if (H <= 0 || W <= 0 || H % 8 || W % 8) return fail(ctx, ADCT_ERR_SHAPE, "H and W must be positive multiples of 8");
  if (planes > 0 && (!a || !b || !c)) return fail(ctx, ADCT_ERR_INVALID_ARG, "NULL tensor");
  if ((uintptr_t)a % 16 || (uintptr_t)b % 16 || (uintptr_t)c % 16)
    return fail(ctx, ADCT_ERR_ALIGN, "float tensors must be 16-byte aligned");
  return ADCT_OK;
}

std::string graph_key(const adct_image* imgs, int32_t n, const adct_quant* q, int kind, const LaunchShape& sh) {
  std::string k;
  k.reserve(64 + 16 * (size_t)n);
  auto put = [&k](const void* p, size_t sz) { k.append((const char*)p, sz); };
  put(&kind, sizeof kind);
  put(&sh, sizeof sh);
  put(q, sizeof *q);
  put(&n, sizeof n);
  for (int32_t m = 0; m < n; ++m) {
    const int32_t dims[4] = {imgs[m].width, imgs[m].height, imgs[m].channels, imgs[m].layout};
    put(dims, sizeof dims);
  }
  return k;
}

}  // namespace

extern "C" {

const char* adct_status_string(adct_status s) {
  switch (s) {
    case ADCT_OK: return "ADCT_OK";
    case ADCT_ERR_INVALID_ARG: return "ADCT_ERR_INVALID_ARG";
    case ADCT_ERR_SHAPE: return "ADCT_ERR_SHAPE";
    case ADCT_ERR_ALIGN: return "ADCT_ERR_ALIGN";
    case ADCT_ERR_OOM: return "ADCT_ERR_OOM";
    case ADCT_ERR_CUDA: return "ADCT_ERR_CUDA";
    case ADCT_ERR_TIMEOUT: return "ADCT_ERR_TIMEOUT";
    case ADCT_ERR_UNSUPPORTED: return "ADCT_ERR_UNSUPPORTED";
    case ADCT_ERR_TOO_LARGE: return "ADCT_ERR_TOO_LARGE";
    case ADCT_ERR_CANCELLED: return "ADCT_ERR_CANCELLED";
  }
  return "ADCT_ERR_UNKNOWN";
}

const char* adct_last_error(adct_context* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

adct_status adct_create(adct_context** out, int32_t device) {
  if (!out) return ADCT_ERR_INVALID_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return ADCT_ERR_INVALID_ARG;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return ADCT_ERR_CUDA;
  if (prop.major != 10 || prop.minor != 3) return ADCT_ERR_UNSUPPORTED;  // kernels are built for sm_103a only
  adct_context* ctx = new adct_context();
  ctx->device = device;
  ctx->sm_count = prop.multiProcessorCount;
  DeviceGuard guard(device);
  for (auto& s : ctx->slots) {
    if (cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.uploaded, cudaEventDisableTiming) != cudaSuccess) {
      adct_destroy(ctx);
      return ADCT_ERR_CUDA;
    }
  }
  if (cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
    adct_destroy(ctx);
    return ADCT_ERR_CUDA;
  }
  if (device_alloc((void**)&ctx->fault, sizeof(unsigned int)) != cudaSuccess ||
      cudaMemset(ctx->fault, 0, sizeof(unsigned int)) != cudaSuccess) {
    cudaGetLastError();
    adct_destroy(ctx);
    return ADCT_ERR_OOM;
  }
  *out = ctx;
  return ADCT_OK;
}

void adct_destroy(adct_context* ctx) {
  if (!ctx) return;
  DeviceGuard guard(ctx->device);
  if (ctx->fault) {
    cudaDeviceSynchronize();
    cudaFree(ctx->fault);
  }
  for (auto& s : ctx->slots) {
    if (s.done) {
      if (s.pending) cudaEventSynchronize(s.done);
      cudaEventDestroy(s.done);
    }
    if (s.uploaded) cudaEventDestroy(s.uploaded);
    if (s.dev) cudaFree(s.dev);
    if (s.host) cudaFreeHost(s.host);
  }
  for (auto& kv : ctx->graphs) {
    GraphEntry& g = kv.second;
    if (g.pending) cudaEventSynchronize(g.done);
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    if (g.done) cudaEventDestroy(g.done);
    if (g.dev) cudaFree(g.dev);
    if (g.host) cudaFreeHost(g.host);
  }
  for (auto& p : ctx->pipe) {
    if (p.stream) {
      cudaStreamSynchronize(p.stream);
      cudaStreamDestroy(p.stream);
    }
    if (p.src) cudaFree(p.src);
    if (p.dst) cudaFree(p.dst);
    if (p.coef) cudaFree(p.coef);
  }
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  for (auto& pr : ctx->tev) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  delete ctx;
}

adct_status adct_set_launch(adct_context* ctx, const adct_launch* l) {
  if (!ctx || !l) return ADCT_ERR_INVALID_ARG;
  LaunchShape sh = ctx->shape;
  if (l->reserved) return fail(ctx, ADCT_ERR_INVALID_ARG, "reserved must be 0");
  if (l->threads_per_cta) sh.threads = l->threads_per_cta;
  if (l->ctas_per_sm) sh.ctas_per_sm = l->ctas_per_sm < 0 ? 0 : l->ctas_per_sm;
  sh.stage_coef = l->stage_coef;
  adct_status st = check_shape(ctx, sh);
  if (st != ADCT_OK) return st;
  ctx->shape = sh;
  return ADCT_OK;
}

adct_status adct_get_launch(adct_context* ctx, adct_launch* l) {
  if (!ctx || !l) return ADCT_ERR_INVALID_ARG;
  l->threads_per_cta = ctx->shape.threads;
  l->ctas_per_sm = ctx->shape.ctas_per_sm;
  l->stage_coef = ctx->shape.stage_coef;
  l->reserved = 0;
  return ADCT_OK;
}

adct_status adct_kernel_timing(adct_context* ctx, int32_t enable) {
  if (!ctx) return ADCT_ERR_INVALID_ARG;
  ctx->timing = enable != 0;
  return ADCT_OK;
}

adct_status adct_checked_faults(adct_context* ctx, uint32_t* faults) {
  if (!ctx || !faults) return ADCT_ERR_INVALID_ARG;
  *faults = 0;
#ifdef ADCT_CHECKED
  DeviceGuard guard(ctx->device);
  ADCT_CUDA(ctx, cudaDeviceSynchronize());
  unsigned int w = 0;
  ADCT_CUDA(ctx, cudaMemcpy(&w, ctx->fault, sizeof w, cudaMemcpyDeviceToHost));
  ADCT_CUDA(ctx, cudaMemset(ctx->fault, 0, sizeof w));
  *faults = w;
  return ADCT_OK;
#else
  return fail(ctx, ADCT_ERR_UNSUPPORTED, "bounds checks exist in the checked build only (libadct_checked.so)");
#endif
}

adct_status adct_kernel_time(adct_context* ctx, double* total_ms, int64_t* launches) {
  if (!ctx) return ADCT_ERR_INVALID_ARG;
  DeviceGuard guard(ctx->device);
  double sum = 0.0;
  for (size_t k = 0; k < ctx->tev_used; ++k) {
    ADCT_CUDA(ctx, cudaEventSynchronize(ctx->tev[k].second));
    float ms = 0.f;
    ADCT_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->tev[k].first, ctx->tev[k].second));
    sum += ms;
  }
  if (total_ms) *total_ms = sum;
  if (launches) *launches = ctx->launches;
  ctx->tev_used = 0;
  ctx->launches = 0;
  return ADCT_OK;
}

adct_status adct_forward(adct_context* ctx, const adct_image* imgs, int32_t n, adct_stream_t stream) {
  Range nvtx("adct_forward");
  return run_codec(ctx, imgs, n, nullptr, K_FORWARD, (cudaStream_t)stream, ctx ? ctx->shape : LaunchShape{});
}

adct_status adct_quantise(adct_context* ctx, const adct_image* imgs, int32_t n, const adct_quant* quant,
                          adct_stream_t stream) {
  Range nvtx("adct_quantise");
  return run_codec(ctx, imgs, n, quant, K_QUANTISE, (cudaStream_t)stream, ctx ? ctx->shape : LaunchShape{});
}

adct_status adct_inverse(adct_context* ctx, const adct_image* imgs, int32_t n, const adct_quant* quant,
                         adct_stream_t stream) {
  Range nvtx("adct_inverse");
  return run_codec(ctx, imgs, n, quant, K_INVERSE, (cudaStream_t)stream, ctx ? ctx->shape : LaunchShape{});
}

adct_status adct_roundtrip(adct_context* ctx, const adct_image* imgs, int32_t n, const adct_quant* quant,
                           adct_stream_t stream) {
  Range nvtx("adct_roundtrip");
  if (!ctx) return ADCT_ERR_INVALID_ARG;
  if (n < 0 || (n > 0 && !imgs)) return fail(ctx, ADCT_ERR_INVALID_ARG, "bad image list");
  bool ok = true;
  const int kind = kind_for_roundtrip(imgs, n, ok);
  if (!ok) return fail(ctx, ADCT_ERR_INVALID_ARG, "coef/dst must be set on all images or on none");
  if (n > 0 && !imgs[0].coef && !imgs[0].dst) return fail(ctx, ADCT_ERR_INVALID_ARG, "need coef or dst");
  return run_codec(ctx, imgs, n, quant, kind, (cudaStream_t)stream, ctx->shape);
}

adct_status adct_quality(adct_context* ctx, const adct_image* imgs, int32_t n, const adct_quant* quant, uint64_t* sse,
                         adct_stream_t stream) {
  Range nvtx("adct_quality");
  if (!ctx) return ADCT_ERR_INVALID_ARG;
  if (n > 0 && !sse) return fail(ctx, ADCT_ERR_INVALID_ARG, "sse is NULL");
  if ((uintptr_t)sse % 8) return fail(ctx, ADCT_ERR_ALIGN, "sse must be 8-byte aligned");
  return run_codec(ctx, imgs, n, quant, K_RT_SSE, (cudaStream_t)stream, ctx->shape, (unsigned long long*)sse);
}

adct_status adct_quality_dct(adct_context* ctx, const adct_image* imgs, int32_t n, int32_t r, uint64_t* sse,
                             adct_stream_t stream) {
  Range nvtx("adct_quality_dct");
  if (!ctx) return ADCT_ERR_INVALID_ARG;
  ctx->last_error.clear();
  if (r < 0 || r > 64) return fail(ctx, ADCT_ERR_INVALID_ARG, "r outside 0..64");
  if (n > 0 && !sse) return fail(ctx, ADCT_ERR_INVALID_ARG, "sse is NULL");
  if ((uintptr_t)sse % 8) return fail(ctx, ADCT_ERR_ALIGN, "sse must be 8-byte aligned");
  for (int32_t m = 0; m < n && imgs; ++m)
    if (imgs[m].layout != ADCT_LAYOUT_PLANAR || imgs[m].width % 8 || imgs[m].height % 8)
      return fail(ctx, ADCT_ERR_UNSUPPORTED, "the DCT comparator takes planar images with sides multiple of 8");
  Tables& t = scratch_tables();
  adct_status st = build_tables(ctx, imgs, n, NEED_SRC, false, 64, t);
  if (st != ADCT_OK) return st;
  if (t.blocks == 0) return ADCT_OK;
  const std::vector<PlaneDesc>& planes = t.planes[0];
  const std::vector<int64_t>& starts = t.starts[0];
  // the orthonormal DCT-II matrix and the zig-zag zonal mask
  float c[64];
  for (int k = 0; k < 8; ++k)
    for (int j = 0; j < 8; ++j)
      c[8 * k + j] = (float)((k == 0 ? std::sqrt(0.125) : 0.5) * std::cos(M_PI * (2 * j + 1) * k / 16.0));
  int rank[64];
  zigzag_rank(rank);
  uint64_t mask = 0;
  for (int k = 0; k < 64; ++k)
    if (rank[k] < r) mask |= 1ull << k;
  DeviceGuard guard(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = t.blob.size();
  Slot* slot = find_cached_slot(ctx, t.blob, s);
  if (!slot) {
    st = acquire_slot(ctx, bytes, &slot);
    if (st != ADCT_OK) return st;
    std::memcpy(slot->host, t.blob.data(), bytes);
    ADCT_CUDA(ctx, cudaMemcpyAsync(slot->dev, slot->host, bytes, cudaMemcpyHostToDevice, s));
    ADCT_CUDA(ctx, cudaEventRecord(slot->uploaded, s));
    slot->bytes = bytes;
  }
  ADCT_CUDA(ctx, cudaMemsetAsync(sse, 0, planes.size() * sizeof(uint64_t), s));
  TimedLaunch tl(ctx, s);
  cudaError_t e = launch_dct_quality((const PlaneDesc*)((const char*)slot->dev + t.off_planes[0]),
                                     (const int64_t*)((const char*)slot->dev + t.off_starts[0]),
                                     (int32_t)planes.size(), starts.back(), c, mask, (unsigned long long*)sse,
                                     ctx->sm_count, s);
  tl.done();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "dct quality launch");
  ADCT_CUDA(ctx, cudaEventRecord(slot->done, s));
  slot->pending = true;
  slot->stream = s;
  return ADCT_OK;
}

adct_status adct_forward_f32(adct_context* ctx, const float* x, float* y, int64_t planes, int32_t H, int32_t W,
                             const float* Qsoft, adct_stream_t stream) {
  Range nvtx("adct_forward_f32");
  adct_status st = check_float(ctx, x, y, y, planes, H, W);
  if (st != ADCT_OK) return st;
  FloatParams fp;
  if (Qsoft && (st = float_params(ctx, Qsoft, fp)) != ADCT_OK) return st;
  DeviceGuard guard(ctx->device);
  TimedLaunch tl(ctx, (cudaStream_t)stream);
  cudaError_t e = launch_float_forward(x, y, planes, H, W, Qsoft ? &fp : nullptr, ctx->sm_count, (cudaStream_t)stream);
  tl.done();
  return e == cudaSuccess ? ADCT_OK : cuda_fail(ctx, e, "float forward launch");
}

adct_status adct_backward_f32(adct_context* ctx, const float* x, const float* gy, float* gx, int64_t planes,
                              int32_t H, int32_t W, const float* Qsoft, adct_stream_t stream) {
  Range nvtx("adct_backward_f32");
  adct_status st = check_float(ctx, x, gy, gx, planes, H, W);
  if (st != ADCT_OK) return st;
  FloatParams fp;
  if (Qsoft && (st = float_params(ctx, Qsoft, fp)) != ADCT_OK) return st;
  DeviceGuard guard(ctx->device);
  TimedLaunch tl(ctx, (cudaStream_t)stream);
  cudaError_t e =
      launch_float_backward(x, gy, gx, planes, H, W, Qsoft ? &fp : nullptr, ctx->sm_count, (cudaStream_t)stream);
  tl.done();
  return e == cudaSuccess ? ADCT_OK : cuda_fail(ctx, e, "float backward launch");
}

adct_status adct_roundtrip_graph(adct_context* ctx, const adct_image* imgs, int32_t n, const adct_quant* quant,
                                 adct_stream_t stream, int32_t* replayed) {
  Range nvtx("adct_roundtrip_graph");
  if (!ctx) return ADCT_ERR_INVALID_ARG;
  ctx->last_error.clear();
  if (replayed) *replayed = 0;
  if (n < 0 || (n > 0 && !imgs)) return fail(ctx, ADCT_ERR_INVALID_ARG, "bad image list");
  bool ok = true;
  const int kind = kind_for_roundtrip(imgs, n, ok);
  if (!ok) return fail(ctx, ADCT_ERR_INVALID_ARG, "coef/dst must be set on all images or on none");
  if (n > 0 && !imgs[0].coef && !imgs[0].dst) return fail(ctx, ADCT_ERR_INVALID_ARG, "need coef or dst");
  adct_status st = check_shape(ctx, ctx->shape);
  if (st != ADCT_OK) return st;
  CodecLaunch cl{};
  cl.kind = kind;
  cl.fault = ctx->fault;
  if (!quant) return fail(ctx, ADCT_ERR_INVALID_ARG, "quant is NULL");
  st = build_quant(ctx, quant, true, cl.qp, cl.evenq);
  if (st != ADCT_OK) return st;
  cl.qmode = quant->mode;
  Tables& t = scratch_tables();
  st = build_tables(ctx, imgs, n, need_for_kind(kind), false, coef_per_block(quant), t);
  if (st != ADCT_OK) return st;
  if (t.blocks == 0) return ADCT_OK;
  DeviceGuard guard(ctx->device);
  const std::string key = graph_key(imgs, n, quant, kind, ctx->shape);
  auto it = ctx->graphs.find(key);
  const size_t bytes = t.blob.size();
  if (it == ctx->graphs.end()) {
    GraphEntry g;
    g.bytes = bytes;
    if (device_alloc(&g.dev, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, ADCT_ERR_OOM, "graph workspace cudaMalloc failed");
    }
    if (cudaMallocHost(&g.host, bytes) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(g.dev);
      return fail(ctx, ADCT_ERR_OOM, "graph workspace cudaMallocHost failed");
    }
    ADCT_CUDA(ctx, cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming));
    cudaStream_t cs = ctx->capture_stream;
    // The graph holds the launches only; the table they read is uploaded
    // outside it, and only when it changes (below).
    ADCT_CUDA(ctx, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const adct_status s2 = launch_groups(ctx, cl, t, (const char*)g.dev, ctx->shape, cs, false);
    cudaError_t e3 = cudaStreamEndCapture(cs, &g.graph);
    if (s2 != ADCT_OK || e3 != cudaSuccess) {
      cudaGetLastError();
      if (g.graph) cudaGraphDestroy(g.graph);
      cudaEventDestroy(g.done);
      cudaFree(g.dev);
      cudaFreeHost(g.host);
      return fail(ctx, ADCT_ERR_CUDA, "graph capture failed");
    }
    ADCT_CUDA(ctx, cudaGraphInstantiate(&g.exec, g.graph, 0));
    it = ctx->graphs.emplace(key, g).first;
  } else if (replayed) {
    *replayed = 1;
  }
  GraphEntry& g = it->second;
  // Same shapes with other buffers give another table: wait until the last
  // replay has read the old one, then upload.  A batch replayed on the same
  // buffers (the steady state) uploads nothing and never waits on the host.
  if (g.uploaded.size() != bytes || std::memcmp(g.uploaded.data(), t.blob.data(), bytes) != 0) {
    if (g.pending) {
      ADCT_CUDA(ctx, cudaEventSynchronize(g.done));
      g.pending = false;
    }
    std::memcpy(g.host, t.blob.data(), bytes);
    ADCT_CUDA(ctx, cudaMemcpyAsync(g.dev, g.host, bytes, cudaMemcpyHostToDevice, (cudaStream_t)stream));
    g.uploaded.assign(t.blob.begin(), t.blob.end());
  }
  TimedLaunch tl(ctx, (cudaStream_t)stream);
  cudaError_t eg = cudaGraphLaunch(g.exec, (cudaStream_t)stream);
  tl.done();
  if (eg != cudaSuccess) return cuda_fail(ctx, eg, "cudaGraphLaunch");
  ADCT_CUDA(ctx, cudaEventRecord(g.done, (cudaStream_t)stream));
  g.pending = true;
  return ADCT_OK;
}

adct_status adct_autotune(adct_context* ctx, const adct_image* imgs, int32_t n, const adct_quant* quant,
                          adct_stream_t stream, int32_t reps, adct_launch* best, float* best_us) {
  Range nvtx("adct_autotune");
  if (!ctx || !best || reps < 1) return ADCT_ERR_INVALID_ARG;
  bool ok = true;
  if (n < 1 || !imgs) return fail(ctx, ADCT_ERR_INVALID_ARG, "autotune needs at least one image");
  const int kind = kind_for_roundtrip(imgs, n, ok);
  if (!ok) return fail(ctx, ADCT_ERR_INVALID_ARG, "coef/dst must be set on all images or on none");
  DeviceGuard guard(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  ADCT_CUDA(ctx, cudaEventCreate(&e0));
  ADCT_CUDA(ctx, cudaEventCreate(&e1));
  const int threads_c[] = {32, 64, 96, 128};
  const int ctas_c[] = {2, 3, 4, 5, 6, 8, 10, 12};
  float best_t = 1e30f;
  LaunchShape best_sh = ctx->shape;
  adct_status result = ADCT_OK;
  for (int stage : {0, 1})
  for (int th : threads_c) {
    for (int cps : ctas_c) {
      if (th * cps > 2048) continue;
      if ((size_t)cps * codec_smem_bytes(LaunchShape{th, cps, stage}, kind) > 200 * 1024) continue;  // shared memory per SM
      LaunchShape sh{th, cps, stage};
      adct_status st = run_codec(ctx, imgs, n, quant, kind, s, sh);  // warm-up
      if (st != ADCT_OK) { result = st; goto done; }
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps; ++r) {
        st = run_codec(ctx, imgs, n, quant, kind, s, sh);
        if (st != ADCT_OK) { result = st; goto done; }
      }
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) { result = cuda_fail(ctx, cudaGetLastError(), "autotune"); goto done; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const float us = 1000.f * ms / reps;
      if (us < best_t) { best_t = us; best_sh = sh; }
    }
  }
  ctx->shape = best_sh;
  best->threads_per_cta = best_sh.threads;
  best->ctas_per_sm = best_sh.ctas_per_sm;
  best->stage_coef = best_sh.stage_coef;
  best->reserved = 0;
  if (best_us) *best_us = best_t;
done:
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return result;
}

adct_status adct_roundtrip_host(adct_context* ctx, const adct_image* himgs, int32_t n, const adct_quant* quant,
                                int64_t chunk_bytes) {
  Range nvtx("adct_roundtrip_host");
  if (!ctx) return ADCT_ERR_INVALID_ARG;
  ctx->last_error.clear();
  if (n < 0 || (n > 0 && !himgs)) return fail(ctx, ADCT_ERR_INVALID_ARG, "bad image list");
  if (chunk_bytes <= 0) chunk_bytes = 32ll << 20;  // measured best: 16-32 MB
  bool ok = true;
  const int kind = kind_for_roundtrip(himgs, n, ok);
  if (!ok) return fail(ctx, ADCT_ERR_INVALID_ARG, "coef/dst must be set on all images or on none");
  if (n == 0) return ADCT_OK;
  if (!himgs[0].coef && !himgs[0].dst) return fail(ctx, ADCT_ERR_INVALID_ARG, "need coef or dst");
  // Host-side validation up front (shapes and pointers); device alignment is ours.
  for (int32_t m = 0; m < n; ++m) {
    const adct_image& im = himgs[m];
    if (im.layout != ADCT_LAYOUT_PLANAR)
      return fail(ctx, ADCT_ERR_UNSUPPORTED, "host buffers: planar images only (image " + std::to_string(m) + ")");
    if (im.width <= 0 || im.height <= 0 || im.width % 8 || im.height % 8 || im.width > 65536 || im.height > 65536 ||
        im.channels < 1 || im.pitch < im.width || (im.channels > 1 && im.plane_stride < im.pitch * im.height) ||
        !im.src)
      return fail(ctx, ADCT_ERR_SHAPE, "bad host image " + std::to_string(m) + " (sides multiples of 8)");
  }
  DeviceGuard guard(ctx->device);
  // chunk boundaries over whole images
  std::vector<int32_t> bounds{0};
  int64_t acc = 0;
  for (int32_t m = 0; m < n; ++m) {
    const int64_t pix = (int64_t)himgs[m].width * himgs[m].height * himgs[m].channels;
    if (acc > 0 && acc + pix > chunk_bytes) {
      bounds.push_back(m);
      acc = 0;
    }
    acc += pix;
  }
  bounds.push_back(n);
  size_t max_pix = 0, max_imgs = 0;
  for (size_t c = 0; c + 1 < bounds.size(); ++c) {
    size_t pix = 0;
    for (int32_t m = bounds[c]; m < bounds[c + 1]; ++m)
      pix += (size_t)himgs[m].width * himgs[m].height * himgs[m].channels;
    max_pix = std::max(max_pix, pix);
    max_imgs = std::max(max_imgs, (size_t)(bounds[c + 1] - bounds[c]));
  }
  const bool want_coef = himgs[0].coef != nullptr, want_dst = himgs[0].dst != nullptr;
  const int32_t cpb = coef_per_block(quant);
  for (auto& p : ctx->pipe) {
    if (!p.stream) ADCT_CUDA(ctx, cudaStreamCreateWithFlags(&p.stream, cudaStreamNonBlocking));
    const size_t pix_cap = (max_pix + 255) / 256 * 256;
    if (p.pix_cap < pix_cap) {
      cudaStreamSynchronize(p.stream);
      if (p.src) cudaFree(p.src);
      if (p.dst) cudaFree(p.dst);
      p.src = p.dst = nullptr;
      p.pix_cap = 0;
      if (device_alloc((void**)&p.src, pix_cap) != cudaSuccess ||
          device_alloc((void**)&p.dst, pix_cap) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, ADCT_ERR_OOM, "pipeline staging cudaMalloc failed");
      }
      p.pix_cap = pix_cap;
    }
    // coefficients: at most 128 bytes per 64 pixels, plus up to 16 bytes of
    // alignment padding per image (the packed layout's images are not
    // multiples of 16 bytes)
    const size_t coef_cap = 2 * pix_cap + 16 * max_imgs;
    if (p.coef_cap < coef_cap) {
      cudaStreamSynchronize(p.stream);
      if (p.coef) cudaFree(p.coef);
      p.coef = nullptr;
      p.coef_cap = 0;
      if (device_alloc((void**)&p.coef, coef_cap) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, ADCT_ERR_OOM, "pipeline staging cudaMalloc failed");
      }
      p.coef_cap = coef_cap;
    }
  }
  // 1D copies of contiguous images are merged with their neighbours when both
  // sides are contiguous, so a batch laid out back to back moves in a few
  // large copies instead of one per plane.
  struct Run {
    char* dst;
    const char* src;
    size_t bytes;
  };
  auto add_run = [](std::vector<Run>& runs, void* dst, const void* src, size_t bytes) {
    if (!runs.empty() && runs.back().dst + runs.back().bytes == (char*)dst &&
        runs.back().src + runs.back().bytes == (const char*)src)
      runs.back().bytes += bytes;
    else
      runs.push_back(Run{(char*)dst, (const char*)src, bytes});
  };
  std::vector<adct_image> dimgs;
  std::vector<Run> h2d, d2h_coef, d2h_pix;
  for (size_t c = 0; c + 1 < bounds.size(); ++c) {
    PipeSlot& p = ctx->pipe[c % kPipeSlots];
    cudaStream_t s = p.stream;
    dimgs.clear();
    h2d.clear();
    d2h_coef.clear();
    d2h_pix.clear();
    size_t off = 0, coff = 0;  // pixel and coefficient offsets into the staging buffers
    for (int32_t m = bounds[c]; m < bounds[c + 1]; ++m) {
      const adct_image& h = himgs[m];
      const size_t plane = (size_t)h.width * h.height;
      const bool packed = h.pitch == h.width && (h.channels == 1 || h.plane_stride == (int64_t)plane);
      adct_image d{};
      d.src = p.src + off;
      d.dst = want_dst ? p.dst + off : nullptr;
      d.coef = want_coef ? p.coef + coff : nullptr;
      d.width = h.width;
      d.height = h.height;
      d.channels = h.channels;
      d.pitch = h.width;
      d.plane_stride = (int64_t)plane;
      if (packed) {
        add_run(h2d, p.src + off, h.src, plane * h.channels);
      } else {
        for (int32_t ch = 0; ch < h.channels; ++ch)
          ADCT_CUDA(ctx, cudaMemcpy2DAsync(p.src + off + ch * plane, h.width, h.src + (int64_t)ch * h.plane_stride,
                                           h.pitch, h.width, h.height, cudaMemcpyHostToDevice, s));
      }
      if (want_coef) add_run(d2h_coef, h.coef, d.coef, plane / 64 * cpb * h.channels * sizeof(int16_t));
      if (want_dst) {
        if (packed) add_run(d2h_pix, h.dst, d.dst, plane * h.channels);
      }
      dimgs.push_back(d);
      off += plane * h.channels;
      coff += (plane / 64 * cpb * h.channels + 7) / 8 * 8;  // cpb int16 per block; 16-byte aligned images
    }
    for (const Run& r : h2d) ADCT_CUDA(ctx, cudaMemcpyAsync(r.dst, r.src, r.bytes, cudaMemcpyHostToDevice, s));
    adct_status st = run_codec(ctx, dimgs.data(), (int32_t)dimgs.size(), quant, kind, s, ctx->shape);
    if (st != ADCT_OK) return st;
    for (const Run& r : d2h_coef) ADCT_CUDA(ctx, cudaMemcpyAsync(r.dst, r.src, r.bytes, cudaMemcpyDeviceToHost, s));
    for (const Run& r : d2h_pix) ADCT_CUDA(ctx, cudaMemcpyAsync(r.dst, r.src, r.bytes, cudaMemcpyDeviceToHost, s));
    if (want_dst) {
      for (size_t k = 0; k < dimgs.size(); ++k) {
        const adct_image& h = himgs[bounds[c] + (int32_t)k];
        const adct_image& d = dimgs[k];
        const size_t plane = (size_t)h.width * h.height;
        const bool packed = h.pitch == h.width && (h.channels == 1 || h.plane_stride == (int64_t)plane);
        if (packed) continue;
        for (int32_t ch = 0; ch < h.channels; ++ch)
          ADCT_CUDA(ctx, cudaMemcpy2DAsync(h.dst + (int64_t)ch * h.plane_stride, h.pitch, d.dst + ch * plane, h.width,
                                           h.width, h.height, cudaMemcpyDeviceToHost, s));
      }
    }
  }
  for (auto& p : ctx->pipe) ADCT_CUDA(ctx, cudaStreamSynchronize(p.stream));
  return ADCT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Sharding plan for several GPUs (host only).
extern "C" adct_status adct_shard_plan(const adct_image* imgs, int32_t n, int32_t world, int32_t rank, int32_t* out,
                                       int32_t* count, int64_t* max_blocks) {
  if (world < 1 || rank < 0 || rank >= world || n < 0 || (n > 0 && !imgs) || !out || !count)
    return ADCT_ERR_INVALID_ARG;
  std::vector<int64_t> blocks((size_t)n);
  for (int32_t m = 0; m < n; ++m) {
    const adct_image& im = imgs[m];
    const bool inter = im.layout == ADCT_LAYOUT_INTERLEAVED;
    if (im.width <= 0 || im.height <= 0 || im.width > 65536 || im.height > 65536 || im.channels < 1 ||
        (im.layout != ADCT_LAYOUT_PLANAR && !inter) || (inter && im.channels != 3 && im.channels != 4))
      return ADCT_ERR_SHAPE;
    // any side: edge blocks count as whole blocks (ceil(side / 8) per side)
    blocks[m] = (int64_t)((im.width + 7) / 8) * ((im.height + 7) / 8) * im.channels;
  }
  std::vector<int32_t> order((size_t)n);
  for (int32_t m = 0; m < n; ++m) order[m] = m;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return blocks[a] > blocks[b]; });
  // min-heap of (load, rank): the least-loaded rank, lowest rank first on ties
  std::vector<std::pair<int64_t, int32_t>> heap;
  for (int32_t r = 0; r < world; ++r) heap.emplace_back(0, r);
  auto greater = [](const std::pair<int64_t, int32_t>& a, const std::pair<int64_t, int32_t>& b) { return a > b; };
  std::make_heap(heap.begin(), heap.end(), greater);
  std::vector<int32_t> owner((size_t)n);
  for (int32_t m : order) {
    std::pop_heap(heap.begin(), heap.end(), greater);
    owner[m] = heap.back().second;
    heap.back().first += blocks[m];
    std::push_heap(heap.begin(), heap.end(), greater);
  }
  int32_t k = 0;
  for (int32_t m = 0; m < n; ++m)
    if (owner[m] == rank) out[k++] = m;
  *count = k;
  if (max_blocks) {
    int64_t mx = 0;
    for (const auto& h : heap) mx = std::max(mx, h.first);
    *max_blocks = mx;
  }
  return ADCT_OK;
}

// ---------------------------------------------------------------------------
// Host-side diagnostic: the kernels' own butterfly templates on a counting type.
namespace {
thread_local int64_t g_adds = 0;
struct Counted {
  int64_t v;
};
// Host and device so that the butterfly templates (host-device functions)
// instantiate cleanly for it; only host calls exist, and only they count.
__host__ __device__ inline Counted operator+(Counted a, Counted b) {
#ifndef __CUDA_ARCH__
  ++g_adds;
#endif
  return Counted{a.v + b.v};
}
__host__ __device__ inline Counted operator-(Counted a, Counted b) {
#ifndef __CUDA_ARCH__
  ++g_adds;
#endif
  return Counted{a.v - b.v};
}
}  // namespace

extern "C" adct_status adct_butterfly_host(int32_t* vec8, int64_t count, int32_t inverse, int32_t* adds) {
  if (count < 0 || (count > 0 && !vec8)) return ADCT_ERR_INVALID_ARG;
  int64_t per = -1;
  for (int64_t c = 0; c < count; ++c) {
    Counted v[8];
    for (int k = 0; k < 8; ++k) v[k].v = vec8[8 * c + k];
    g_adds = 0;
    if (inverse) inv8<1>(v);
    else fwd8<1>(v);
    if (per < 0) per = g_adds;
    if (per != g_adds) return ADCT_ERR_INVALID_ARG;
    for (int k = 0; k < 8; ++k) vec8[8 * c + k] = (int32_t)v[k].v;
  }
  if (adds) {
    if (per < 0) {
      Counted v[8] = {};
      g_adds = 0;
      if (inverse) inv8<1>(v);
      else fwd8<1>(v);
      per = g_adds;
    }
    *adds = (int32_t)per;
  }
  return ADCT_OK;
}

// ---------------------------------------------------------------------------
// adct_roundtrip_noalloc: the round trip for callers that cannot allocate.
// The descriptor table that adct_roundtrip keeps in a context workspace lives
// here in a fixed device array instead; the kernel is the same.
namespace {

constexpr int kNoAllocPlanes = ADCT_NOALLOC_MAX_PLANES;
constexpr size_t kNoAllocTable = kNoAllocPlanes * sizeof(PlaneDesc);
constexpr size_t kNoAllocBytes = kNoAllocTable + (kNoAllocPlanes + kGroups) * sizeof(int64_t);

// Held by every device that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Host-side view of g_noalloc_scratch: its device address and the SM count,
// looked up once per device (with that device current).  The symbol's name in
// host code is only a stand-in; the kernel must get the looked-up address.
constexpr int kNoAllocMaxDevices = 64;
struct NoAllocDevice {
  bool ready = false;
  void* scratch = nullptr;
  int sm_count = 0;
};
NoAllocDevice g_noalloc_devices[kNoAllocMaxDevices];
std::mutex g_noalloc_mutex;

// Host copy of the table, built call by call in this one buffer (guarded by
// g_noalloc_table_mutex) and copied into g_noalloc_scratch: the same layout.
struct NoAllocTable {
  PlaneDesc planes[kNoAllocPlanes];
  int64_t starts[kNoAllocPlanes + kGroups];
};
static_assert(sizeof(NoAllocTable) == kNoAllocBytes, "host table layout matches the device array");
NoAllocTable g_noalloc_table;
std::mutex g_noalloc_table_mutex;

adct_status noalloc_device(int dev, void** scratch, int* sm_count) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return ADCT_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  NoAllocDevice& d = g_noalloc_devices[dev];
  if (!d.ready) {
    int major = 0, minor = 0, sms = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return ADCT_ERR_CUDA;
    }
    if (major != 10 || minor != 3) return ADCT_ERR_UNSUPPORTED;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return ADCT_ERR_CUDA;
    }
    d.scratch = p;
    d.sm_count = sms;
    d.ready = true;
  }
  *scratch = d.scratch;
  *sm_count = d.sm_count;
  return ADCT_OK;
}

}  // namespace

extern "C" adct_status adct_roundtrip_noalloc(const adct_image* imgs, int32_t n, const adct_quant* quant,
                                              adct_stream_t stream) {
  Range nvtx("adct_roundtrip_noalloc");
  if (n < 0 || (n > 0 && !imgs) || !quant) return ADCT_ERR_INVALID_ARG;
  if (n == 0) return ADCT_OK;
  const bool want_coef = imgs[0].coef != nullptr, want_dst = imgs[0].dst != nullptr;
  if (!want_coef && !want_dst) return ADCT_ERR_INVALID_ARG;
  CodecLaunch cl{};  // cl.fault stays null: no context, so a checked build reports no bounds faults here
  cl.kind = (want_coef && want_dst) ? K_RT_FULL : (want_dst ? K_RT_PIX : K_RT_COEF);
  adct_status st = build_quant(nullptr, quant, true, cl.qp, cl.evenq);
  if (st != ADCT_OK) return st;
  cl.qmode = quant->mode;

  // Validation first (nothing shared is touched): the plane count is checked
  // against the table's capacity before it is added, so no channel count,
  // however large, can overflow the sum.
  const int need = NEED_SRC | (want_coef ? NEED_COEF : 0) | (want_dst ? NEED_DST : 0);
  const int32_t cpb = coef_per_block(quant);
  int32_t planes_total = 0;
  for (int32_t m = 0; m < n; ++m) {
    const adct_image& im = imgs[m];
    if ((im.coef != nullptr) != want_coef || (im.dst != nullptr) != want_dst) return ADCT_ERR_INVALID_ARG;
    const char* why = "";
    st = check_image(im, need, false, &why);
    if (st != ADCT_OK) return st;
    const int32_t add = im.layout == ADCT_LAYOUT_INTERLEAVED ? 1 : im.channels;
    if (add > kNoAllocPlanes - planes_total) return ADCT_ERR_TOO_LARGE;
    planes_total += add;
  }

  // The descriptor tables are built in the library's one host buffer (not on
  // the caller's stack, which may be small on threads that a host application
  // owns), under a lock held until the copy to the device has been issued.
  std::lock_guard<std::mutex> table_lock(g_noalloc_table_mutex);
  NoAllocTable& table = g_noalloc_table;
  // The groups (pixel layout classes) are laid out one after the other, all
  // planes first, then each group's flat-index prefix.
  int32_t np = 0, gfirst[kGroups], gcount[kGroups];
  for (int g = 0; g < kGroups; ++g) {  // one pass per group keeps each group's descriptors together
    gfirst[g] = np;
    int32_t pid = 0;
    for (int32_t m = 0; m < n; ++m) {
      if (group_of(imgs[m], false) == g) describe_image(imgs[m], cpb, false, pid, table.planes, &np);
      pid += imgs[m].channels;
    }
    gcount[g] = np - gfirst[g];
  }
  // prefixes: group g's at starts[gfirst[g] + g .. gfirst[g] + g + gcount[g]]
  for (int g = 0; g < kGroups; ++g) {
    int64_t total = 0;
    int64_t* st0 = table.starts + gfirst[g] + g;
    for (int32_t k = 0; k < gcount[g]; ++k) {
      const PlaneDesc& d = table.planes[gfirst[g] + k];
      st0[k] = total;
      total += (int64_t)d.wb * d.hb;
    }
    st0[gcount[g]] = total;
  }

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return ADCT_ERR_CUDA;
  }
  void* scratch = nullptr;
  int sm_count = 0;
  st = noalloc_device(dev, &scratch, &sm_count);
  if (st != ADCT_OK) return st;
  // planes at offset 0, the groups' prefixes right after them
  const size_t plane_bytes = (size_t)np * sizeof(PlaneDesc);
  const size_t start_bytes = (size_t)(np + kGroups) * sizeof(int64_t);
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(scratch, table.planes, plane_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync((char*)scratch + plane_bytes, table.starts, start_bytes, cudaMemcpyHostToDevice, s) !=
          cudaSuccess) {
    cudaGetLastError();
    return ADCT_ERR_CUDA;
  }
  const LaunchShape shape{128, 0, 1};
  for (int g = 0; g < kGroups; ++g) {
    if (gcount[g] == 0) continue;
    cl.planes = (const PlaneDesc*)scratch + gfirst[g];
    cl.starts = (const int64_t*)((char*)scratch + plane_bytes) + gfirst[g] + g;
    cl.nplanes = gcount[g];
    cl.total = table.starts[gfirst[g] + g + gcount[g]];
    cl.nch = kGroupNch[g];
    cl.edge = kGroupEdge[g];
    if (launch_codec(cl, shape, sm_count, s) != cudaSuccess) {
      cudaGetLastError();
      return ADCT_ERR_CUDA;
    }
  }
  return ADCT_OK;
}
