/*
 * adct.h -- C ABI of the GB300 (sm_103a) library for the 14-addition orthogonal
 * approximate DCT of Bayer & Cintra, "DCT-like Transform for Image Compression
 * Requires 14 Additions Only" (arXiv 1702.00817).
 *
 * What the library computes (notation of the paper):
 *   T      the 8x8 matrix with entries in {0, +1, -1} (Sec. 2);
 *   D      diag(1/sqrt8, 1/sqrt2, 1/2, 1/sqrt2, 1/sqrt8, 1/sqrt2, 1/2, 1/sqrt2), so
 *          D^2 = diag(2^-a_i), a = (3,1,2,1,3,1,2,1), and C^ = D T is orthogonal (Sec. 2);
 *   fast algorithm  T = P A3 A2 A1: 14 additions per 8-point transform (Sec. 2, Table 1).
 * The image codec follows the paper's JPEG-style experiment (Sec. 3): every 8x8
 * block of a uint8 plane (each channel of a planar or interleaved image, edge
 * blocks extended by replication) goes through the separable 2D transform,
 * then a quantiser, then the inverse procedure:
 *   forward      Z = T (X - 128) T^T                       rows, then columns, integers
 *   quantise     STEP : q = sgn(Z) floor((2|Z| + Q) / (2Q))  (round half away from zero)
 *                ZONAL: q = Z if zig-zag rank(i,j) < r, else 0   (Sec. 3)
 *                STEP_ZONAL: STEP, then the ZONAL mask; NONE: q = Z;
 *                ZONAL_ZZ: ZONAL, storing only the r kept values in zig-zag order
 *   dequantise   S_ij = q_ij Q_ij 2^(6 - a_i - a_j)           (D^2 merged into the step, Sec. 2)
 *   inverse      R = T^T S T                                (T^-1 = T^T D^2, Sec. 2)
 *   reconstruct  pixel = clamp(floor((R + 32) / 64) + 128, 0, 255)
 * Every integer result is exact (no rounding other than the two stated above).
 *
 * Conventions for every entry point:
 *   - Pointers named in adct_image and the float tensors are DEVICE memory
 *     owned by the caller; the library never frees or retains them after a call
 *     completes on its stream.  The adct_image and adct_quant arrays themselves
 *     are HOST memory, read during the call only.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL is the legacy
 *     default stream).  Argument errors are detected on the host before any
 *     launch and nothing is launched.  CUDA errors return ADCT_ERR_CUDA with the
 *     CUDA message kept in adct_last_error().
 *   - A context is not thread-safe: use one per host thread.
 *   - A context allocates a small device workspace for per-call descriptor
 *     tables; calls may overlap on different streams (the workspace is a ring of
 *     slots guarded by events).
 */
#ifndef ADCT_H
#define ADCT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream handle (identical to cudaStream_t). */
typedef struct CUstream_st* adct_stream_t;

typedef enum {
  ADCT_OK = 0,
  ADCT_ERR_INVALID_ARG = 1, /* null pointer, bad count, bad quantiser or launch parameter */
  ADCT_ERR_SHAPE = 2,       /* width/height outside 1..65536 (multiples of 8 where required), bad pitch/stride */
  ADCT_ERR_ALIGN = 3,       /* src/dst/pitch/plane_stride not 8-byte, coef not 16-byte aligned */
  ADCT_ERR_OOM = 4,         /* workspace allocation failed */
  ADCT_ERR_CUDA = 5,        /* a CUDA call failed; see adct_last_error */
  ADCT_ERR_TIMEOUT = 6,     /* a bounded wait gave up */
  ADCT_ERR_UNSUPPORTED = 7, /* device is not sm_103 / feature not available */
  ADCT_ERR_TOO_LARGE = 8,   /* more planes than adct_roundtrip_noalloc can hold */
  ADCT_ERR_CANCELLED = 9    /* a server request withdrawn by adct_server_cancel before it ran */
} adct_status;

/* Quantiser modes (adct_quant.mode). */
enum { ADCT_Q_NONE = 0, ADCT_Q_STEP = 1, ADCT_Q_ZONAL = 2, ADCT_Q_STEP_ZONAL = 3, ADCT_Q_ZONAL_ZZ = 4 };

typedef struct adct_context adct_context;

/* Pixel layouts (adct_image.layout). */
enum { ADCT_LAYOUT_PLANAR = 0, ADCT_LAYOUT_INTERLEAVED = 1 };

/*
 * One uint8 image of `channels` channels, height x width pixels (each side
 * 1..65536).  Sides that are not multiples of 8 are covered by ceil(side / 8)
 * blocks whose missing pixels replicate the last column / row of the image
 * (JPEG-style edge extension); reconstructions write only the image's pixels.
 *   layout ADCT_LAYOUT_PLANAR: `channels` planes, rows `pitch` bytes apart
 *          (pitch >= width), planes `plane_stride` bytes apart
 *          (plane_stride >= pitch * height when channels > 1).
 *   layout ADCT_LAYOUT_INTERLEAVED: channels = 3 or 4 interleaved per pixel
 *          (HWC: pixel (y, x), channel c at y * pitch + x * channels + c), rows
 *          `pitch` bytes apart (pitch >= width * channels); plane_stride unused.
 * src and dst share the layout, pitch and plane_stride; pitch and plane_stride
 * are multiples of 8, and every row of a plane or image, the last one
 * included, spans `pitch` addressable bytes (the kernels read whole 8-byte
 * chunks up to ceil8(width * channels), never beyond pitch).
 *   src   pixels read by the forward transform            (8-byte aligned)
 *   dst   reconstructed pixels (may equal src)            (8-byte aligned)
 *   coef  int16 coefficients, planar and block-major for both pixel layouts:
 *         coef[((c * Hb + by) * Wb + bx) * 64 + i * 8 + j]
 *         with Hb = ceil(height / 8), Wb = ceil(width / 8), (i, j) = (row, column)
 *         frequency  (16-byte aligned).
 *         With the quantiser mode ADCT_Q_ZONAL_ZZ coef is packed instead: r int16
 *         per block, coef[((c * Hb + by) * Wb + bx) * r + t] = the coefficient at
 *         zig-zag position t (t < r); only 2-byte alignment of the plane blocks
 *         follows from this, the image's coef pointer stays 16-byte aligned.
 * A pointer an entry point does not use may be NULL.
 * Coefficient range: |Z_ij| <= 128 * 2^(a_i + a_j) <= 8192, so int16 is exact.
 */
typedef struct {
  const uint8_t* src;
  uint8_t* dst;
  int16_t* coef;
  int32_t width;
  int32_t height;
  int32_t channels;
  int32_t layout; /* ADCT_LAYOUT_* */
  int64_t pitch;
  int64_t plane_stride;
} adct_image;

/*
 * Quantiser.  mode: ADCT_Q_*.  Q: step table, row-major (i*8 + j), each entry in
 * [1, 65535] (used by STEP and STEP_ZONAL, ignored otherwise: Q = 1).
 * r: number of zig-zag coefficients kept, 0..64 (ZONAL, STEP_ZONAL, ZONAL_ZZ).
 * ADCT_Q_ZONAL_ZZ is the ZONAL quantiser (q = Z at the first r zig-zag
 * positions, 0 elsewhere) with the packed coefficient layout of adct_image:
 * only the r kept values are stored, 2r bytes per block instead of 128.  It is
 * written by the round trip entry points and read by adct_inverse;
 * adct_quantise returns ADCT_ERR_UNSUPPORTED for it (the layouts differ).
 */
typedef struct {
  int32_t mode;
  int32_t r;
  uint16_t Q[64];
} adct_quant;

/*
 * Launch shape of the integer kernels (one 8x8 block per thread, each warp a
 * tile of 32 blocks, up to 16.5 KB of shared memory per warp).  Zero fields of
 * threads_per_cta / ctas_per_sm keep the current value.
 *   threads_per_cta   multiple of 32 in [32, 128] (default 128)
 *   ctas_per_sm       CTAs per SM the persistent grid is sized for (1..32); capped
 *                     at the number that can be resident at once.  A negative
 *                     value (and a new context) leaves the choice to the
 *                     library, per kernel: 4, or 3 for the encode with dense
 *                     coefficient output; adct_get_launch then reports 0.
 *                     In that mode the launches for channel-interleaved images
 *                     use CTAs of 32 threads, 12 per SM, whatever
 *                     threads_per_cta says
 *   stage_coef        0: each thread stores its 128 coefficient bytes directly;
 *                     1: coefficients are staged through shared memory and
 *                        written by the warp as contiguous 512-byte stores;
 *                    -1 (a new context): the library's choice per call, 1
 *                        except for the packed zonal round trip with r <= 8,
 *                        whose few coefficients per block go out directly
 *   reserved          must be 0
 */
typedef struct {
  int32_t threads_per_cta;
  int32_t ctas_per_sm;
  int32_t stage_coef;
  int32_t reserved;
} adct_launch;

/* Create a context on CUDA device `device` (checks for compute capability 10.3).
 * On success *ctx owns a workspace; release it with adct_destroy. */
adct_status adct_create(adct_context** ctx, int32_t device);

/* Destroy a context after synchronising its workspace events.  NULL is a no-op. */
void adct_destroy(adct_context* ctx);

/*
 * Forward 2D transform (Sec. 2 matrix T applied as the 14-addition fast
 * algorithm T = P A3 A2 A1, rows then columns; Sec. 3 blockwise over 8x8
 * blocks): coef = Z = T (src - 128) T^T for every block of the n images.
 * Uses src and coef.  One launch over all planes of all images.
 */
adct_status adct_forward(adct_context* ctx, const adct_image* imgs, int32_t n, adct_stream_t stream);

/*
 * Quantise coefficients in place (Sec. 2 D^2 merged step quantiser, Sec. 3
 * zig-zag zonal retention): coef <- q(coef).  Uses coef only.  The input must
 * hold forward coefficients (|Z_ij| <= 8192); larger magnitudes give
 * unspecified (but memory-safe) results.
 */
adct_status adct_quantise(adct_context* ctx, const adct_image* imgs, int32_t n, const adct_quant* quant,
                          adct_stream_t stream);

/*
 * Dequantise with D^2 merged (S_ij = q_ij Q_ij 2^(6 - a_i - a_j), Q = 1 for NONE
 * and ZONAL), invert R = T^T S T with the transposed 14-addition flow graph, and
 * reconstruct dst = clamp(floor((R + 32) / 64) + 128, 0, 255) (Sec. 2
 * orthogonality; Sec. 3 "inverse procedure").  Uses coef and dst.  coef must
 * hold quantiser output for this quant, which guarantees |q_ij Q_ij| <= 16384
 * and keeps the 32-bit arithmetic exact; other values give unspecified (but
 * memory-safe) pixels.
 */
adct_status adct_inverse(adct_context* ctx, const adct_image* imgs, int32_t n, const adct_quant* quant,
                         adct_stream_t stream);

/*
 * Fused round trip in one pass over HBM: forward, quantise, then (if dst is
 * non-NULL) dequantise + inverse + reconstruct.  q is written to coef when coef
 * is non-NULL.  At least one of coef and dst must be non-NULL.  dst may alias
 * src (each block is read before it is written).  Results equal adct_forward,
 * adct_quantise, adct_inverse run in sequence, bit for bit.
 */
adct_status adct_roundtrip(adct_context* ctx, const adct_image* imgs, int32_t n, const adct_quant* quant,
                           adct_stream_t stream);

/*
 * Quality of the round trip (Sec. 3, the figures of merit of the image
 * experiment): runs forward, quantise, dequantise and inverse like
 * adct_roundtrip but writes no pixels or coefficients; instead sse[p] receives
 * the sum over plane p of (reconstructed pixel - src pixel)^2 (exact, 64-bit).
 * Planes are numbered image by image, channel by channel.  Uses src only.
 * sse: DEVICE array of one uint64 per plane (8-byte aligned), overwritten.
 * MSE = sse / (width * height); PSNR = 10 log10(255^2 / MSE).
 */
adct_status adct_quality(adct_context* ctx, const adct_image* imgs, int32_t n, const adct_quant* quant, uint64_t* sse,
                         adct_stream_t stream);

/*
 * The exact-DCT comparator of the quality experiment (Sec. 3 compares the
 * approximation against the DCT): zonal round trip with the orthonormal 8x8
 * DCT-II in float32, keeping the first r zig-zag coefficients, reconstruction
 * rounded to nearest (ties to even) and clamped to 0..255; sse as for
 * adct_quality.  r in 0..64.
 */
adct_status adct_quality_dct(adct_context* ctx, const adct_image* imgs, int32_t n, int32_t r, uint64_t* sse,
                             adct_stream_t stream);

/*
 * Differentiable float32 variant (Sec. 2 C^ = D T).  x, y: [planes][H][W]
 * float32 row-major device tensors (H, W multiples of 8, 16-byte aligned).
 * y = D T x T^T D per 8x8 block, followed, when Qsoft (HOST array of 64
 * positive floats, row-major i*8+j) is non-NULL, by the soft quantiser
 * y <- y - (Q/2pi) sin(2pi y / Q).
 */
adct_status adct_forward_f32(adct_context* ctx, const float* x, float* y, int64_t planes, int32_t H, int32_t W,
                             const float* Qsoft, adct_stream_t stream);

/*
 * Adjoint of adct_forward_f32 with respect to x (hand-written backward):
 * gx = T^T D (gy * (1 - cos(2pi y / Q))) D T per block, y recomputed from x
 * (the factor is 1 when Qsoft is NULL).  Same layout rules as the forward.
 */
adct_status adct_backward_f32(adct_context* ctx, const float* x, const float* gy, float* gx, int64_t planes,
                              int32_t H, int32_t W, const float* Qsoft, adct_stream_t stream);

/* Set / read the launch shape used by the integer entry points of ctx. */
adct_status adct_set_launch(adct_context* ctx, const adct_launch* launch);
adct_status adct_get_launch(adct_context* ctx, adct_launch* launch);

/*
 * Round trip through a CUDA graph cached in ctx per batch signature (image
 * count, sizes, channel counts, quantiser mode, launch shape and which of
 * coef/dst are used).  The first call with a signature captures the kernel
 * launches (one per pixel layout class) reading a descriptor table owned by
 * the graph; each call uploads that table on `stream` only when it differs
 * from the one already on the device (other buffers of the same shapes),
 * after waiting on the host for the graph's previous replay, and then
 * replays.  A batch replayed on the same buffers uploads nothing and does not
 * wait.  Results are identical to adct_roundtrip.  *replayed (nullable) is
 * set to 1 when a cached graph was replayed.
 */
adct_status adct_roundtrip_graph(adct_context* ctx, const adct_image* imgs, int32_t n, const adct_quant* quant,
                                 adct_stream_t stream, int32_t* replayed);

/*
 * Autotune the launch shape for this batch: times each candidate (threads per
 * CTA x CTAs per SM x coefficient staging) with CUDA events
 * over `reps` round trips after one warm-up, keeps the fastest in ctx and
 * writes it to *best, its mean time in microseconds to *best_us (nullable).
 * Runs synchronously on `stream`; outputs of the batch are overwritten.
 */
adct_status adct_autotune(adct_context* ctx, const adct_image* imgs, int32_t n, const adct_quant* quant,
                          adct_stream_t stream, int32_t reps, adct_launch* best, float* best_us);

/*
 * End-to-end round trip on HOST buffers: the adct_image pointers (src, dst,
 * coef) are host memory (pinned memory gives full copy bandwidth).  Images are
 * processed in chunks of about chunk_bytes of pixels (<= 0: 32 MiB), each chunk copied to the
 * device, transformed with adct_roundtrip and copied back, with chunks
 * pipelined over the context's copy/compute streams.  Device staging is owned
 * by ctx and grows to the largest chunk.  Synchronous: returns when every
 * output is in host memory.  Planar images with sides that are multiples of 8
 * only: ADCT_ERR_UNSUPPORTED for an interleaved image, ADCT_ERR_SHAPE for
 * other sides (the device entry points take any size).
 */
adct_status adct_roundtrip_host(adct_context* ctx, const adct_image* host_imgs, int32_t n, const adct_quant* quant,
                                int64_t chunk_bytes);

/*
 * Bounds-check report of the checked build (libadct_checked.so, compiled with
 * ADCT_CHECKED; the paper has no counterpart -- a stand-in for a memory
 * checker).  Its kernels verify that every tile position lies inside its
 * plane's blocks and that no pixel copy passes the end of a row; a violation
 * sets a bit (1: position, 2: row bytes) in a per-context device word and the
 * access is skipped.  This call waits for the device, returns the word in
 * *faults and clears it.  The release build returns ADCT_ERR_UNSUPPORTED with
 * *faults = 0.
 */
adct_status adct_checked_faults(adct_context* ctx, uint32_t* faults);

/*
 * Multi-GPU sharding of one batch, with no collective (the blocks of different
 * images never interact, Sec. 3): a deterministic partition of the n images
 * over `world` ranks balanced by 8x8 block count -- images taken largest first
 * (ties: lower index), each given to the rank with the fewest blocks so far
 * (ties: lower rank).  Every rank computes the same plan on its own.  Only the
 * shape fields of imgs are read (pointers may be NULL); shapes are validated
 * as for adct_roundtrip.  Writes the indices of the images of `rank`, in
 * increasing order, to out (host array with room for n) and their number to
 * *count; *max_blocks (nullable) receives the largest per-rank block total.
 * Host only: no device or context is used.  Errors: ADCT_ERR_INVALID_ARG for
 * world < 1, rank outside [0, world) or NULL out/count; ADCT_ERR_SHAPE for a
 * bad image shape.
 */
adct_status adct_shard_plan(const adct_image* imgs, int32_t n, int32_t world, int32_t rank, int32_t* out,
                            int32_t* count, int64_t* max_blocks);

/*
 * Diagnostic (host-side, no GPU needed): run the library's own 8-point
 * butterfly -- the same template the kernels instantiate -- on `count`
 * vectors of 8 int32 in place, forward (X = T x) or inverse (x = T^T X), and
 * report the number of additions/subtractions one 8-point transform performs
 * in *adds (nullable).  Table 1 of the paper gives 14.
 */
adct_status adct_butterfly_host(int32_t* vec8, int64_t count, int32_t inverse, int32_t* adds);

/*
 * Kernel timing for benchmarks.  adct_kernel_timing(ctx, 1) makes every
 * kernel (or captured graph) the context launches from then on be bracketed
 * by a pair of CUDA events recorded on the launch stream; 0 stops it.
 * adct_kernel_time waits for those events and returns the summed device time
 * of the bracketed launches in *total_ms and the number of kernels launched by
 * the context since the previous query in *launches (both nullable), then
 * resets the two counters.
 */
adct_status adct_kernel_timing(adct_context* ctx, int32_t enable);
adct_status adct_kernel_time(adct_context* ctx, double* total_ms, int64_t* launches);

/*
 * Round trip that allocates nothing.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc, such as plug-ins that
 * must stay inside a device-memory pool or budget owned by their host
 * application, latency-critical loops that cannot afford the implicit device
 * synchronisation of cudaMalloc/cudaFree, and services that must not meet an
 * out-of-memory failure after start-up.
 *
 * Same arguments and results as adct_roundtrip (bit for bit), but no context:
 * the per-call plane descriptor table lives in a fixed device array inside the
 * library, sized for ADCT_NOALLOC_MAX_PLANES planes (a plane is one channel of
 * one image; an interleaved image counts as one): 73,776 bytes (1024 64-byte
 * descriptors plus 1030 8-byte block-count prefixes) that every GPU which
 * loads the library keeps until the process exits.  A batch with more planes
 * returns ADCT_ERR_TOO_LARGE and launches nothing.  It runs on the calling
 * thread's current CUDA device; the first call on a device looks up that
 * array's device address, so make the first call before any stream capture.
 * The table is built in one host buffer of the same size inside the library
 * (not on the caller's stack, so threads with small stacks can call it),
 * under a lock that calls from several host threads take in turn, and copied on
 * `stream` (a copy from pageable memory, so the call waits for the work
 * already queued on that stream).  Every call shares the one device array and
 * it keeps the last call's table; nothing in it needs clearing, because each
 * call writes the whole table it reads.  Calls whose work overlaps on the GPU
 * (on different streams, or from different host threads) race on the array:
 * serialise them on one stream.  Argument errors return the same codes as
 * adct_roundtrip (there is no context, so no adct_last_error message, and in
 * the checked build the kernels' bounds checks have no fault word to report
 * to on this path: a tile outside its plane is skipped without a report).
 */
#define ADCT_NOALLOC_MAX_PLANES 1024
adct_status adct_roundtrip_noalloc(const adct_image* imgs, int32_t n, const adct_quant* quant, adct_stream_t stream);

/*
 * Continuous-batching encode/decode server (serving; the paper's encode and
 * decode procedures of Sec. 3 as a request stream).  A scheduler thread owns a
 * context, a device-memory arena of budget_bytes (one cudaMalloc at creation)
 * and an on-device store of quantised coefficients.  Requests submitted while
 * others run are admitted as arena space frees up (the oldest store entries
 * that no pending decode uses are evicted when needed); each scheduler pass
 * packs its admissions into one encode launch and one decode launch on the next
 * of its streams, so batches overlap on the device.  Results are identical to
 * adct_roundtrip / adct_inverse on the same inputs.
 *   encode: host pixels (width x height uint8, rows pitch bytes apart; width
 *           and height multiples of 8 up to 65536, else ADCT_ERR_SHAPE) are
 *           copied in, forward-transformed and quantised; the coefficients stay
 *           in the store under the handle reported by the completion (2r bytes
 *           per block with ADCT_Q_ZONAL_ZZ, 128 otherwise).
 *   decode: a stored handle is dequantised and inverted; the pixels are copied
 *           to host memory `out` (rows pitch bytes apart; width/height of the
 *           encoded image are returned).  The handle is pinned from submission
 *           to completion.
 * Host buffers must stay valid until the request completes; pinned memory gives
 * asynchronous copies.  Timestamps are seconds on adct_server_clock()'s
 * monotonic clock (t_submit may be supplied by the caller on that clock, else
 * the submission time is used).  Submission and polling are thread-safe.
 */
typedef struct adct_server adct_server;

typedef struct {
  int64_t budget_bytes; /* device memory for in-flight work and the store (0: 4 GiB) */
  int32_t streams;      /* CUDA streams used to overlap batches (0: 4) */
  int32_t max_batch;    /* requests packed into one launch (0: 256) */
  adct_quant quant;     /* quantiser of every request */
} adct_server_config;

typedef struct {
  uint64_t request_id;
  int32_t status;  /* ADCT_OK; ADCT_ERR_INVALID_ARG: handle unknown; ADCT_ERR_OOM: larger than the budget; ADCT_ERR_CUDA */
  int32_t kind;    /* 0 encode, 1 decode */
  uint64_t handle; /* encode: handle of the stored coefficients; decode: the handle decoded */
  double t_submit, t_admit, t_done;
} adct_completion;

/*
 * Server counters.  latency_hist[b] counts completed requests whose latency
 * (t_done - t_submit) fell in [2^b, 2^(b+1)) microseconds (b = 0 also takes
 * shorter ones, b = 31 longer ones).
 */
typedef struct {
  int64_t launches, admitted, evicted, unknown_handle, oversized, errors, store_entries, arena_free_bytes;
  int32_t max_overlap, reserved;
  int64_t cancelled;
  int64_t latency_hist[32];
} adct_server_stats_t;

adct_status adct_server_create(adct_server** srv, int32_t device, const adct_server_config* cfg);
/* Stops the scheduler after the batches in flight complete, then frees everything. */
void adct_server_destroy(adct_server* srv);
adct_status adct_server_encode(adct_server* srv, const uint8_t* pixels, int32_t width, int32_t height, int64_t pitch,
                               double t_submit, uint64_t* request_id);
/* Fails at once (ADCT_ERR_INVALID_ARG) for a handle not in the store. */
adct_status adct_server_decode(adct_server* srv, uint64_t handle, uint8_t* out, int64_t pitch, double t_submit,
                               uint64_t* request_id, int32_t* width, int32_t* height);
/*
 * Withdraws a request that has not been admitted yet: it will not run, and its
 * completion reports ADCT_ERR_CANCELLED (a cancelled decode releases its pin
 * on the handle).  A request already admitted runs to completion as usual.
 * ADCT_ERR_INVALID_ARG: no such pending request (unknown, or already complete).
 */
adct_status adct_server_cancel(adct_server* srv, uint64_t request_id);
/* Moves up to max completions into out, waiting up to wait_us for the first; returns the count. */
int32_t adct_server_poll(adct_server* srv, adct_completion* out, int32_t max, int32_t wait_us);
adct_status adct_server_stats(adct_server* srv, adct_server_stats_t* stats);
/* The server's clock: seconds, CLOCK_MONOTONIC (the clock of Python's time.perf_counter on Linux). */
double adct_server_clock(void);

/* Human-readable name of a status code (static string). */
const char* adct_status_string(adct_status status);

/* Last error message recorded in ctx ("" if none).  Valid until the next call on ctx. */
const char* adct_last_error(adct_context* ctx);

#ifdef __cplusplus
}
#endif

#endif /* ADCT_H */
