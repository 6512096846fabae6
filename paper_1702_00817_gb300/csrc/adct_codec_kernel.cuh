// Integer codec kernel for sm_103a (templates, instantiated by adct_codec.cu
// for every kind and quantiser mode, by adct_codec_zonal_*.cu specialised on
// the zonal zone, by adct_codec_edge.cu for planar images with edge blocks and
// by adct_codec_interleaved*.cu for HWC images): the blockwise 2D 14-addition
// transform (Sec. 2 fast algorithm T = P A3 A2 A1; Sec. 3 8x8 blocks), the
// D^2-merged quantiser and the inverse, as one persistent kernel over a
// flattened block index.  The path is add-only and bound by HBM bytes, so no
// tensor cores.
//
// Work split.  The grid is sized to the SMs; each warp owns a contiguous
// chunk of the flat block index and walks it in tiles of 32 blocks (32 pixel
// positions of C channels for interleaved images), one 8x8 block per lane.  An
// 8x8 block lives in 64 registers, so both passes of the separable transform
// and the transpose between them are register renaming.
//
// Memory pipeline per warp (all in the warp's slice of shared memory):
//   - the next tile's input is prefetched with cp.async while the current one
//     is computed (pixels: each lane copies its block's 8 rows, 8 bytes each
//     -- 8 C bytes for interleaved images -- so one copy instruction of the
//     warp moves 256 contiguous bytes; coefficients: the warp copies the
//     tile's contiguous 4 KB, 512 bytes per instruction, into a 16-byte-chunk
//     XOR swizzle);
//   - quantised coefficients of a full tile are staged in the same swizzle and
//     written back as 512-byte contiguous warp stores (one L2 request per
//     128-byte line instead of one per 16 bytes); packed zonal coefficients
//     are staged per lane and written back as one contiguous range;
//   - reconstructed pixels are stored directly (256 contiguous bytes per warp
//     instruction already), or, for interleaved images, put back into the
//     channels' planar tiles and stored by each lane as re-interleaved rows
//     once every channel is done.
//
// Arithmetic per block (one lane):
//   forward  raw bytes -> 8 row butterflies -> 8 column butterflies (Z + 8192 e0e0^T);
//   quantise n = Z + c (bias, offset and level shift folded into one constant,
//            added by the last butterfly stage), m = umulhi(n, magic) = floor(n / Q),
//            q = m - K; for tables with even steps the sign of Z moves the bias by
//            one so that ties round away from zero;
//   dequant  S = q w, w = 4 Q 2^(6 - a_i - a_j) (D^2 merged), + 4 * 8224 at (0, 0)
//            (rounding and level shift of every pixel: T^T e0 = 1);
//   inverse  8 column then 8 row transposed butterflies;
//   output   pixel = high byte of saturate_u16(R), i.e. saturate_u8(R / 256).
#pragma once

#include <cuda_runtime.h>

#include "adct_internal.h"

namespace adct {
namespace {

constexpr int kMaxThreads = 128;  // with 3 CTAs per SM: up to 168 registers per thread
// output staging: 32 blocks of int16 coefficients (4096 bytes), or 32 packed
// blocks of r at a padded lane stride of up to 66 values (4224 bytes)
constexpr int kTileBytesOut = 4224;

__device__ __forceinline__ int32_t sext_lo16(uint32_t w) { return (int32_t)(int16_t)(w & 0xFFFFu); }
__device__ __forceinline__ int32_t sext_hi16(uint32_t w) { return ((int32_t)w) >> 16; }
__device__ __forceinline__ uint32_t pack16(int32_t lo, int32_t hi) {
  return __byte_perm((uint32_t)lo, (uint32_t)hi, 0x5410);
}
// One byte permute: selector 0xBBBB gives -1 for x < 0 and 0 otherwise (the
// sign of byte 3 replicated into every byte), 0x4444 gives 0 (a byte of the
// zero operand).
__device__ __forceinline__ int32_t sign_sel(int32_t x, uint32_t sel) {
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(0u), "r"(sel));
  return (int32_t)r;
}
// (sat_u16(a) << 16) | sat_u16(b)
__device__ __forceinline__ uint32_t cvt_pack_u16(int32_t a, int32_t b) {
  uint32_t d;
  asm("cvt.pack.sat.u16.s32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
// Four reconstructed values 4 (R + 8224) -> four saturated pixels, p0 in the
// lowest byte.  The dequantisation weights carry a factor 4, so that
// pixel = clamp((R + 8224) >> 6, 0, 255) is the high byte of
// clamp(4 (R + 8224), 0, 65535): two saturating packs of two values each and
// one byte permute, instead of a shift per value and two packs.
__device__ __forceinline__ uint32_t pixels4(int32_t r0, int32_t r1, int32_t r2, int32_t r3) {
  return __byte_perm(cvt_pack_u16(r1, r0), cvt_pack_u16(r3, r2), 0x7531);
}

// Bytes [0, n) of the little-endian 8-byte row r to p (8-byte aligned),
// 0 <= n <= 8: at most three stores (4, 2 and 1 bytes, each aligned).
__device__ __forceinline__ void store_prefix8(uint8_t* p, uint64_t r, int n) {
  if (n >= 8) {
    *(uint2*)p = make_uint2((uint32_t)r, (uint32_t)(r >> 32));
    return;
  }
  int off = 0;
  if (n & 4) {
    *(uint32_t*)p = (uint32_t)r;
    r >>= 32;
    off = 4;
  }
  if (n & 2) {
    *(uint16_t*)(p + off) = (uint16_t)r;
    r >>= 16;
    off += 2;
  }
  if (n & 1) p[off] = (uint8_t)r;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// 16-byte chunk c of block b inside a 32-block coefficient tile, XOR-swizzled
// so that 8 consecutive lanes touching one chunk each hit distinct banks.
__device__ __forceinline__ int swz(int b, int c) { return b * 128 + ((c ^ (b & 7)) << 4); }

// Reconstruction offset carried by S_00: 32 (rounding of R / 64) + 128 * 64
// (level shift); T^T e0 = 1 spreads it to every pixel of the block.
constexpr int32_t kDcBias = 4 * (32 + 128 * 64);  // times the factor 4 of the weights

template <int KIND>
struct KindTraits {
  static constexpr bool in_pix =
      (KIND == K_FORWARD || KIND == K_RT_FULL || KIND == K_RT_PIX || KIND == K_RT_COEF || KIND == K_RT_SSE);
  static constexpr bool quant =
      (KIND == K_QUANTISE || KIND == K_RT_FULL || KIND == K_RT_PIX || KIND == K_RT_COEF || KIND == K_RT_SSE);
  static constexpr bool write_coef = (KIND == K_FORWARD || KIND == K_QUANTISE || KIND == K_RT_FULL || KIND == K_RT_COEF);
  static constexpr bool inv = (KIND == K_INVERSE || KIND == K_RT_FULL || KIND == K_RT_PIX || KIND == K_RT_SSE);
  static constexpr bool sse = (KIND == K_RT_SSE);  // compare with the input instead of storing pixels
};

// Position of one lane's block: plane index and block coordinates (by, bx);
// plane < 0 past the end of the warp's chunk.  Addresses are recomputed from
// the plane descriptor (an L1 hit) when needed, which keeps the per-lane state
// of the two tiles in flight to six registers.
struct Pos {
  int plane;
  uint32_t by, bx;
};

__device__ __forceinline__ int64_t pix_off(const PlaneDesc* d, const Pos& q) {
  return (int64_t)(8 * q.by) * __ldg(&d->pitch) + 8 * q.bx;
}
__device__ __forceinline__ const uint8_t* src_of(const PlaneDesc* d) {
  return (const uint8_t*)__ldg((const unsigned long long*)&d->src);
}
__device__ __forceinline__ uint8_t* dst_of(const PlaneDesc* d) {
  return (uint8_t*)__ldg((const unsigned long long*)&d->dst);
}
// Coefficients of block (by, bx) of channel ch (always 0 for a planar plane).
__device__ __forceinline__ int16_t* coef_of(const PlaneDesc* d, const Pos& q, int ch = 0) {
  const int16_t* c = (const int16_t*)__ldg((const unsigned long long*)&d->coef);
  return (int16_t*)c + ch * __ldg(&d->cstride) + ((int64_t)q.by * __ldg(&d->cwb) + q.bx) * 64;
}
// Valid pixel columns and rows of a block (8 inside the image; 1..8 in the
// last block column / row of an image whose side is not a multiple of 8).
__device__ __forceinline__ int valid_cols(const PlaneDesc* d, const Pos& q) {
  return q.bx + 1 == (uint32_t)__ldg(&d->wb) ? (int)__ldg(&d->ew) : 8;
}
__device__ __forceinline__ int valid_rows(const PlaneDesc* d, const Pos& q) {
  return q.by + 1 == (uint32_t)__ldg(&d->hb) ? (int)__ldg(&d->eh) : 8;
}

// Lane stride, in int16, of the packed staging: r, padded by 2 when r is a
// multiple of 4 so that the 32 lanes' stores of one position t fall in 32
// distinct banks (an odd word stride, or an odd value stride).
__device__ __forceinline__ int zz_stride(int r) { return r + ((r & 3) == 0 ? 2 : 0); }

__device__ __forceinline__ int16_t* coef_of_zz(const PlaneDesc* d, const Pos& q, int r, int ch = 0) {
  const int16_t* c = (const int16_t*)__ldg((const unsigned long long*)&d->coef);
  return (int16_t*)c + ch * __ldg(&d->cstride) + ((int64_t)q.by * __ldg(&d->cwb) + q.bx) * r;
}

// Plane cursor of one lane: the flat index only grows (by 32 per tile), so the
// plane index only moves forward and (by, bx) advance incrementally; a
// division by the plane's width is needed only when a tile crosses a block
// row.  Offsets are 32-bit, relative to the warp's chunk start.
struct Cursor {
  int p;
  int32_t first, next_start;  // plane p spans [first, next_start) relative to the chunk start
  Pos last;                   // position returned by the previous call (plane < 0: none)

  template <bool MASK>
  __device__ __forceinline__ Pos locate(const PlaneDesc* __restrict__ planes, const int64_t* __restrict__ starts,
                                        int64_t begin, int32_t r, int32_t rend) {
    Pos q;
    if (r >= rend) {
      q.plane = -1; q.by = 0; q.bx = 0;
      last = q;
      return q;
    }
    bool moved = false;
    if (r >= next_start) {
      do {
        ++p;
        next_start = (int32_t)min(__ldg(starts + p + 1) - begin, (int64_t)0x7fffffff);
      } while (r >= next_start);
      first = (int32_t)(__ldg(starts + p) - begin);
      moved = true;
    }
    const uint32_t wb = (uint32_t)__ldg(&planes[p].wb);
    if (!moved && last.plane == p && last.bx + 32 < wb) {  // same block row, 32 blocks further
      q = last;
      q.bx += 32;
    } else {
      const uint32_t f = (uint32_t)(r - first);
      q.plane = p;
      q.by = f / wb;
      q.bx = f - q.by * wb;
    }
    last = q;
    // MASK: a descriptor whose last block column belongs to another launch
    // (the interior of an image with edge blocks, marked ew = 0: its flat rows
    // span the whole coefficient row so that tiles stay aligned) skips it.
    if (MASK && q.bx + 1 == wb && __ldg(&planes[p].ew) == 0) q.plane = -1;
    return q;
  }
};

// One 8x8 block per lane: a warp walks its chunk in tiles of 32 blocks.  (Two
// blocks per lane measured slower: the instruction count per block stays the
// same and the shared memory per CTA doubles.)
constexpr int kTile = 32;

// Marker zone of the packed zonal layout with r = 64: every coefficient is
// kept and stored in zig-zag order, 128 bytes per block like the dense
// layout, so these kernels stage and read coefficients as the dense ones do
// (16-byte chunks, 512-byte warp copies), with the zig-zag order a renaming
// of registers.
constexpr int kZoneZZ64 = 15;

// Input stages per warp: while tile i is computed the copies of tiles
// i + 1 .. i + stages - 1 are in flight.  Two stages measured best: a third
// stage for pixel input (4 KB in flight per warp) made the kernels with the
// least arithmetic per block slower by up to 20 % at the same occupancy.
//
// NCH > 1 (interleaved images): a tile is 32 pixel positions of NCH channels;
// its input stage holds the 8 rows of 32 x 8 NCH interleaved bytes, rewritten
// in place as NCH planar tiles of 2 KB; each channel's reconstruction goes back
// into its planar tile before the rows are re-interleaved and stored.  The
// inverse from coefficients uses the stage only for the reconstruction.
#ifndef ADCT_DEEP_ZONE
#define ADCT_DEEP_ZONE -1  // zonal kernels of zones up to this one get ADCT_DEEP_STAGES input stages
#endif
#ifndef ADCT_DEEP_STAGES
#define ADCT_DEEP_STAGES 2
#endif
template <int KIND, int NCH = 1, int ZS = 14>
struct SmemPlan {
  static constexpr int stages = (KindTraits<KIND>::in_pix && NCH == 1 && ZS <= ADCT_DEEP_ZONE) ? ADCT_DEEP_STAGES : 2;
  static constexpr int in_stage =
      (KindTraits<KIND>::in_pix || NCH > 1) ? 2048 * NCH : 4096;  // one 32-block (or 32-position) tile of input
  static constexpr int out_stage = KindTraits<KIND>::write_coef ? kTileBytesOut : 0;
  static constexpr int warp = stages * in_stage + out_stage;
};

// Bytes p0..p3 of the byte sequence held in w (byte p is byte p & 3 of
// w[p >> 2]) as one word, p0 lowest, with one byte permute per distinct
// source word after the second (1 to 3 permutes: 2 for the 4 bytes of one
// channel of a 3-channel span, against 3 for pairwise gathering, which took
// the interleaved round trip from 404 us to 395 us).  Called with constant
// positions inside unrolled loops, so all the selection below folds away.
__device__ __forceinline__ uint32_t gather4(const uint32_t* w, int p0, int p1, int p2, int p3) {
  const int x0 = p0 >> 2, x1 = p1 >> 2, x2 = p2 >> 2, x3 = p3 >> 2;
  // distinct source words A, B, C, D in order of first use (-1: none)
  const int A = x0;
  const int B = x1 != A ? x1 : x2 != A ? x2 : x3 != A ? x3 : -1;
  const int C = (x2 != A && x2 != B) ? x2 : (x3 != A && x3 != B) ? x3 : -1;
  const int D = (x3 != A && x3 != B && x3 != C) ? x3 : -1;
  // first permute: bytes of A (selector b) and B (4 + b)
  auto s1 = [&](int x, int p) { return (uint32_t)(x == A ? (p & 3) : x == B ? 4 + (p & 3) : 0); };
  uint32_t r = __byte_perm(w[A], w[B < 0 ? A : B], s1(x0, p0) | s1(x1, p1) << 4 | s1(x2, p2) << 8 | s1(x3, p3) << 12);
  // then one permute per further word: keep byte t, or take byte b of it
  if (C >= 0) {
    auto s2 = [&](int x, int p, int t) { return (uint32_t)(x == C ? 4 + (p & 3) : t); };
    r = __byte_perm(r, w[C], s2(x0, p0, 0) | s2(x1, p1, 1) << 4 | s2(x2, p2, 2) << 8 | s2(x3, p3, 3) << 12);
  }
  if (D >= 0) {
    auto s3 = [&](int x, int p, int t) { return (uint32_t)(x == D ? 4 + (p & 3) : t); };
    r = __byte_perm(r, w[D], s3(x0, p0, 0) | s3(x1, p1, 1) << 4 | s3(x2, p2, 2) << 8 | s3(x3, p3, 3) << 12);
  }
  return r;
}

// Interleaved tiles.  The input stage of a tile of 32 pixel positions holds, for
// row i, lane l's 8 NCH interleaved bytes at (i * 32 + l) * 8 NCH (byte b of a
// lane's row span is pixel b / NCH, channel b % NCH).  deinterleave_tile
// rewrites it in place as NCH planar tiles: channel c's row i of lane l's
// block at c * 2048 + (i * 32 + l) * 8, the layout of a planar tile, so the
// blocks then run the planar code.
template <int NCH>
__device__ __forceinline__ void deinterleave_tile(uint8_t* stage, int lane) {
  uint32_t w[8][2 * NCH];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const uint2* sp = (const uint2*)(stage + (i * 32 + lane) * 8 * NCH);
#pragma unroll
    for (int k = 0; k < NCH; ++k) {
      const uint2 u = sp[k];
      w[i][2 * k] = u.x;
      w[i][2 * k + 1] = u.y;
    }
  }
  __syncwarp();  // every lane has read its spans before any planar row overwrites them
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      const uint32_t a = gather4(w[i], c, c + NCH, c + 2 * NCH, c + 3 * NCH);
      const uint32_t b = gather4(w[i], c + 4 * NCH, c + 5 * NCH, c + 6 * NCH, c + 7 * NCH);
      ((uint2*)(stage + c * 2048))[i * 32 + lane] = make_uint2(a, b);
    }
}

// Byte selectors that take channel c's bytes out of an interleaved row span
// (byte b of the span is pixel b / NCH, channel b % NCH): they depend on c
// only, so one channel loop serves every channel.  NCH = 3: pixels 0-3 of
// channel c are span bytes c, c + 3, c + 6, c + 9 in words 0-2, gathered by
// one permute of words 0 and 1 (selector a; its third byte is overwritten
// when c = 2) and one with word 2 (selector b); pixels 4-7 the same from words
// 3-5.  NCH = 4: pixel j of channel c is byte c of word j; a takes it from
// two words at once and b joins two such pairs.
struct ChanSel {
  uint32_t a, b;
};
template <int NCH>
__device__ __forceinline__ ChanSel chan_sel(int c) {
  if (NCH == 3) return {0x0630u + 0x0111u * (uint32_t)c, c == 2 ? 0x7410u : 0x5210u + 0x1000u * (uint32_t)c};
  return {0x40u + 0x11u * (uint32_t)c, 0x5410u};
}
// Channel c's 8 bytes of one row (span words w[0 .. 2 NCH)) as pixels 0-3, 4-7.
template <int NCH>
__device__ __forceinline__ uint2 chan_row(const uint32_t* w, ChanSel k) {
  if (NCH == 3)
    return make_uint2(__byte_perm(__byte_perm(w[0], w[1], k.a), w[2], k.b),
                      __byte_perm(__byte_perm(w[3], w[4], k.a), w[5], k.b));
  return make_uint2(__byte_perm(__byte_perm(w[0], w[1], k.a), __byte_perm(w[2], w[3], k.a), k.b),
                    __byte_perm(__byte_perm(w[4], w[5], k.a), __byte_perm(w[6], w[7], k.a), k.b));
}

// Edge blocks: byte j of each row becomes byte min(j, vc - 1), one byte
// permute per 4 bytes (selector nibble j = min(j, vc - 1); the identity for
// full blocks).
__device__ __forceinline__ uint32_t edge_fill_sel(int vc) {
  const uint32_t c = (uint32_t)vc - 1u;
  const uint32_t hi = c >= 7u ? 0u : 0xFFFFFFFFu << (4u * (c + 1u));  // nibbles above c
  return (0x76543210u & ~hi) | (c * 0x11111111u & hi);
}

// Raw pixels of row w (bytes 0-7) into v[8 i .. 8 i + 7], after the edge fill.
template <bool EDGE>
__device__ __forceinline__ void unpack_row(uint2 w, uint32_t sel, int i, int32_t (&v)[64]) {
  if (EDGE) {
    const uint2 raw = w;
    w.x = __byte_perm(raw.x, raw.y, sel & 0xFFFFu);
    w.y = __byte_perm(raw.x, raw.y, sel >> 16);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    v[8 * i + j] = (int32_t)__byte_perm(w.x, 0u, 0x4440 | j);
    v[8 * i + 4 + j] = (int32_t)__byte_perm(w.y, 0u, 0x4440 | j);
  }
}

// Interleaved input read per channel: channel ch of lane's block straight from
// the tile's interleaved stage (its 8 NCH-byte row spans), unpacked into v.
template <int NCH, bool EDGE>
__device__ __forceinline__ void read_interleaved(const uint8_t* __restrict__ in, const PlaneDesc* __restrict__ planes,
                                                 const Pos& pos, int ch, int lane, int32_t (&v)[64]) {
  const ChanSel k = chan_sel<NCH>(ch);
  const uint32_t sel = EDGE ? edge_fill_sel(valid_cols(planes + pos.plane, pos)) : 0x76543210u;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const uint2* sp = (const uint2*)(in + (i * 32 + lane) * 8 * NCH);
    uint32_t w[2 * NCH];
#pragma unroll
    for (int t = 0; t < NCH; ++t) {
      const uint2 u = sp[t];
      w[2 * t] = u.x;
      w[2 * t + 1] = u.y;
    }
    unpack_row<EDGE>(chan_row<NCH>(w, k), sel, i, v);
  }
}

// Reconstructed planar tile of one channel in lane-major order (the
// per-channel interleaved pipeline): lane l's rows 2k and 2k + 1 form the
// 16-byte chunk at l * 64 + ((k ^ ((l >> 1) & 3)) << 4), so that the 8 lanes
// of each quarter warp store or load one chunk each in 8 distinct 16-byte
// bank groups.
__device__ __forceinline__ int recon_chunk(int lane, int k) { return lane * 64 + ((k ^ ((lane >> 1) & 3)) << 4); }

// Arithmetic of one 8x8 block: read its input from the input stage, quantise,
// stage or store q, dequantise, invert and store the pixels.
//
// NCH > 1: channel ch of an interleaved image, whose planar tile (made by
// deinterleave_tile) starts at ch * 2048 in the stage; the reconstructed rows
// go back to the same place.
//
// EDGE: the launch may contain blocks on the right or bottom edge of an image
// whose side is not a multiple of 8 (compiled out of the launches that have
// none).
//
// PRE: v already holds the block's raw pixels (read_interleaved); its
// reconstruction goes to channel ch's planar tile in `recon` instead of `in`.
template <int KIND, int QMODE, bool EVENQ, int ZS, int NCH, bool EDGE, bool PRE = false>
__device__ __forceinline__ uint32_t block_step(int32_t (&v)[64], uint8_t* __restrict__ in, uint8_t* recon,
                                               uint8_t* __restrict__ stage_out, const PlaneDesc* __restrict__ planes,
                                               const Pos& pos, int ch, int stage_coef, const QuantParams& qp,
                                               int lane) {
  using KT = KindTraits<KIND>;
  // With a zonal quantiser every coefficient beyond anti-diagonal ZS is zero
  // (the kept r fit in diagonals 0..ZS): known at compile time, so the forward
  // outputs there are never computed and the inverse skips their terms.
  constexpr bool kZonal = (QMODE == QM_ZONAL || QMODE == QM_ZONAL_ZZ || QMODE == QM_STEP_ZONAL);
  constexpr int kZoneN = zone_count(ZS);
  if (pos.plane < 0) return 0;
  const PlaneDesc* d = planes + pos.plane;
  // valid columns / rows (edge blocks: the rest replicates the last valid one;
  // the input stage already holds the last valid row in place of the others)
  const int vc = EDGE ? valid_cols(d, pos) : 8, vr = EDGE ? valid_rows(d, pos) : 8;
  if (KT::in_pix) {
    if (!PRE) {
      const uint2* st = (const uint2*)(in + (NCH > 1 ? ch * 2048 : 0));
      const uint32_t sel = EDGE ? edge_fill_sel(vc) : 0x76543210u;
#pragma unroll
      for (int i = 0; i < 8; ++i) unpack_row<EDGE>(st[i * 32 + lane], sel, i, v);
    }
    fwd2d(v);  // Z + 8192 e0 e0^T (raw pixels; the level shift lives in the constants)
  } else if (QMODE == QM_ZONAL_ZZ && ZS != kZoneZZ64) {
    // packed input: the first r zig-zag coefficients of this block
    constexpr ZigZag zz = make_zigzag();
    const int16_t* c = coef_of_zz(d, pos, qp.r, ch);
#pragma unroll
    for (int k = 0; k < 64; ++k) v[k] = 0;
#pragma unroll
    for (int t = 0; t < kZoneN; ++t) v[zz.pos[t]] = (t < qp.r) ? (int32_t)__ldg(c + t) : 0;
  } else if (NCH > 1) {
    // inverse into an interleaved image: this channel's block straight from memory
    const int4* cp = (const int4*)coef_of(d, pos, ch);
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int4 u = __ldg(cp + t);
      v[8 * t + 0] = sext_lo16(u.x); v[8 * t + 1] = sext_hi16(u.x);
      v[8 * t + 2] = sext_lo16(u.y); v[8 * t + 3] = sext_hi16(u.y);
      v[8 * t + 4] = sext_lo16(u.z); v[8 * t + 5] = sext_hi16(u.z);
      v[8 * t + 6] = sext_lo16(u.w); v[8 * t + 7] = sext_hi16(u.w);
    }
  } else {
    // the staged coefficient tile (packed r = 64: chunk t holds zig-zag positions 8 t .. 8 t + 7)
    constexpr ZigZag zz = make_zigzag();
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int4 u = *(const int4*)(in + swz(lane, t));
      const int32_t e[8] = {sext_lo16(u.x), sext_hi16(u.x), sext_lo16(u.y), sext_hi16(u.y),
                            sext_lo16(u.z), sext_hi16(u.z), sext_lo16(u.w), sext_hi16(u.w)};
#pragma unroll
      for (int m = 0; m < 8; ++m) v[ZS == kZoneZZ64 ? zz.pos[8 * t + m] : 8 * t + m] = e[m];
    }
  }

  // ---- packed zonal output: the first r zig-zag coefficients, staged per lane ----
  if (QMODE == QM_ZONAL_ZZ && KT::write_coef && ZS == kZoneZZ64) {
    // r = 64: eight 16-byte chunks of eight zig-zag positions each, staged
    // like dense rows (or stored directly)
    constexpr ZigZag zz = make_zigzag();
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      int32_t zq[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int k = zz.pos[8 * t + m];
        zq[m] = v[k] + ((KT::in_pix && k == 0) ? -8192 : 0);  // the true coefficient
      }
      const int4 u = make_int4((int)pack16(zq[0], zq[1]), (int)pack16(zq[2], zq[3]), (int)pack16(zq[4], zq[5]),
                               (int)pack16(zq[6], zq[7]));
      if (stage_coef) *(int4*)(stage_out + swz(lane, t)) = u;
      else __stcs((int4*)coef_of(d, pos, ch) + t, u);
    }
  } else if (QMODE == QM_ZONAL_ZZ && KT::write_coef) {
    constexpr ZigZag zz = make_zigzag();
    int16_t* out = stage_coef ? (int16_t*)stage_out + lane * zz_stride(qp.r) : coef_of_zz(d, pos, qp.r, ch);
#pragma unroll
    for (int t = 0; t < kZoneN; ++t) {
      const int k = zz.pos[t];
      const int32_t zq = v[k] + ((KT::in_pix && k == 0) ? -8192 : 0);  // the true coefficient
      if (t < qp.r) out[t] = (int16_t)zq;
    }
  }

  // ---- quantise (q, stored row by row) and dequantise in place (v <- S) ----
  // S = q * w with w = Q 2^(6 - a_i - a_j) (D^2 merged), plus kDcBias at
  // (0, 0).  For STEP it is formed from m directly (S = m * w + kw, kw =
  // -K * w (+ kDcBias)), independent of the q = m - K that goes to memory.
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int32_t q[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = 8 * i + j;
      const int32_t bias = (k == 0) ? kDcBias : 0;
      const int32_t z = v[k];  // raw: Z + 8192 at (0, 0) when the input was pixels
      // T (X - 128) T^T = T X T^T - 8192 e0 e0^T  (T 1 = 8 e0)
      const int32_t zoff = (KT::in_pix && k == 0) ? -8192 : 0;
      if (kZonal && i + j > ZS) {  // outside the zone (k = 0 never is)
        q[j] = 0;
        v[k] = 0;
      } else if (KIND == K_INVERSE) {
        q[j] = z;
        v[k] = (int32_t)((uint32_t)z * (uint32_t)qp.w[k] + (uint32_t)bias);
      } else if (QMODE == QM_ZONAL_ZZ) {
        v[k] = (int32_t)((uint32_t)((z + zoff) & qp.keep[k]) * (uint32_t)qp.w[k] + (uint32_t)bias);
      } else if (QMODE == QM_STEP || QMODE == QM_STEP_ZONAL) {
        int32_t n = z + qp.c[k];
        if (EVENQ) n += sign_sel(z + zoff, qp.ssel[k]);
        const uint32_t m = __umulhi((uint32_t)n, qp.magic[k]);
        int32_t qq = (int32_t)m - qp.K[k];
        if (QMODE == QM_STEP_ZONAL) qq &= qp.keep[k];
        q[j] = qq;
        if (KT::inv)
          v[k] = (QMODE == QM_STEP_ZONAL) ? (int32_t)((uint32_t)qq * (uint32_t)qp.w[k] + (uint32_t)bias)
                                          : (int32_t)(m * (uint32_t)qp.w[k] + (uint32_t)qp.kw[k]);
      } else {
        int32_t qq = z + zoff;  // the true coefficient
        if (QMODE == QM_ZONAL) qq &= qp.keep[k];
        q[j] = qq;
        if (KT::inv) v[k] = (int32_t)((uint32_t)qq * (uint32_t)qp.w[k] + (uint32_t)bias);
      }
    }
    if (KT::write_coef && QMODE != QM_ZONAL_ZZ) {
      int4 u;
      u.x = (int)pack16(q[0], q[1]);
      u.y = (int)pack16(q[2], q[3]);
      u.z = (int)pack16(q[4], q[5]);
      u.w = (int)pack16(q[6], q[7]);
      if (stage_coef) *(int4*)(stage_out + swz(lane, i)) = u;
      else __stcs((int4*)coef_of(d, pos, ch) + i, u);
    }
  }

  // ---- inverse (8 column, then 8 row transposed butterflies) and output ----
  // Blocks on the right or bottom edge of an image whose side is not a
  // multiple of 8 store (and compare) only their valid rows and columns.
  uint32_t err = 0;
  if (KT::inv) {
    inv2d(v);
    if (KT::sse) {
      // squared error against the input rows, still in the input stage
      const uint2* st = (const uint2*)(in + (NCH > 1 ? ch * 2048 : 0));
      const uint32_t m0 = vc >= 4 ? 0xffffffffu : (1u << (8 * vc)) - 1u;
      const uint32_t m1 = vc >= 8 ? 0xffffffffu : vc <= 4 ? 0u : (1u << (8 * (vc - 4))) - 1u;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const uint2 x = st[i * 32 + lane];
        const uint32_t e0 = __vabsdiffu4(pixels4(v[8 * i + 0], v[8 * i + 1], v[8 * i + 2], v[8 * i + 3]), x.x) & m0;
        const uint32_t e1 = __vabsdiffu4(pixels4(v[8 * i + 4], v[8 * i + 5], v[8 * i + 6], v[8 * i + 7]), x.y) & m1;
        if (i < vr) {
          err = __dp4a(e0, e0, err);
          err = __dp4a(e1, e1, err);
        }
      }
    } else if (NCH == 1) {
      const int64_t pitch = __ldg(&d->pitch);
      uint8_t* o = dst_of(d) + (int64_t)(8 * pos.by) * pitch + 8 * pos.bx;
      uint2 w[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        w[i].x = pixels4(v[8 * i + 0], v[8 * i + 1], v[8 * i + 2], v[8 * i + 3]);
        w[i].y = pixels4(v[8 * i + 4], v[8 * i + 5], v[8 * i + 6], v[8 * i + 7]);
      }
      if (!EDGE || ((vc == 8) & (vr == 8))) {  // one branch per block, not per row
#pragma unroll
        for (int i = 0; i < 8; ++i) __stcs((uint2*)(o + i * pitch), w[i]);
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (i < vr) store_prefix8(o + i * pitch, ((uint64_t)w[i].y << 32) | w[i].x, vc);
      }
    } else {
      // interleaved: the reconstructed rows back into this channel's planar
      // tile (its input is consumed), interleaved and stored once every
      // channel is done
      if (PRE) {
        // lane-major tile (recon_chunk): rows 2k and 2k + 1 in one 16-byte store
        uint8_t* pl = recon + ch * 2048;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int i = 2 * k;
          *(uint4*)(pl + recon_chunk(lane, k)) =
              make_uint4(pixels4(v[8 * i + 0], v[8 * i + 1], v[8 * i + 2], v[8 * i + 3]),
                         pixels4(v[8 * i + 4], v[8 * i + 5], v[8 * i + 6], v[8 * i + 7]),
                         pixels4(v[8 * i + 8], v[8 * i + 9], v[8 * i + 10], v[8 * i + 11]),
                         pixels4(v[8 * i + 12], v[8 * i + 13], v[8 * i + 14], v[8 * i + 15]));
        }
      } else {
        uint2* pl = (uint2*)(in + ch * 2048);
#pragma unroll
        for (int i = 0; i < 8; ++i)
          pl[i * 32 + lane] = make_uint2(pixels4(v[8 * i + 0], v[8 * i + 1], v[8 * i + 2], v[8 * i + 3]),
                                         pixels4(v[8 * i + 4], v[8 * i + 5], v[8 * i + 6], v[8 * i + 7]));
      }
    }
  }
  return err;
}

// Store the reconstructed interleaved pixels of a 32-position tile from its
// NCH planar tiles: each row's channel words are interleaved in registers
// (byte b of the span is byte (b / NCH) & 3 of channel b % NCH's word
// (b / NCH) / 4) and written with NCH 8-byte stores, so the warp covers 256 NCH
// contiguous bytes per row; on the image's right edge only the valid bytes
// of each 8-byte part (store_prefix8).  LM: the planar tiles are in the
// lane-major order of recon_chunk and are read two rows per 16-byte load.
template <int NCH, bool EDGE, bool LM = false>
__device__ __forceinline__ void write_pixels_interleaved(const uint8_t* __restrict__ stage,
                                                        const PlaneDesc* __restrict__ planes, const Pos& pos,
                                                        int lane) {
  if (pos.plane < 0) return;
  const PlaneDesc* d = planes + pos.plane;
  const int64_t pitch = __ldg(&d->pitch);
  uint8_t* o = dst_of(d) + (int64_t)(8 * pos.by) * pitch + 8 * NCH * pos.bx;
  const int vc = EDGE ? valid_cols(d, pos) : 8, vr = EDGE ? valid_rows(d, pos) : 8;
  uint4 pair[NCH];  // LM: channel c's rows 2k and 2k + 1
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    if (i >= vr) break;
    uint32_t q[2 * NCH];  // channel c's pixels 0-3 and 4-7 at q[2c], q[2c + 1]
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      if (LM) {
        if ((i & 1) == 0) pair[c] = *(const uint4*)(stage + c * 2048 + recon_chunk(lane, i >> 1));
        q[2 * c] = (i & 1) ? pair[c].z : pair[c].x;
        q[2 * c + 1] = (i & 1) ? pair[c].w : pair[c].y;
      } else {
        const uint2 u = ((const uint2*)(stage + c * 2048))[i * 32 + lane];
        q[2 * c] = u.x;
        q[2 * c + 1] = u.y;
      }
    }
    uint32_t span[2 * NCH];
#pragma unroll
    for (int m = 0; m < 2 * NCH; ++m) {
      int pos4[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int b = 4 * m + t, px = b / NCH, c = b % NCH;
        pos4[t] = 4 * (2 * c + (px >> 2)) + (px & 3);
      }
      span[m] = gather4(q, pos4[0], pos4[1], pos4[2], pos4[3]);
    }
    if (vc == 8) {
#pragma unroll
      for (int k = 0; k < NCH; ++k) __stcs((uint2*)(o + i * pitch) + k, make_uint2(span[2 * k], span[2 * k + 1]));
    } else {
#pragma unroll
      for (int k = 0; k < NCH; ++k)  // valid bytes of each 8-byte part
        store_prefix8(o + i * pitch + 8 * k, ((uint64_t)span[2 * k + 1] << 32) | span[2 * k],
                      max(0, NCH * vc - 8 * k));
    }
  }
}

// Write a staged 32-block half-tile of coefficients back with 512-byte warp
// stores when the active lanes' blocks are consecutive in memory (one
// contiguous range: the usual case; not when the tile crosses a plane, or a
// block row of a descriptor narrower than its coefficient rows).  MASKED
// (interiors with a masked column): inactive lanes may sit anywhere in the
// warp, not only past the end of the chunk; their blocks are left untouched.
template <bool MASKED>
__device__ __forceinline__ void write_back(const uint8_t* __restrict__ stage_out, const PlaneDesc* __restrict__ planes,
                                          const Pos& pos, int lane, int ch) {
  const bool active = pos.plane >= 0;
  const unsigned act = __ballot_sync(0xffffffffu, active);
  if (MASKED && act == 0) return;
  int16_t* mine = active ? coef_of(planes + pos.plane, pos, ch) : nullptr;
  const int f = MASKED ? __ffs(act) - 1 : 0;  // first active lane
  int16_t* const base = (int16_t*)__shfl_sync(0xffffffffu, (unsigned long long)mine, f) - 64 * f;
  // Instruction k moves bytes [512 k, 512 k + 512) of the half-tile: lane l
  // takes 16-byte chunk (l & 7) of block 4 k + (l >> 3), i.e. byte 512 k + 16 l;
  // in shared memory that chunk sits at one of two lane-specific offsets (the
  // swizzle depends on k only through k & 1) plus 512 k.
  const int pb = lane >> 3, pc = lane & 7;
  const uint32_t rd0 = pb * 128 + ((pc ^ pb) << 4), rd1 = pb * 128 + ((pc ^ (pb + 4)) << 4);
  if (__all_sync(0xffffffffu, !active || mine == base + 64 * lane)) {
    int4* gp = (int4*)base + lane;
    const int nact = __popc(act);  // without MASKED the active lanes are a prefix of the warp
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const bool wr = MASKED ? ((act >> (4 * k + pb)) & 1u) != 0 : 4 * k + pb < nact;
      if (wr) __stcs(gp + 32 * k, *(const int4*)(stage_out + 512 * k + ((k & 1) ? rd1 : rd0)));
    }
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int b = 4 * k + pb;
      int16_t* cb = (int16_t*)__shfl_sync(0xffffffffu, (unsigned long long)mine, b);
      if (cb) __stcs((int4*)cb + pc, *(const int4*)(stage_out + 512 * k + ((k & 1) ? rd1 : rd0)));
    }
  }
}

// Write a staged 32-block half-tile of packed zonal coefficients (r int16 per
// block, r <= NMAX; lane l's at [l sp, l sp + r), sp = zz_stride(r)) back to
// memory.  When the active lanes' blocks are consecutive in memory the
// half-tile is one contiguous range of nact r values, written as 4-byte words when aligned (all
// loads of the warp issued before its stores); otherwise each lane writes its
// own r.  With padding (r a multiple of 4) value e of the range sits at
// e + 2 (e / r) in the staging, so word w at w + w / (r / 2); the division is a
// multiply by mh = ceil(2^20 / (r / 2)), exact for w < 2^10.
template <int NMAX, bool MASKED>
__device__ __forceinline__ void write_back_zz(const uint8_t* __restrict__ stage_out,
                                             const PlaneDesc* __restrict__ planes, const Pos& pos, int lane, int r,
                                             uint32_t mh, int ch) {
  const bool active = pos.plane >= 0;
  const unsigned act = __ballot_sync(0xffffffffu, active);
  int16_t* mine = active ? coef_of_zz(planes + pos.plane, pos, r, ch) : nullptr;
  const int16_t* st16 = (const int16_t*)stage_out;
  const bool padded = (r & 3) == 0;
  int16_t* const base = (int16_t*)__shfl_sync(0xffffffffu, (unsigned long long)mine, 0);
  const bool prefix = !MASKED || (act & (act + 1u)) == 0;  // active lanes are a prefix of the warp
  if (prefix && __all_sync(0xffffffffu, !active || mine == base + r * lane)) {
    const int n = __popc(act) * r;  // values to write
    if (((uintptr_t)base & 3) == 0 && (n & 1) == 0) {
      constexpr int kWords = (NMAX + 1) / 2;  // words per lane at most (32 r / 2 / 32)
      uint32_t* gw = (uint32_t*)base;
      const uint32_t* sw = (const uint32_t*)st16;
      const int nw = n / 2;
      uint32_t val[kWords];
#pragma unroll
      for (int j = 0; j < kWords; ++j) {
        const int w = lane + 32 * j;
        if (w < nw) val[j] = sw[padded ? w + ((w * mh) >> 20) : w];
      }
#pragma unroll
      for (int j = 0; j < kWords; ++j) {
        const int w = lane + 32 * j;
        if (w < nw) __stcs(gw + w, val[j]);
      }
    } else {
      for (int e = lane; e < n; e += 32) base[e] = st16[padded ? e + 2 * (e / r) : e];
    }
  } else if (active) {
    const int sp = zz_stride(r);
    for (int t = 0; t < r; ++t) mine[t] = st16[lane * sp + t];
  }
}

// Three CTAs of 4 warps per SM (up to 168 registers), four for the packed
// zonal kernels of zones 6-8 (128 registers, no spills): r = 25 on 256 x
// 1080x1920 takes 275.6 us against 298 us at 158 registers and 3 CTAs per
// SM; zone 5 (113 registers) and the others are unchanged or slower at 128.
template <int QMODE, int ZS>
constexpr int codec_min_ctas() { return (QMODE == QM_ZONAL_ZZ && ZS >= 6 && ZS <= 8) ? 4 : 3; }

template <int KIND, int QMODE, bool EVENQ, int ZS, int NCH = 1, int EDGE = kEdgeNone>
__global__ void __launch_bounds__(kMaxThreads, codec_min_ctas<QMODE, ZS>())
k_codec(const PlaneDesc* __restrict__ planes, const int64_t* __restrict__ starts, int32_t nplanes, int64_t total,
        int64_t chunk, int stage_coef, unsigned long long* __restrict__ sse, unsigned int* __restrict__ fault,
        const QuantParams qp) {
  using KT = KindTraits<KIND>;
  using SP = SmemPlan<KIND, NCH, ZS>;
  constexpr int S = SP::stages;
  constexpr bool EB = EDGE == kEdgeBlocks;      // edge blocks: clamped copies, column fill, partial stores
  constexpr bool MASKED = EDGE == kEdgeMasked;  // interiors whose last block column is masked
  // Interleaved pixel input of the step-quantised kinds that reconstruct
  // pixels (not the squared-error kind): one input stage, read per channel
  // (read_interleaved) and refilled with the next tile once the last channel
  // has read it; the second stage holds the channels' reconstructed planar
  // tiles.  The other kinds and modes keep the in-place de-interleave:
  // issuing the next tile's copies while a block is live in registers made
  // them spill.
  constexpr bool kLazy = NCH > 1 && KT::in_pix && KT::inv && !KT::sse && (QMODE == QM_STEP || QMODE == QM_STEP_ZONAL);
  static_assert(!kLazy || S == 2, "the interleaved pipeline uses two stages");
  extern __shared__ __align__(128) uint8_t smem[];
  const int lane = threadIdx.x & 31;
  uint8_t* wsm = smem + (threadIdx.x >> 5) * SP::warp;
  uint8_t* stage_out = wsm + S * SP::in_stage;

  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t begin = gwarp * chunk;
  // Programmatic dependent launch.  The interiors of split images (MASKED)
  // let the launch of their images' edge strips, which follows them with the
  // programmatic serialisation attribute, start at once: its CTAs take SM
  // slots as this grid's CTAs retire.  The edge kernel (EB) waits for the
  // grid before it, if any, before it exits, so that its completion still
  // implies that grid's (later work on the stream sees both done); launched
  // without the attribute it has nothing to wait for.
  if (MASKED) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (begin >= total) {  // whole warp exits together
    if (EB) asm volatile("griddepcontrol.wait;" ::: "memory");
    return;
  }
  const int64_t end = min(total, begin + chunk);
  const int32_t rend = (int32_t)(end - begin);  // chunk length (< 2^31 blocks)

  Cursor cur;
  {
    int lo = 0, hi = nplanes;  // largest p with starts[p] <= begin
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(starts + mid) <= begin) lo = mid; else hi = mid;
    }
    cur.p = lo;
    cur.first = (int32_t)(__ldg(starts + lo) - begin);
    cur.next_start = (int32_t)min(__ldg(starts + lo + 1) - begin, (int64_t)0x7fffffff);
    cur.last.plane = -1;
    cur.last.by = cur.last.bx = 0;
  }

  // Checked builds (ADCT_CHECKED): a position outside its plane's blocks is
  // reported in the fault word and dropped (every address of a block derives
  // from its plane descriptor and (by, bx)); release builds return it as is.
  auto checked = [&](Pos q) {
#ifdef ADCT_CHECKED
    if (q.plane >= 0 && (q.plane >= nplanes || q.by >= (uint32_t)__ldg(&planes[q.plane].hb) ||
                         q.bx >= (uint32_t)__ldg(&planes[q.plane].wb))) {
      if (fault) atomicOr(fault, FAULT_POSITION);
      q.plane = -1;
    }
#endif
    return q;
  };

  // Issue the asynchronous input copies of one tile into stage st (lanes past
  // the end of the chunk copy nothing; the group is committed regardless).
  // Pixels: lane l's 8 NCH bytes of row i go to (i * 32 + l) * 8 NCH, so the
  // warp's copies of one row cover 256 NCH contiguous bytes.
  auto issue = [&](int st, const Pos& q) {
    const uint32_t sa = smem_addr(wsm + st * SP::in_stage);
    if (KT::in_pix && NCH > 1 && !EB) {
      // Interleaved tile without edge blocks: lane l copies 8-byte chunk
      // 32 k + l of every row of the tile (position (32 k + l) / NCH, part
      // (32 k + l) % NCH), taking that position's row address from its lane,
      // so each warp copy instruction reads 256 contiguous bytes when the
      // positions are consecutive (each lane copying its own 8 NCH bytes
      // touched 8 NCH partly used 32-byte sectors per instruction).  The
      // stage layout is the same.
      const uint8_t* mine = nullptr;
      int64_t mpitch = 0;
      if (q.plane >= 0) {
        const PlaneDesc* d = planes + q.plane;
        mpitch = __ldg(&d->pitch);
        mine = src_of(d) + (int64_t)(8 * q.by) * mpitch + 8 * NCH * q.bx;
#ifdef ADCT_CHECKED
        if (8 * NCH * ((int64_t)__ldg(&d->bx0) + q.bx) + 8 * NCH > mpitch) {  // a copy would pass the end of the row
          if (fault) atomicOr(fault, FAULT_ROW_BYTES);
          mine = nullptr;
        }
#endif
      }
#pragma unroll
      for (int k = 0; k < NCH; ++k) {
        const int c = 32 * k + lane, p = c / NCH, part = c - p * NCH;
        const uint8_t* b = (const uint8_t*)__shfl_sync(0xffffffffu, (unsigned long long)mine, p);
        const int64_t pt = __shfl_sync(0xffffffffu, mpitch, p);
        if (b) {
#pragma unroll
          for (int i = 0; i < 8; ++i) cp_async8(sa + (i * 32 * NCH + c) * 8, b + 8 * part + (int64_t)i * pt);
        }
      }
    } else if (KT::in_pix) {
      if (q.plane >= 0) {
        const PlaneDesc* d = planes + q.plane;
        const int64_t pitch = __ldg(&d->pitch);
        const uint8_t* src = src_of(d) + (int64_t)(8 * q.by) * pitch + 8 * NCH * q.bx;
        // Edge blocks copy the last valid row in place of the missing ones and
        // only the 8-byte chunks that hold valid pixels (they end at or
        // before ceil8(width * NCH) <= pitch, inside the row); the missing
        // columns are filled from the last valid one when the block is read.
        const int vc = EB ? valid_cols(d, q) : 8, vr = EB ? valid_rows(d, q) : 8;
        const int nchunk = EB ? (NCH * vc + 7) / 8 : NCH;
#ifdef ADCT_CHECKED
        if (8 * NCH * ((int64_t)__ldg(&d->bx0) + q.bx) + 8 * nchunk > pitch) {  // a copy would pass the end of the row
          if (fault) atomicOr(fault, FAULT_ROW_BYTES);
          cp_async_commit();
          return;
        }
#endif
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const uint8_t* row = src + (int64_t)(EB ? min(i, vr - 1) : i) * pitch;
#pragma unroll
          for (int k = 0; k < NCH; ++k)
            if (!EB || k < nchunk) cp_async8(sa + ((i * 32 + lane) * NCH + k) * 8, row + 8 * k);
        }
      }
    } else if ((QMODE != QM_ZONAL_ZZ || ZS == kZoneZZ64) && NCH == 1) {
      // Coefficients: lane copies 16-byte chunk c of block b (512 contiguous
      // bytes per warp instruction when the tile lies in one plane).
      const int16_t* mine = q.plane >= 0 ? coef_of(planes + q.plane, q) : nullptr;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int b = 4 * k + (lane >> 3), c = lane & 7;
        const int16_t* cb = (const int16_t*)__shfl_sync(0xffffffffu, (unsigned long long)mine, b);
        if (cb) cp_async16(sa + swz(b, c), cb + 8 * c);
      }
    }
    cp_async_commit();
  };

  // packed staging with padding: word w of a half-tile is in block w / (r / 2)
  const uint32_t zz_mh =
      (QMODE == QM_ZONAL_ZZ && qp.r >= 4) ? ((1u << 20) + (qp.r >> 1) - 1) / (uint32_t)(qp.r >> 1) : 0;
  // K_RT_SSE: this lane's error sums for the channels of descriptor acc_plane
  unsigned long long acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
  int acc_plane = -1;
  auto flush = [&]() {
    if (acc_plane < 0) return;
    const int pid = __ldg(&planes[acc_plane].plane_id);
    atomicAdd(sse + pid, acc0);
    if (NCH > 1) atomicAdd(sse + pid + 1, acc1);
    if (NCH > 2) atomicAdd(sse + pid + 2, acc2);
    if (NCH > 3) atomicAdd(sse + pid + 3, acc3);
    acc0 = acc1 = acc2 = acc3 = 0;
  };
  Pos ring[S - 1];  // positions of tiles i .. i + S - 2, whose copies are issued
#pragma unroll
  for (int k = 0; k < S - 1; ++k) {
    ring[k] = checked(cur.template locate<MASKED>(planes, starts, begin, kTile * k + lane, rend));
    issue(k, ring[k]);
  }
  int s = 0;  // stage of tile i
  for (int32_t base = 0; base < rend; base += kTile) {
    __syncwarp();  // every lane is done reading tile i - 1's stage, refilled now
    const Pos pl = checked(cur.template locate<MASKED>(planes, starts, begin, base + kTile * (S - 1) + lane, rend));
    if (!kLazy) {
      issue(s == 0 ? S - 1 : s - 1, pl);
      cp_async_wait<S - 1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();

    const Pos pc = ring[0];
    uint8_t* stage = wsm + s * SP::in_stage;
    uint8_t* recon = kLazy ? wsm + SP::in_stage : stage;  // reconstructed planar tiles
    if (NCH > 1 && KT::in_pix && !kLazy) {
      deinterleave_tile<NCH>(stage, lane);
      __syncwarp();
    }
    if (KT::sse && pc.plane >= 0 && pc.plane != acc_plane) {  // one atomic per lane and channel per plane visited
      flush();
      acc_plane = pc.plane;
    }
    auto channel = [&](int ch) {
      int32_t v[64];
      if (kLazy) {
        if (pc.plane >= 0) read_interleaved<NCH, EB>(stage, planes, pc, ch, lane, v);
        if (ch == NCH - 1) {  // every channel's input is read: the stage takes the next tile
          __syncwarp();
          issue(0, pl);
        }
      }
      const uint32_t e = block_step<KIND, QMODE, EVENQ, ZS, NCH, EB, kLazy>(v, stage, recon, stage_out, planes, pc,
                                                                            ch, stage_coef, qp, lane);
      if (KT::sse) {
        if (ch == 0) acc0 += e;
        else if (ch == 1) acc1 += e;
        else if (ch == 2) acc2 += e;
        else acc3 += e;
      }
      if (KT::write_coef && stage_coef) {
        __syncwarp();
        if (QMODE == QM_ZONAL_ZZ && ZS != kZoneZZ64)
          write_back_zz<zone_count(ZS), MASKED>(stage_out, planes, pc, lane, qp.r, zz_mh, ch);
        else write_back<MASKED>(stage_out, planes, pc, lane, ch);
        __syncwarp();
      }
    };
    if (NCH == 1) {
      channel(0);
    } else {
#pragma unroll 1
      for (int ch = 0; ch < NCH; ++ch) channel(ch);
    }
    if (NCH > 1 && KT::inv && !KT::sse) write_pixels_interleaved<NCH, EB, kLazy>(recon, planes, pc, lane);
#pragma unroll
    for (int k = 0; k + 1 < S - 1; ++k) ring[k] = ring[k + 1];
    ring[S - 2] = pl;
    if (!kLazy && ++s == S) s = 0;
  }
  if (KT::sse) flush();
  cp_async_wait<0>();
  if (EB) asm volatile("griddepcontrol.wait;" ::: "memory");
}

// The kernels of one zone ZS for the zonal kinds that have them; nullptr otherwise.
template <int ZS>
KernelFn pick_zone(int kind, int qmode) {
  const bool zz = qmode == QM_ZONAL_ZZ;
  if (qmode != QM_ZONAL && !zz) return nullptr;
  switch (kind) {
    case K_RT_FULL: return zz ? k_codec<K_RT_FULL, QM_ZONAL_ZZ, false, ZS> : k_codec<K_RT_FULL, QM_ZONAL, false, ZS>;
    case K_RT_COEF: return zz ? k_codec<K_RT_COEF, QM_ZONAL_ZZ, false, ZS> : k_codec<K_RT_COEF, QM_ZONAL, false, ZS>;
    case K_RT_PIX: return k_codec<K_RT_PIX, QM_ZONAL, false, ZS>;
    case K_RT_SSE: return k_codec<K_RT_SSE, QM_ZONAL, false, ZS>;
    case K_INVERSE: return zz ? k_codec<K_INVERSE, QM_ZONAL_ZZ, false, ZS> : nullptr;
    default: return nullptr;
  }
}

// The full-zone kernels of one pixel layout / edge class (NCH channels per
// descriptor, EDGE handling) for every kind that touches pixels; nullptr for
// the coefficient-only quantiser.
template <int KIND, int NCH, int EDGE>
KernelFn pick_full_mode(int qmode, bool evenq) {
  switch (qmode) {
    case QM_STEP:
      return evenq ? k_codec<KIND, QM_STEP, true, 14, NCH, EDGE> : k_codec<KIND, QM_STEP, false, 14, NCH, EDGE>;
    case QM_ZONAL: return k_codec<KIND, QM_ZONAL, false, 14, NCH, EDGE>;
    case QM_STEP_ZONAL:
      return evenq ? k_codec<KIND, QM_STEP_ZONAL, true, 14, NCH, EDGE>
                   : k_codec<KIND, QM_STEP_ZONAL, false, 14, NCH, EDGE>;
    case QM_ZONAL_ZZ:
      return (KIND == K_RT_FULL || KIND == K_RT_COEF) ? k_codec<KIND, QM_ZONAL_ZZ, false, 14, NCH, EDGE>
                                                       : k_codec<KIND, QM_ZONAL, false, 14, NCH, EDGE>;
    default: return k_codec<KIND, QM_NONE, false, 14, NCH, EDGE>;
  }
}

template <int NCH, int EDGE>
KernelFn pick_full(int kind, int qmode, bool evenq) {
  switch (kind) {
    case K_FORWARD: return k_codec<K_FORWARD, QM_NONE, false, 14, NCH, EDGE>;
    case K_INVERSE:
      return qmode == QM_ZONAL_ZZ ? k_codec<K_INVERSE, QM_ZONAL_ZZ, false, 14, NCH, EDGE>
                                  : k_codec<K_INVERSE, QM_NONE, false, 14, NCH, EDGE>;
    case K_RT_FULL: return pick_full_mode<K_RT_FULL, NCH, EDGE>(qmode, evenq);
    case K_RT_PIX: return pick_full_mode<K_RT_PIX, NCH, EDGE>(qmode, evenq);
    case K_RT_COEF: return pick_full_mode<K_RT_COEF, NCH, EDGE>(qmode, evenq);
    case K_RT_SSE: return pick_full_mode<K_RT_SSE, NCH, EDGE>(qmode, evenq);
    default: return nullptr;
  }
}

}  // namespace
}  // namespace adct
