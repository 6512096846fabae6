// Differentiable float32 variant of the transform (Sec. 2: C^ = D T is
// orthogonal) for sm_103a.  Forward: y = D T x T^T D per 8x8 block, then the
// optional soft quantiser z = y - (Q/2pi) sin(2pi y/Q).  Backward (adjoint):
// gx = T^T D (gy * (1 - cos(2pi y/Q))) D T, with y recomputed from x so the
// forward saves nothing but x.  T and T^T are applied with the same
// 14-addition butterflies as the integer codec (fadd only); D enters as one
// multiply per coefficient.
//
// Work split: one thread per 8x8 block, a warp on 32 consecutive blocks (a
// "tile").  Each warp copies its next tile (x, and gy for the adjoint) into
// shared memory with cp.async while it computes the current one, so that the
// loads of one tile overlap the arithmetic of the previous one: 8 rows of 64
// 16-byte chunks per tensor, each warp copy instruction moving 512 contiguous
// bytes when the tile lies in one block row.  One stage per tensor is enough,
// because a thread moves its block from shared memory into registers before
// the next copy into that stage is issued.  The forward also stages its
// output tile, so that its stores are 512-byte warp writes too; the adjoint
// stages its output in the gy tile once that has been read, and issues the
// next gy copy after the write-back (a third tile would cost warps; measured:
// 104.5 us -> 100.3 us against direct stores, 64 x 3 x 512x512).
//
// Soft quantiser phase: sin and cos of 2 pi h, h = y / Q, by range reduction
// (h minus the nearest integer, then the symmetries sin(2 pi b) = sin(2 pi
// (1/2 - b)) and cos(2 pi b) = -cos(2 pi (1/2 - b))) to b in [0, 1/4], and
// the Taylor series of sin and cos there, truncated after the x^11 and x^12
// terms of x = 2 pi b <= pi / 2: the truncation errors are below
// (pi/2)^13 / 13! < 6e-8 and (pi/2)^14 / 14! < 1e-9, under float32 rounding.
#include <cuda_runtime.h>

#include "adct_internal.h"

namespace adct {
namespace {

// One warp per CTA, 12 CTAs per SM (registers allow 12 warps): measured on
// 64 x 3 x 512x512, the forward + adjoint pair runs in 168.7 us against
// 174.5 us with CTAs of 4 warps, 3 per SM (the forward 69 us against 75 us).
constexpr int kFloatThreads = 32;
constexpr int kFloatMinCtas = 384 / kFloatThreads;  // 12 warps per SM

// d_i = 2^(-a_i / 2): 1/sqrt8, 1/sqrt2, 1/2 (Sec. 2, matrix D)
__host__ __device__ constexpr float d_of(int i) {
  return scale_exp(i) == 3 ? 0.35355339059327373f : (scale_exp(i) == 2 ? 0.5f : 0.70710678118654752f);
}

// Taylor coefficient of the power 2m + odd of sin (odd = 1) or cos (odd = 0)
// of 2 pi b, as a polynomial in b: (-1)^m (2 pi)^n / n!, n = 2m + odd.
constexpr double kTwoPi = 6.283185307179586476925286766559;
__host__ __device__ constexpr double taylor_coef(int m, int odd) {
  const int n = 2 * m + odd;
  double c = 1.0;
  for (int k = 1; k <= n; ++k) c *= kTwoPi / k;
  return (m % 2) ? -c : c;
}

// h -> (b', w, b): w = h - nearest integer in [-1/2, 1/2], b = |w|,
// b' = min(b, 1/2 - b) in [0, 1/4].
struct Phase {
  float w, b, bp;
};
__device__ __forceinline__ Phase reduce_phase(float h) {
  Phase p;
  p.w = h - rintf(h);  // exact
  p.b = fabsf(p.w);
  p.bp = fminf(p.b, 0.5f - p.b);
  return p;
}

// sin(2 pi h)
__device__ __forceinline__ float sin_2pi(float h) {
  constexpr float s0 = (float)taylor_coef(0, 1), s1 = (float)taylor_coef(1, 1), s2 = (float)taylor_coef(2, 1);
  constexpr float s3 = (float)taylor_coef(3, 1), s4 = (float)taylor_coef(4, 1), s5 = (float)taylor_coef(5, 1);
  const Phase p = reduce_phase(h);
  const float x = p.bp * p.bp;
  const float s = fmaf(fmaf(fmaf(fmaf(fmaf(s5, x, s4), x, s3), x, s2), x, s1), x, s0);
  return copysignf(s * p.bp, p.w);
}

// cos(2 pi h)
__device__ __forceinline__ float cos_2pi(float h) {
  constexpr float c0 = (float)taylor_coef(0, 0), c1 = (float)taylor_coef(1, 0), c2 = (float)taylor_coef(2, 0);
  constexpr float c3 = (float)taylor_coef(3, 0), c4 = (float)taylor_coef(4, 0), c5 = (float)taylor_coef(5, 0);
  constexpr float c6 = (float)taylor_coef(6, 0);
  const Phase p = reduce_phase(h);
  const float x = p.bp * p.bp;
  const float c = fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(c6, x, c5), x, c4), x, c3), x, c2), x, c1), x, c0);
  return copysignf(c, p.bp - p.b);  // negative exactly when b > 1/4
}

// ---- tiles in shared memory ----
// A tile is 8 rows of 32 blocks x 8 floats = 8 rows x 64 chunks of 16 bytes.
// Chunk q (block q / 2, half q % 2) of row i sits at slot i * 64 + swz(q):
// lanes reading chunk 2 l + c, and lanes copying chunk 32 k + l, fall in
// distinct 16-byte bank groups within each quarter warp.
constexpr int kTileBytes = 8 * 64 * 16;
__device__ __forceinline__ int swz(int q) { return q ^ ((q >> 3) & 1); }

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Shape of one launch: total blocks over all planes, blocks per plane and per
// block row, the row length in floats.  When total < 2^31 the divisions by nb
// and wb are multiply-highs: with k = 31 + ceil(log2 d), m = ceil(2^k / d)
// and e = m d - 2^k in [0, d), n m / 2^k = n / d + n e / (d 2^k), where
// n e < 2^31 d <= 2^k: the excess is below 1 / d, too little to carry n / d
// (whose fraction is at most (d - 1) / d) past the next integer, so
// (n m) >> k = floor(n / d) for every n < 2^31.
struct FloatShape {
  int64_t total, nb;
  int32_t wb, W;
  uint32_t mnb, mwb;  // magic multipliers (small launches)
  int32_t knb, kwb;   // their shifts
  bool small;         // total < 2^31
};

__device__ __forceinline__ uint32_t div_magic(uint32_t n, uint32_t m, int k) {
  return (uint32_t)(((uint64_t)n * m) >> k);
}

// Offset (floats) of lane's block g0 + lane, or -1 past the end.  A plane
// holds nb blocks of 64 floats.
__device__ __forceinline__ int64_t lane_block(const FloatShape& s, int64_t g0, int lane) {
  const int64_t g = g0 + lane;
  if (g >= s.total) return -1;
  int64_t plane, by, bx;
  if (s.small) {
    const uint32_t n = (uint32_t)g;
    const uint32_t p = div_magic(n, s.mnb, s.knb);
    const uint32_t f = n - p * (uint32_t)s.nb;
    const uint32_t y = div_magic(f, s.mwb, s.kwb);
    plane = p;
    by = y;
    bx = f - y * (uint32_t)s.wb;
  } else {
    plane = g / s.nb;
    const int64_t f = g - plane * s.nb;
    by = f / s.wb;
    bx = f - by * s.wb;
  }
  return plane * s.nb * 64 + 8 * by * (int64_t)s.W + 8 * bx;
}

// Copies tile g0 of tensor t into `tile` (not committed): lane l copies
// chunks 32 k + l (k = 0, 1) of every row, i.e. half q % 2 of block q / 2,
// whose offset it takes from that block's lane.  Blocks past the end copy
// nothing.
__device__ __forceinline__ void issue_tile(uint8_t* tile, const float* __restrict__ t, int64_t my_off,
                                           const FloatShape& s, int lane) {
  const uint32_t sa = smem_addr(tile);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int q = 32 * k + lane;
    const int64_t off = __shfl_sync(0xffffffffu, my_off, q >> 1);
    if (off >= 0) {
      const float* src = t + off + 4 * (q & 1);
#pragma unroll
      for (int i = 0; i < 8; ++i) cp_async16(sa + (i * 64 + swz(q)) * 16, src + (int64_t)i * s.W);
    }
  }
}

// Lane's block from the tile, row-major into v.
__device__ __forceinline__ void read_block(const uint8_t* tile, int lane, float* v) {
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float4 u = *(const float4*)(tile + (i * 64 + swz(2 * lane + c)) * 16);
      v[8 * i + 4 * c + 0] = u.x;
      v[8 * i + 4 * c + 1] = u.y;
      v[8 * i + 4 * c + 2] = u.z;
      v[8 * i + 4 * c + 3] = u.w;
    }
}

// Forward: each warp walks tiles g0, g0 + step, ... (step = all threads of
// the grid), copying tile n + 1 while computing tile n.  The results go
// through a second tile in shared memory (same layout), from which the warp
// writes 512 contiguous bytes per store instruction instead of each lane's
// 16-byte halves 32 bytes apart (measured: 77.9 us -> 74.2 us for
// 64 x 3 x 512x512).
template <bool SOFT>
__global__ void __launch_bounds__(kFloatThreads, kFloatMinCtas) k_float_fwd(const float* __restrict__ x, float* __restrict__ y,
                                                             const FloatShape s, const FloatParams fp) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int lane = threadIdx.x & 31;
  uint8_t* tile = smem + (threadIdx.x >> 5) * kTileBytes;
  uint8_t* out = smem + (blockDim.x >> 5) * kTileBytes + (threadIdx.x >> 5) * kTileBytes;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  int64_t g0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
  if (g0 >= s.total) return;
  int64_t off = lane_block(s, g0, lane);
  issue_tile(tile, x, off, s, lane);
  cp_async_commit();
  for (; g0 < s.total; g0 += step) {
    cp_async_wait<0>();
    __syncwarp();
    float v[64];
    read_block(tile, lane, v);
    __syncwarp();
    const int64_t cur = off;
    off = lane_block(s, g0 + step, lane);
    issue_tile(tile, x, off, s, lane);
    cp_async_commit();
    if (cur >= 0) {
      fwd2d(v);
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int k = 8 * i + j;
          const float t = v[k] * (d_of(i) * d_of(j));
          v[k] = SOFT ? fmaf(-fp.c2pi[k], sin_2pi(t * fp.rq[k]), t) : t;
        }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int c = 0; c < 2; ++c)
          *(float4*)(out + (i * 64 + swz(2 * lane + c)) * 16) =
              make_float4(v[8 * i + 4 * c], v[8 * i + 4 * c + 1], v[8 * i + 4 * c + 2], v[8 * i + 4 * c + 3]);
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int q = 32 * k + lane;
      const int64_t o = __shfl_sync(0xffffffffu, cur, q >> 1);
      if (o >= 0) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
          __stcs((float4*)(y + o + 4 * (q & 1) + (int64_t)i * s.W), *(const float4*)(out + (i * 64 + swz(q)) * 16));
      }
    }
  }
  cp_async_wait<0>();
}

// Adjoint.  SOFT: the x tile n + 1 is copied while tile n's y and
// d_i d_j (1 - cos(2pi y / Q)) are computed, and the gy tile n + 1 (issued
// once tile n's gx has been staged in the gy tile and written back) while
// tile n + 1's y is recomputed.  Copy groups are committed in the order
// x_{n+1}, gy_{n+1}, so "all but the newest group done" first means x_n is
// in, then (after x_{n+1} was committed) that gy_n is in.
template <bool SOFT>
__global__ void __launch_bounds__(kFloatThreads, kFloatMinCtas) k_float_bwd(const float* __restrict__ x, const float* __restrict__ gy,
                                                             float* __restrict__ gx, const FloatShape s,
                                                             const FloatParams fp) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int lane = threadIdx.x & 31;
  uint8_t* tx = smem + (threadIdx.x >> 5) * (SOFT ? 2 : 1) * kTileBytes;
  uint8_t* tg = SOFT ? tx + kTileBytes : tx;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  int64_t g0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
  if (g0 >= s.total) return;  // whole warp
  int64_t off = lane_block(s, g0, lane);
  if (SOFT) {
    issue_tile(tx, x, off, s, lane);
    cp_async_commit();
  }
  issue_tile(tg, gy, off, s, lane);
  cp_async_commit();
  for (; g0 < s.total; g0 += step) {
    const int64_t cur = off;
    off = lane_block(s, g0 + step, lane);
    float v[64];  // SOFT: d_i d_j dz/dy, then the adjoint's input D (gy dz/dy) D
    if (SOFT) {
      cp_async_wait<1>();
      __syncwarp();
      read_block(tx, lane, v);
      __syncwarp();
      issue_tile(tx, x, off, s, lane);
      cp_async_commit();
      if (cur >= 0) {
        fwd2d(v);
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int k = 8 * i + j;
            const float dd = d_of(i) * d_of(j);
            v[k] = fmaf(-dd, cos_2pi(v[k] * fp.g[k]), dd);
          }
      }
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float4 u = *(const float4*)(tg + (i * 64 + swz(2 * lane + c)) * 16);
        const float r[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int j = 4 * c + e, k = 8 * i + j;
          v[k] = SOFT ? r[e] * v[k] : r[e] * (d_of(i) * d_of(j));
        }
      }
    // the gy tile has been read: stage this tile's gx in it and write it back
    // with 512-byte warp stores, then refill it with the next gy tile
    __syncwarp();
    if (cur >= 0) {
      inv2d(v);
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int c = 0; c < 2; ++c)
          *(float4*)(tg + (i * 64 + swz(2 * lane + c)) * 16) =
              make_float4(v[8 * i + 4 * c], v[8 * i + 4 * c + 1], v[8 * i + 4 * c + 2], v[8 * i + 4 * c + 3]);
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int q = 32 * k + lane;
      const int64_t o = __shfl_sync(0xffffffffu, cur, q >> 1);
      if (o >= 0) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
          __stcs((float4*)(gx + o + 4 * (q & 1) + (int64_t)i * s.W), *(const float4*)(tg + (i * 64 + swz(q)) * 16));
      }
    }
    __syncwarp();
    issue_tile(tg, gy, off, s, lane);
    cp_async_commit();
  }
  cp_async_wait<0>();
}

template <class K>
cudaError_t launch_float(K kernel, size_t smem, int64_t total, int sm_count, cudaStream_t stream,
                         void (*go)(K, int, size_t, cudaStream_t, void*), void* args) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kFloatThreads, smem);
  if (e != cudaSuccess) return e;
  int64_t want = (total + kFloatThreads - 1) / kFloatThreads;
  const int64_t cap = (int64_t)sm_count * (per_sm < 1 ? 1 : per_sm);
  if (want > cap) want = cap;
  go(kernel, (int)(want < 1 ? 1 : want), smem, stream, args);
  return cudaGetLastError();
}

// Multiplier and shift for exact n / d, n < 2^31, 1 <= d < 2^31 (FloatShape).
void magic_for(int64_t d, uint32_t* m, int32_t* k) {
  int lg = 0;
  while ((int64_t(1) << lg) < d) ++lg;  // ceil(log2 d)
  *k = 31 + lg;
  *m = (uint32_t)(((uint64_t(1) << *k) + (uint64_t)d - 1) / (uint64_t)d);
}

FloatShape float_shape(int64_t planes, int32_t H, int32_t W) {
  FloatShape s{};
  s.wb = W / 8;
  s.nb = (int64_t)(H / 8) * s.wb;
  s.total = planes * s.nb;
  s.W = W;
  s.small = s.total < (int64_t(1) << 31);
  if (s.small) {
    magic_for(s.nb, &s.mnb, &s.knb);
    magic_for(s.wb, &s.mwb, &s.kwb);
  }
  return s;
}

}  // namespace

cudaError_t launch_float_forward(const float* x, float* y, int64_t planes, int32_t H, int32_t W,
                                 const FloatParams* fp, int sm_count, cudaStream_t stream) {
  const FloatShape s = float_shape(planes, H, W);
  if (s.total <= 0) return cudaSuccess;
  FloatParams none{};
  struct A { const float* x; float* y; FloatShape s; const FloatParams* fp; } a{x, y, s, fp ? fp : &none};
  using K = void (*)(const float*, float*, const FloatShape, const FloatParams);
  auto go = [](K k, int grid, size_t smem, cudaStream_t st, void* p) {
    const A& a = *(const A*)p;
    k<<<grid, kFloatThreads, smem, st>>>(a.x, a.y, a.s, *a.fp);
  };
  const size_t smem = (size_t)(kFloatThreads / 32) * 2 * kTileBytes;
  return fp ? launch_float<K>(k_float_fwd<true>, smem, s.total, sm_count, stream, go, &a)
            : launch_float<K>(k_float_fwd<false>, smem, s.total, sm_count, stream, go, &a);
}

cudaError_t launch_float_backward(const float* x, const float* gy, float* gx, int64_t planes, int32_t H,
                                  int32_t W, const FloatParams* fp, int sm_count, cudaStream_t stream) {
  const FloatShape s = float_shape(planes, H, W);
  if (s.total <= 0) return cudaSuccess;
  FloatParams none{};
  struct A { const float* x; const float* gy; float* gx; FloatShape s; const FloatParams* fp; } a{
      x, gy, gx, s, fp ? fp : &none};
  using K = void (*)(const float*, const float*, float*, const FloatShape, const FloatParams);
  auto go = [](K k, int grid, size_t smem, cudaStream_t st, void* p) {
    const A& a = *(const A*)p;
    k<<<grid, kFloatThreads, smem, st>>>(a.x, a.gy, a.gx, a.s, *a.fp);
  };
  const size_t smem = (size_t)(kFloatThreads / 32) * (fp ? 2 : 1) * kTileBytes;
  return fp ? launch_float<K>(k_float_bwd<true>, smem, s.total, sm_count, stream, go, &a)
            : launch_float<K>(k_float_bwd<false>, smem, s.total, sm_count, stream, go, &a);
}

}  // namespace adct
