// Device helpers shared by the libsrn kernels: the per-grid affine map (Eq. 1),
// the corner-aligned cell/weight set-up of Eq. 2, Philox4x32-10, bf16 packing and
// the brick/tile bookkeeping of the batched launches.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/srn.h"

namespace srn {

constexpr int kHidden = 64;
constexpr int kMaxK = 128;
constexpr int kMaxGrids = 128;
constexpr int kSortBits = 5;                       // 32^3 Morton bins per brick
constexpr int kSortBins = 1 << (3 * kSortBits);
constexpr int kUnitBits = kSortBits - 1;          // a unit is 2 x 2 x 2 bins
constexpr int kUnits = 1 << (3 * kUnitBits);

// Per-launch description of the bricks: points of brick b are [off[b], off[b+1]).
// When `dev` is non-NULL the offsets are read from device memory at kernel start
// (counts produced on the device, e.g. by the renderer's bucketing).
struct Bricks {
  int32_t n;
  const int64_t* dev;
  int64_t off[SRN_MAX_BRICKS + 1];
};

// Copy of the launch's brick offsets in shared memory (call from every thread;
// contains a __syncthreads).
__device__ __forceinline__ void load_bricks(const Bricks& in, Bricks& sh) {
  if (threadIdx.x == 0) {
    sh.n = in.n;
    sh.dev = nullptr;
    for (int b = 0; b <= in.n; ++b) sh.off[b] = in.dev ? in.dev[b] : in.off[b];
  }
  __syncthreads();
}

// Model tensors as the kernels see them.  Brick b's tensor X is at X + b * sX.
struct Model {
  const float* G;        // [B][M][12]
  const float* range;    // [B][2]
  const float* F32;      // FP32 master features (FP32 kernels)
  const __nv_bfloat16* F16;  // BF16 shadow features (BF16 kernels)
  const float* W1f; const float* W2f; const float* w3;       // FP32 decoder
  const __nv_bfloat16* W1h; const __nv_bfloat16* W2h;       // BF16 decoder
  int64_t sF, sW1, sW2, sw3, sG;
  int M, C, R, K, p;
};

struct Grads {
  float* dF; float* dW1; float* dW2; float* dw3;
  int64_t sF, sW1, sW2, sw3;
};

// Workspace pieces the training kernels write.
struct TrainWs {
  float* rho;       // [N] feature density of each point (Eq. 7)
  float* herr;      // [N] per-point squared error h(x)
  double* acc;      // [B][kAccPerBrick] float64 accumulators
  double* gsum;     // [B][M][13] float64 sums for dL_den/dG
  double* rsum;     // [B][M][12] float64 dL/dG through the features (rec_dg), laid out as G
  int32_t rec_dg;   // 1: accumulate rsum (SRN_REC_DG)
  int32_t* status;  // device status word
  int32_t upstream; // 1: the target slot holds dL/df (no L_rec); 0: MSE against targets
  __nv_bfloat16* Y;   // [N][K] features (BF16 training pass)
  __nv_bfloat16* dY;  // [N][M][C] dL/dy, point-major like Y (BF16 training pass)
  // [decoder tiles][M] the bf16 bits of the largest |dL/dy| of each grid over each
  // 128-point decoder tile (tiles numbered as build_tile_map numbers them for 128), or
  // NULL when the decoder does not produce them (the scatter then finds its scales itself)
  uint16_t* gmax_blk;
  int32_t* ustart;    // [B][kUnits + 1] first point of each Morton unit (BF16 scatter tiles)
  const uint32_t* bin_start;   // [B][kSortBins] the sampler's bin starts of this batch, or NULL
  struct ScatTile* tiles;  // scatter tiles (BF16 training pass)
  int32_t* tile_ctr;  // [0] tiles written, [1] next tile to take
  const struct BrickSched* sched;   // per-brick training routine, or NULL (caller's flags)
  float eps;          // the density loss's epsilon (Eq. 8-9)
};

// A tile of the encoder and the scatter: `count` (<= the tuning's tile_points, at most
// 1024) consecutive points of one brick, all in the aligned Morton range of 2^L units
// starting at unit u0 when the brick's points are sorted by Morton bin.
// code = brick << 20 | L << 16 | u0.
struct ScatTile {
  int64_t start;
  int32_t count;
  uint32_t code;
};
// Per-brick float64 accumulator slots.
enum { ACC_SUM_R2 = 0, ACC_SUM_RHO = 1, ACC_C = 2, ACC_LDEN = 3, kAccPerBrick = 4 };

// ------------------------------------------------------------------ Eq. 1 / Eq. 2
// Derivative of Eq. 2's interpolant with respect to s inside cell c, for the scalar
// field whose corner values are a[k] (k = dx + 2 dy + 4 dz): along x the four
// x-edges' differences weighted by the y and z weights, and likewise for y and z.
__device__ __forceinline__ void trilinear_ds(const float (&a)[8], float wx, float wy, float wz,
                                             float& dx, float& dy, float& dz) {
  const float ax = 1.f - wx, ay = 1.f - wy, az = 1.f - wz;
  dx = az * (ay * (a[1] - a[0]) + wy * (a[3] - a[2])) + wz * (ay * (a[5] - a[4]) + wy * (a[7] - a[6]));
  dy = az * (ax * (a[2] - a[0]) + wx * (a[3] - a[1])) + wz * (ax * (a[6] - a[4]) + wx * (a[7] - a[5]));
  dz = ay * (ax * (a[4] - a[0]) + wx * (a[5] - a[1])) + wy * (ax * (a[6] - a[2]) + wx * (a[7] - a[3]));
}

struct Cell {
  int cx, cy, cz;
  float wx, wy, wz;
  bool inside;
};

// Eq. 1 with G_i given as 12 floats (row-major 3x4).
__device__ __forceinline__ void affine(const float* g, float x, float y, float z,
                                       float& ux, float& uy, float& uz) {
  ux = fmaf(g[0], x, fmaf(g[1], y, fmaf(g[2], z, g[3])));
  uy = fmaf(g[4], x, fmaf(g[5], y, fmaf(g[6], z, g[7])));
  uz = fmaf(g[8], x, fmaf(g[9], y, fmaf(g[10], z, g[11])));
}

// Eq. 2 set-up on an R^3 grid with vertices at the extents: s = (u+1)(R-1)/2,
// cell c = min(floor(s), R-2), weight w = s - c; `inside` is -1 <= u <= 1 on all axes.
__device__ __forceinline__ Cell make_cell(float ux, float uy, float uz, int R) {
  Cell c;
  c.inside = (ux >= -1.f) & (ux <= 1.f) & (uy >= -1.f) & (uy <= 1.f) & (uz >= -1.f) & (uz <= 1.f);
  const float h = 0.5f * (float)(R - 1);
  float sx = fmaf(ux, h, h), sy = fmaf(uy, h, h), sz = fmaf(uz, h, h);
  sx = fminf(fmaxf(sx, 0.f), (float)(R - 1));
  sy = fminf(fmaxf(sy, 0.f), (float)(R - 1));
  sz = fminf(fmaxf(sz, 0.f), (float)(R - 1));
  c.cx = min((int)sx, R - 2);
  c.cy = min((int)sy, R - 2);
  c.cz = min((int)sz, R - 2);
  c.wx = sx - (float)c.cx;
  c.wy = sy - (float)c.cy;
  c.wz = sz - (float)c.cz;
  return c;
}

// x^E by repeated squaring (E known at compile time).
template <int E>
__device__ __forceinline__ float powi(float x) {
  if constexpr (E == 0) {
    return 1.f;
  } else if constexpr (E == 1) {
    return x;
  } else if constexpr (E % 2 == 0) {
    const float h = powi<E / 2>(x);
    return h * h;
  } else {
    return x * powi<E - 1>(x);
  }
}

// exp(-sum_d u_d^(2p)) of Eq. 7, and optionally 2p u_d^(2p-1) for its gradient.
// Returns 0 (and zero derivatives) once the exponent passes 87, where the float32
// exponential is below the smallest normal number.  p = 10 (the paper's value) takes
// a fixed squaring chain; other p loop.
__device__ __forceinline__ float flat_top(float ux, float uy, float uz, int p,
                                          float* dx = nullptr, float* dy = nullptr,
                                          float* dz = nullptr) {
  const float x2 = ux * ux, y2 = uy * uy, z2 = uz * uz;
  float px, py, pz;  // u^(2(p-1))
  if (p == 10) {
    px = powi<9>(x2); py = powi<9>(y2); pz = powi<9>(z2);
  } else {
    px = 1.f; py = 1.f; pz = 1.f;
    for (int k = 1; k < p; ++k) { px *= x2; py *= y2; pz *= z2; }
  }
  const float s = fmaf(px, x2, fmaf(py, y2, pz * z2));
  if (!(s <= 87.f)) {
    if (dx) { *dx = 0.f; *dy = 0.f; *dz = 0.f; }
    return 0.f;
  }
  const float e = __expf(-s);
  if (dx) {
    const float tp = 2.f * (float)p;
    *dx = tp * px * ux; *dy = tp * py * uy; *dz = tp * pz * uz;
  }
  return e;
}

// ------------------------------------------------------------------ packed float pairs
// Two float32 values in one 64-bit register pair, for the f32x2 arithmetic of sm_100+
// (one instruction issues both lanes' operation).
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t f2_pack(float lo, float hi) {
  return (f2_t)__float_as_uint(lo) | ((f2_t)__float_as_uint(hi) << 32);
}
__device__ __forceinline__ float f2_lo(f2_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float f2_hi(f2_t v) { return __uint_as_float((uint32_t)(v >> 32)); }
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b) {
  f2_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
  f2_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b) {
  f2_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// 3x3 determinant of the left block of a 3x4 row-major transform.
__device__ __forceinline__ float det3(const float* g) {
  return g[0] * (g[5] * g[10] - g[6] * g[9]) - g[1] * (g[4] * g[10] - g[6] * g[8]) +
         g[2] * (g[4] * g[9] - g[5] * g[8]);
}

// ------------------------------------------------------------------ bf16 helpers
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float2 unpack_bf16(uint32_t v) {
  __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162*>(&v);
  return __bfloat1622float2(b);
}

// ------------------------------------------------------------------ Morton order
// Morton code of the batch sampler's bins: bit 3k is bit k of the x bin, bit 3k+1 of
// the y bin, bit 3k+2 of the z bin, with 2^kSortBits bins per axis over [-1, 1].
__device__ __forceinline__ uint32_t spread3(uint32_t v) {  // 10 bits -> every third bit
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0xff0000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}
__device__ __forceinline__ uint32_t compact3(uint32_t v) {  // every third bit -> 10 bits
  v &= 0x09249249u;
  v = (v ^ (v >> 2)) & 0x030c30c3u;
  v = (v ^ (v >> 4)) & 0x0300f00fu;
  v = (v ^ (v >> 8)) & 0xff0000ffu;
  v = (v ^ (v >> 16)) & 0x000003ffu;
  return v;
}
__device__ __forceinline__ uint32_t morton_bin(float x, float y, float z) {
  const float s = (float)(1 << kSortBits) * 0.5f;
  const uint32_t ix = (uint32_t)min(max((int)((x + 1.f) * s), 0), (1 << kSortBits) - 1);
  const uint32_t iy = (uint32_t)min(max((int)((y + 1.f) * s), 0), (1 << kSortBits) - 1);
  const uint32_t iz = (uint32_t)min(max((int)((z + 1.f) * s), 0), (1 << kSortBits) - 1);
  return spread3(ix) | (spread3(iy) << 1) | (spread3(iz) << 2);
}

// ------------------------------------------------------------------ Philox4x32-10
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// ------------------------------------------------------------------ tiles over bricks
// The tiles of a batched launch: brick b owns ceil(n_b / T) consecutive tiles.
struct TileMap {
  int32_t first[SRN_MAX_BRICKS + 1];
};

__device__ __forceinline__ void build_tile_map(const Bricks& br, int T, TileMap& tm) {
  int acc = 0;
  for (int b = 0; b < br.n; ++b) {
    tm.first[b] = acc;
    acc += (int)((br.off[b + 1] - br.off[b] + T - 1) / T);
  }
  tm.first[br.n] = acc;
}

__device__ __forceinline__ int brick_of_tile(const TileMap& tm, int nb, int tile, int hint) {
  int b = hint < 0 ? 0 : hint;
  while (b + 1 <= nb && tm.first[b + 1] <= tile) ++b;
  return b;
}

}  // namespace srn
