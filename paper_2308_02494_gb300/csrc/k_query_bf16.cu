// BF16 fused point-query kernel: encoder (Eq. 1-3) -> decoder (Sec. 4.1.2) ->
// in training, L_rec (Sec. 4.3.1) and its gradient into the feature grids and
// the decoder, plus the per-point feature density of Eq. 7.
//
// One persistent CTA per SM walks a contiguous range of 128-point tiles; tiles
// of different bricks (domain-decomposition models, Sec. 5) may follow each
// other, and the CTA reloads that brick's decoder and transforms when the brick
// changes.  Per tile:
//   encode   thread (point, half of the grids): Eq. 1 in registers (the N x M
//            local coordinates are never stored), Eq. 2 by eight corner loads of
//            the BF16 grid through L1, features written to shared memory (BF16)
//   decoder  warp w owns rows 16w..16w+15: two tensor-core layers (m16n8k16,
//            FP32 accumulate), the 64->1 output layer in FP32
//   backward dH2, dH1, dY per warp on tensor cores; dW2 = dH2^T H1 and
//            dW1 = dH1^T Y across the tile, accumulated in registers over every
//            tile of the brick and flushed once
//   scatter  the corner weights are recomputed and dY is added into the FP32
//            gradient grids (8 float2 atomics per point and grid)
#include "common.cuh"
#include "kernels.h"

// Phase markers (no-ops unless a profiling build defines them): SRN_PHASE_BEGIN at
// kernel start, SRN_PHASE(k) after the block-wide barrier that ends phase k.
#ifndef SRN_PHASE
#define SRN_PHASE(k)
#define SRN_PHASE_BEGIN
#endif

namespace srn {
namespace {

constexpr int T = 128;   // points per tile
constexpr int NT = 256;  // threads per CTA

__device__ __forceinline__ uint32_t su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (row, col) of a bf16 matrix with rows of L elements whose
// 16-byte chunks are XOR-swizzled by the row index (conflict-free ldmatrix).
template <int L>
__device__ __forceinline__ int swz(int row, int col) {
  constexpr int chunks = L / 8;
  constexpr int mask = (chunks < 8 ? chunks : 8) - 1;
  return row * (L * 2) + (((col >> 3) ^ (row & mask)) << 4) + ((col & 7) << 1);
}

__device__ __forceinline__ void ldsm4(uint32_t (&r)[4], uint32_t a) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}
__device__ __forceinline__ void ldsm4t(uint32_t (&r)[4], uint32_t a) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}
__device__ __forceinline__ void ldsm2t(uint32_t (&r)[2], uint32_t a) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}
__device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Node loads of a BF16 grid with C channels innermost.
__device__ __forceinline__ float2 node2(const __nv_bfloat16* F, int64_t n) {
  return unpack_bf16(__ldg(reinterpret_cast<const unsigned int*>(F) + n));
}
__device__ __forceinline__ float node1(const __nv_bfloat16* F, int64_t n) {
  return __uint_as_float(static_cast<uint32_t>(__ldg(reinterpret_cast<const unsigned short*>(F) + n)) << 16);
}

// Eq. 2 (inside the grid): trilinear blend of the 8 corners of cell c.
__device__ __forceinline__ void trilinear_bf16(const __nv_bfloat16* Fi, const Cell& c, int R, int C,
                                               float& o0, float& o1) {
  const int64_t b = ((int64_t)c.cz * R + c.cy) * R + c.cx;
  const int64_t sy = R, sz = (int64_t)R * R;
  const float ax = 1.f - c.wx, ay = 1.f - c.wy, az = 1.f - c.wz;
  if (C == 2) {
    const float2 v0 = node2(Fi, b), v1 = node2(Fi, b + 1);
    const float2 v2 = node2(Fi, b + sy), v3 = node2(Fi, b + sy + 1);
    const float2 v4 = node2(Fi, b + sz), v5 = node2(Fi, b + sz + 1);
    const float2 v6 = node2(Fi, b + sz + sy), v7 = node2(Fi, b + sz + sy + 1);
    o0 = az * (ay * (ax * v0.x + c.wx * v1.x) + c.wy * (ax * v2.x + c.wx * v3.x)) +
         c.wz * (ay * (ax * v4.x + c.wx * v5.x) + c.wy * (ax * v6.x + c.wx * v7.x));
    o1 = az * (ay * (ax * v0.y + c.wx * v1.y) + c.wy * (ax * v2.y + c.wx * v3.y)) +
         c.wz * (ay * (ax * v4.y + c.wx * v5.y) + c.wy * (ax * v6.y + c.wx * v7.y));
  } else {
    const float v0 = node1(Fi, b), v1 = node1(Fi, b + 1);
    const float v2 = node1(Fi, b + sy), v3 = node1(Fi, b + sy + 1);
    const float v4 = node1(Fi, b + sz), v5 = node1(Fi, b + sz + 1);
    const float v6 = node1(Fi, b + sz + sy), v7 = node1(Fi, b + sz + sy + 1);
    o0 = az * (ay * (ax * v0 + c.wx * v1) + c.wy * (ax * v2 + c.wx * v3)) +
         c.wz * (ay * (ax * v4 + c.wx * v5) + c.wy * (ax * v6 + c.wx * v7));
    o1 = 0.f;
  }
}

// Adjoint of Eq. 2: add g * weight into each corner of cell c of the FP32 gradient grid.
__device__ __forceinline__ void scatter_f32(float* dFi, const Cell& c, int R, int C, float g0, float g1) {
  const int64_t b = ((int64_t)c.cz * R + c.cy) * R + c.cx;
  const int64_t sy = R, sz = (int64_t)R * R;
  const float ax = 1.f - c.wx, ay = 1.f - c.wy, az = 1.f - c.wz;
  const float w[8] = {az * ay * ax, az * ay * c.wx, az * c.wy * ax, az * c.wy * c.wx,
                      c.wz * ay * ax, c.wz * ay * c.wx, c.wz * c.wy * ax, c.wz * c.wy * c.wx};
  const int64_t o[8] = {b, b + 1, b + sy, b + sy + 1, b + sz, b + sz + 1, b + sz + sy, b + sz + sy + 1};
  if (C == 2) {
    float2* d = reinterpret_cast<float2*>(dFi);
#pragma unroll
    for (int k = 0; k < 8; ++k) atomicAdd(d + o[k], make_float2(g0 * w[k], g1 * w[k]));
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) atomicAdd(dFi + o[k], g0 * w[k]);
  }
}

template <int K>
struct Lay {
  static constexpr int DYS = K + 2;                    // dY row stride in floats
  static constexpr int W1 = 0;                         // [64][K] bf16, swizzled
  static constexpr int W2 = W1 + 64 * K * 2;           // [64][64] bf16
  static constexpr int Y = W2 + 64 * 64 * 2;           // [T][K] bf16 features
  static constexpr int H1 = Y + T * K * 2;             // [T][64] bf16 ReLU(z1)
  static constexpr int DH2 = H1 + T * 64 * 2;          // [T][64] bf16 dL/dz2
  static constexpr int DH1 = DH2 + T * 64 * 2;         // [T][64] bf16 dL/dz1
  static constexpr int DY = DH1 + T * 64 * 2;          // [T][DYS] f32 dL/dy
  static constexpr int W3 = DY + T * DYS * 4;          // [64] f32
  static constexpr int X = (W3 + 64 * 4 + 15) / 16 * 16;  // [T] float4 (x, y, z, target)
  static constexpr int RHO = X + T * 16;               // [2][T] f32 partial densities
  static constexpr int G = RHO + 2 * T * 4;            // [M][12] f32
  static constexpr int DET = G + kMaxGrids * 12 * 4;   // [M] f32
  static constexpr int BOX = DET + kMaxGrids * 4;      // [M] TileBox
  static constexpr int AABB = BOX + kMaxGrids * 32;    // [4][6] f32 per-warp partial bounds
  static constexpr int BYTES = AABB + 4 * 6 * 4;
  // During the encode, H1/DH2/DH1 (free until the decoder runs) hold each grid's
  // staged node box; after the weight gradients, Y..DH1 hold the scatter scratch.
  static constexpr int STG = H1;
  static constexpr int STG_BYTES = 3 * T * 64 * 2;
  static constexpr int SCR = Y;
  static constexpr int SCR_WARP = ((T * K * 2 + STG_BYTES) / 8) / 16 * 16;  // per warp
};

// Node box of one grid covering one tile's points (from the tile's bounding box).
struct TileBox {
  int lo[3];      // first node (x, y, z)
  int n[3];       // nodes per axis (cells per axis + 1); 0 when no point can be inside
  int flags;      // bit 0: staged in shared memory, bit 1: scatter through the box
  int cells;      // (n0 - 1)(n1 - 1)(n2 - 1)
};
enum { BOX_STAGED = 1, BOX_SCATTER = 2 };

// Per-warp scatter scratch: per-cell corner sums, counting-sort arrays, point weights.
template <int K>
struct Scr {
  static constexpr int FIX = T * 2 + T * 12 + T * 2 + 16;  // perm, weights, cell ids, slack
  __host__ __device__ static constexpr int capc(int C) {
    const int c = (Lay<K>::SCR_WARP - FIX) / (32 * C + 4);
    return c > 256 ? 256 : c;
  }
};

__device__ __forceinline__ void cp_async4(uint32_t saddr, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(saddr), "l"(g));
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }

template <int K, int MODE>
__global__ void __launch_bounds__(NT, 1)
k_query_bf16(Model md, Grads gr, Bricks brp, TrainWs ws, const float* __restrict__ xyz,
             const float* __restrict__ target, float* __restrict__ out) {
  constexpr bool TRAIN = MODE >= kTrain;
  constexpr bool DENS = MODE == kTrainDensity;
  constexpr int NW1 = K / 16;   // dW1 n-tiles per warp
  constexpr int NTY = K / 8;    // dY n-tiles per row block
  using L = Lay<K>;
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ TileMap tm;
  __shared__ Bricks br;
  load_bricks(brp, br);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g8 = lane >> 2, t4 = lane & 3;
  const int M = md.M, C = md.C, R = md.R;
  SRN_PHASE_BEGIN
  if (tid == 0) build_tile_map(br, T, tm);
  __syncthreads();
  const int total = tm.first[br.n];
  const int per = (total + gridDim.x - 1) / gridDim.x;
  const int tb = blockIdx.x * per, te = min(total, tb + per);

  float* xs = reinterpret_cast<float*>(sm + L::X);
  float* w3s = reinterpret_cast<float*>(sm + L::W3);
  float* gs = reinterpret_cast<float*>(sm + L::G);
  float* dets = reinterpret_cast<float*>(sm + L::DET);
  float* rhos = reinterpret_cast<float*>(sm + L::RHO);
  float* dys = reinterpret_cast<float*>(sm + L::DY);
  const uint32_t sW1 = su32(sm + L::W1), sW2 = su32(sm + L::W2), sY = su32(sm + L::Y);
  const uint32_t sH1 = su32(sm + L::H1), sDH2 = su32(sm + L::DH2), sDH1 = su32(sm + L::DH1);

  float dw1[NW1][4], dw2[4][4], dw3[8][2];
  double sum_r2 = 0.0, sum_rho = 0.0;
#pragma unroll
  for (int i = 0; i < NW1; ++i) dw1[i][0] = dw1[i][1] = dw1[i][2] = dw1[i][3] = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) dw2[i][0] = dw2[i][1] = dw2[i][2] = dw2[i][3] = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) dw3[i][0] = dw3[i][1] = 0.f;

  // Adds this CTA's decoder-gradient and loss partials of brick b to global memory.
  auto flush = [&](int b) {
    float* gW1 = gr.dW1 + (int64_t)b * gr.sW1;
    float* gW2 = gr.dW2 + (int64_t)b * gr.sW2;
    const int mt = warp & 3;
    const int nb2 = (warp >> 2) * 32, nb1 = (warp >> 2) * (K / 2);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = nb2 + j * 8 + 2 * t4, row = mt * 16 + g8;
      atomicAdd(gW2 + row * 64 + col, dw2[j][0]);
      atomicAdd(gW2 + row * 64 + col + 1, dw2[j][1]);
      atomicAdd(gW2 + (row + 8) * 64 + col, dw2[j][2]);
      atomicAdd(gW2 + (row + 8) * 64 + col + 1, dw2[j][3]);
      dw2[j][0] = dw2[j][1] = dw2[j][2] = dw2[j][3] = 0.f;
    }
#pragma unroll
    for (int j = 0; j < NW1; ++j) {
      const int col = nb1 + j * 8 + 2 * t4, row = mt * 16 + g8;
      atomicAdd(gW1 + row * K + col, dw1[j][0]);
      atomicAdd(gW1 + row * K + col + 1, dw1[j][1]);
      atomicAdd(gW1 + (row + 8) * K + col, dw1[j][2]);
      atomicAdd(gW1 + (row + 8) * K + col + 1, dw1[j][3]);
      dw1[j][0] = dw1[j][1] = dw1[j][2] = dw1[j][3] = 0.f;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        float v = dw3[j][e];
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        v += __shfl_xor_sync(0xffffffffu, v, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 16);
        if (g8 == 0) atomicAdd(gr.dw3 + (int64_t)b * gr.sw3 + j * 8 + 2 * t4 + e, v);
        dw3[j][e] = 0.f;
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      sum_r2 += __shfl_xor_sync(0xffffffffu, sum_r2, o);
      sum_rho += __shfl_xor_sync(0xffffffffu, sum_rho, o);
    }
    if (lane == 0) {
      atomicAdd(ws.acc + b * kAccPerBrick + ACC_SUM_R2, sum_r2);
      if (DENS) atomicAdd(ws.acc + b * kAccPerBrick + ACC_SUM_RHO, sum_rho);
    }
    sum_r2 = 0.0;
    sum_rho = 0.0;
  };

  int cur = -1;
  float span = 0.f, vmin = 0.f, inv_n = 0.f;
  for (int tile = tb; tile < te; ++tile) {
    const int b = brick_of_tile(tm, br.n, tile, cur);
    if (b != cur) {
      if (TRAIN && cur >= 0) flush(cur);
      __syncthreads();
      cur = b;
      {  // this brick's decoder and transforms into shared memory
        const uint4* w1 = reinterpret_cast<const uint4*>(md.W1h + (int64_t)b * md.sW1);
        for (int c = tid; c < 64 * K / 8; c += NT)
          *reinterpret_cast<uint4*>(sm + L::W1 + swz<K>(c / (K / 8), (c % (K / 8)) * 8)) = w1[c];
        const uint4* w2 = reinterpret_cast<const uint4*>(md.W2h + (int64_t)b * md.sW2);
        for (int c = tid; c < 64 * 8; c += NT)
          *reinterpret_cast<uint4*>(sm + L::W2 + swz<64>(c / 8, (c % 8) * 8)) = w2[c];
        if (tid < 64) w3s[tid] = md.w3[(int64_t)b * md.sw3 + tid];
        const float* G = md.G + (int64_t)b * md.sG;
        for (int c = tid; c < M * 12; c += NT) gs[c] = G[c];
        if (tid < M) dets[tid] = det3(G + 12 * tid);
      }
      vmin = md.range[2 * b];
      span = md.range[2 * b + 1] - vmin;
      inv_n = 1.f / (float)(br.off[b + 1] - br.off[b]);
      __syncthreads();
    }
    const int64_t p0 = br.off[b] + (int64_t)(tile - tm.first[b]) * T;
    const int np = (int)min((int64_t)T, br.off[b + 1] - p0);

    // ---- points (and targets) of the tile, and per-warp partial bounding boxes
    float* aabb = reinterpret_cast<float*>(sm + L::AABB);
    TileBox* boxes = reinterpret_cast<TileBox*>(sm + L::BOX);
    if (tid < T) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      const bool ok = tid < np;
      if (ok) {
        const float* q = xyz + 3 * (p0 + tid);
        v.x = q[0]; v.y = q[1]; v.z = q[2];
        if (TRAIN) v.w = target[p0 + tid];
      }
      reinterpret_cast<float4*>(xs)[tid] = v;
      float lo0 = ok ? v.x : INFINITY, lo1 = ok ? v.y : INFINITY, lo2 = ok ? v.z : INFINITY;
      float hi0 = ok ? v.x : -INFINITY, hi1 = ok ? v.y : -INFINITY, hi2 = ok ? v.z : -INFINITY;
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        lo0 = fminf(lo0, __shfl_xor_sync(0xffffffffu, lo0, o));
        lo1 = fminf(lo1, __shfl_xor_sync(0xffffffffu, lo1, o));
        lo2 = fminf(lo2, __shfl_xor_sync(0xffffffffu, lo2, o));
        hi0 = fmaxf(hi0, __shfl_xor_sync(0xffffffffu, hi0, o));
        hi1 = fmaxf(hi1, __shfl_xor_sync(0xffffffffu, hi1, o));
        hi2 = fmaxf(hi2, __shfl_xor_sync(0xffffffffu, hi2, o));
      }
      if (lane == 0) {
        float* a = aabb + 6 * warp;
        a[0] = lo0; a[1] = lo1; a[2] = lo2; a[3] = hi0; a[4] = hi1; a[5] = hi2;
      }
    }
    __syncthreads();
    SRN_PHASE(0);

    // ---- each grid's node box over the tile: the 8 corners of the tile's bounding
    //      box mapped by Eq. 1, widened by 1e-3 cell so float32 rounding of any inner
    //      point stays inside (every use below still bounds-checks the point's cell)
    const int cap_nodes = L::STG_BYTES / (M * 2 * C);
    const int capc = Scr<K>::capc(C);
    if (tid < M) {
      float lo[3], hi[3];
      for (int d = 0; d < 3; ++d) {
        lo[d] = fminf(fminf(aabb[d], aabb[6 + d]), fminf(aabb[12 + d], aabb[18 + d]));
        hi[d] = fmaxf(fmaxf(aabb[3 + d], aabb[9 + d]), fmaxf(aabb[15 + d], aabb[21 + d]));
      }
      float umin[3] = {INFINITY, INFINITY, INFINITY}, umax[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        float u[3];
        affine(gs + 12 * tid, (k & 1) ? hi[0] : lo[0], (k & 2) ? hi[1] : lo[1], (k & 4) ? hi[2] : lo[2],
               u[0], u[1], u[2]);
        for (int d = 0; d < 3; ++d) { umin[d] = fminf(umin[d], u[d]); umax[d] = fmaxf(umax[d], u[d]); }
      }
      TileBox bx;
      bool empty = np == 0;
      const float h = 0.5f * (float)(R - 1);
      for (int d = 0; d < 3; ++d) {
        empty |= !(umax[d] >= -1.f - 1e-4f) || !(umin[d] <= 1.f + 1e-4f);
        const float slo = (fmaxf(umin[d], -1.f) + 1.f) * h - 1e-3f;
        const float shi = (fminf(umax[d], 1.f) + 1.f) * h + 1e-3f;
        const int clo = min(max((int)floorf(slo), 0), R - 2);
        const int chi = min(max((int)floorf(shi), 0), R - 2);
        bx.lo[d] = clo;
        bx.n[d] = chi - clo + 2;
      }
      if (empty) bx.n[0] = bx.n[1] = bx.n[2] = 0;
      const int nodes = bx.n[0] * bx.n[1] * bx.n[2];
      bx.cells = empty ? 0 : (bx.n[0] - 1) * (bx.n[1] - 1) * (bx.n[2] - 1);
      bx.flags = (!empty && nodes <= cap_nodes && C == 2 ? BOX_STAGED : 0) |
                 (!empty && bx.cells <= capc ? BOX_SCATTER : 0);
      boxes[tid] = bx;
    }
    __syncthreads();
    SRN_PHASE(1);

    const __nv_bfloat16* Fb = md.F16 + (int64_t)b * md.sF;
    const int64_t gsz = (int64_t)R * R * R * C;
    // ---- stage each grid's node box (bf16 x 2 channels, 4 bytes a node) in shared
    //      memory with asynchronous 4-byte copies, one box row per lane
    for (int i = warp; i < M; i += NT / 32) {
      const TileBox bx = boxes[i];
      if (!(bx.flags & BOX_STAGED)) continue;
      const uint32_t dst = su32(sm + L::STG) + (uint32_t)(i * cap_nodes * 4);
      const unsigned int* src = reinterpret_cast<const unsigned int*>(Fb + i * gsz);
      const int rows = bx.n[1] * bx.n[2];
      for (int r = lane; r < rows; r += 32) {
        const int qz = r / bx.n[1], qy = r - qz * bx.n[1];
        const int64_t g0 = ((int64_t)(bx.lo[2] + qz) * R + (bx.lo[1] + qy)) * R + bx.lo[0];
        for (int x = 0; x < bx.n[0]; ++x) cp_async4(dst + 4u * (uint32_t)(r * bx.n[0] + x), src + g0 + x);
      }
    }
    cp_async_wait_all();
    __syncthreads();
    SRN_PHASE(2);

    // ---- encode: Eq. 1 and Eq. 2 for (point p, every other grid)
    {
      const int p = (warp & 3) * 32 + lane, gsub = warp >> 2;
      const float4 pt = reinterpret_cast<const float4*>(xs)[p];
      const bool valid = p < np;
      float rho = 0.f;
#pragma unroll 2
      for (int i = gsub; i < M; i += 2) {
        float ux, uy, uz;
        affine(gs + 12 * i, pt.x, pt.y, pt.z, ux, uy, uz);
        const Cell c = make_cell(ux, uy, uz, R);
        float f0 = 0.f, f1 = 0.f;
        if (valid && c.inside) {
          const TileBox& bx = boxes[i];
          const int lx = c.cx - bx.lo[0], ly = c.cy - bx.lo[1], lz = c.cz - bx.lo[2];
          if ((bx.flags & BOX_STAGED) && lx >= 0 && ly >= 0 && lz >= 0 && lx + 1 < bx.n[0] &&
              ly + 1 < bx.n[1] && lz + 1 < bx.n[2]) {
            const uint32_t* s = reinterpret_cast<const uint32_t*>(sm + L::STG) + i * cap_nodes;
            const int sy = bx.n[0], sz = bx.n[0] * bx.n[1];
            const int o = (lz * bx.n[1] + ly) * bx.n[0] + lx;
            const float2 v0 = unpack_bf16(s[o]), v1 = unpack_bf16(s[o + 1]);
            const float2 v2 = unpack_bf16(s[o + sy]), v3 = unpack_bf16(s[o + sy + 1]);
            const float2 v4 = unpack_bf16(s[o + sz]), v5 = unpack_bf16(s[o + sz + 1]);
            const float2 v6 = unpack_bf16(s[o + sz + sy]), v7 = unpack_bf16(s[o + sz + sy + 1]);
            const float ax = 1.f - c.wx, ay = 1.f - c.wy, az = 1.f - c.wz;
            f0 = az * (ay * (ax * v0.x + c.wx * v1.x) + c.wy * (ax * v2.x + c.wx * v3.x)) +
                 c.wz * (ay * (ax * v4.x + c.wx * v5.x) + c.wy * (ax * v6.x + c.wx * v7.x));
            f1 = az * (ay * (ax * v0.y + c.wx * v1.y) + c.wy * (ax * v2.y + c.wx * v3.y)) +
                 c.wz * (ay * (ax * v4.y + c.wx * v5.y) + c.wy * (ax * v6.y + c.wx * v7.y));
          } else {
            trilinear_bf16(Fb + i * gsz, c, R, C, f0, f1);
          }
        }
        if (C == 2)
          *reinterpret_cast<uint32_t*>(sm + L::Y + swz<K>(p, 2 * i)) = pack_bf16(f0, f1);
        else
          *reinterpret_cast<__nv_bfloat16*>(sm + L::Y + swz<K>(p, i)) = __float2bfloat16_rn(f0);
        if (DENS && valid) rho += dets[i] * flat_top(ux, uy, uz, md.p);
      }
      if (DENS) rhos[gsub * T + p] = rho;
    }
    __syncthreads();
    SRN_PHASE(3);
    if (DENS && tid < np) {
      const float r = rhos[tid] + rhos[T + tid];
      ws.rho[p0 + tid] = r;
      sum_rho += (double)r;
    }

    // ---- decoder forward on tensor cores: rows r0..r0+15 of this warp
    const int r0 = warp * 16;
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
    for (int ks = 0; ks < K / 16; ++ks) {
      uint32_t a[4];
      ldsm4(a, sY + swz<K>(r0 + (lane & 15), ks * 16 + (lane >> 4) * 8));
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t bb[4];
        ldsm4(bb, sW1 + swz<K>(q * 16 + (lane & 7) + ((lane >> 4) << 3), ks * 16 + ((lane >> 3) & 1) * 8));
        mma(acc[2 * q], a, bb[0], bb[1]);
        mma(acc[2 * q + 1], a, bb[2], bb[3]);
      }
    }
    uint32_t h1a[4][4];  // ReLU(z1) as bf16 A fragments of the next layer
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      h1a[kk][0] = pack_bf16(fmaxf(acc[2 * kk][0], 0.f), fmaxf(acc[2 * kk][1], 0.f));
      h1a[kk][1] = pack_bf16(fmaxf(acc[2 * kk][2], 0.f), fmaxf(acc[2 * kk][3], 0.f));
      h1a[kk][2] = pack_bf16(fmaxf(acc[2 * kk + 1][0], 0.f), fmaxf(acc[2 * kk + 1][1], 0.f));
      h1a[kk][3] = pack_bf16(fmaxf(acc[2 * kk + 1][2], 0.f), fmaxf(acc[2 * kk + 1][3], 0.f));
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t bb[4];
        ldsm4(bb, sW2 + swz<64>(q * 16 + (lane & 7) + ((lane >> 4) << 3), kk * 16 + ((lane >> 3) & 1) * 8));
        mma(acc[2 * q], h1a[kk], bb[0], bb[1]);
        mma(acc[2 * q + 1], h1a[kk], bb[2], bb[3]);
      }
    }
    // output layer (64 -> 1) in FP32; rows r0+g8 and r0+g8+8
    float mlo = 0.f, mhi = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const float w = w3s[j * 8 + 2 * t4 + e];
        mlo = fmaf(fmaxf(acc[j][e], 0.f), w, mlo);
        mhi = fmaf(fmaxf(acc[j][2 + e], 0.f), w, mhi);
      }
    }
    mlo += __shfl_xor_sync(0xffffffffu, mlo, 1);
    mlo += __shfl_xor_sync(0xffffffffu, mlo, 2);
    mhi += __shfl_xor_sync(0xffffffffu, mhi, 1);
    mhi += __shfl_xor_sync(0xffffffffu, mhi, 2);
    const int rlo = r0 + g8, rhi = r0 + g8 + 8;
    const float flo = fmaf(mlo, span, vmin), fhi = fmaf(mhi, span, vmin);

    if constexpr (!TRAIN) {
      if (t4 == 0) {
        if (rlo < np) out[p0 + rlo] = flo;
        if (rhi < np) out[p0 + rhi] = fhi;
      }
      __syncthreads();
      SRN_PHASE(4);
      continue;
    } else {
      // ---- L_rec and dL/dm = 2 (f - v) (max - min) / N
      float dmlo, dmhi;
      if (ws.upstream) {  // caller-supplied dL/df: dL/dm = dL/df (max - min)
        dmlo = rlo < np ? xs[4 * rlo + 3] * span : 0.f;
        dmhi = rhi < np ? xs[4 * rhi + 3] * span : 0.f;
      } else {
        const float elo = rlo < np ? flo - xs[4 * rlo + 3] : 0.f;
        const float ehi = rhi < np ? fhi - xs[4 * rhi + 3] : 0.f;
        if (t4 == 0) {
          sum_r2 += (double)elo * elo + (double)ehi * ehi;
          if (rlo < np) ws.herr[p0 + rlo] = elo * elo;
          if (rhi < np) ws.herr[p0 + rhi] = ehi * ehi;
        }
        dmlo = 2.f * elo * span * inv_n;
        dmhi = 2.f * ehi * span * inv_n;
      }
      // dL/dw3, dL/dz2 = dm w3 [z2 > 0]
      uint32_t d2a[4][4];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float d[4];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const float w = w3s[j * 8 + 2 * t4 + e];
          const float hl = fmaxf(acc[j][e], 0.f), hh = fmaxf(acc[j][2 + e], 0.f);
          dw3[j][e] = fmaf(dmlo, hl, fmaf(dmhi, hh, dw3[j][e]));
          d[e] = acc[j][e] > 0.f ? dmlo * w : 0.f;
          d[2 + e] = acc[j][2 + e] > 0.f ? dmhi * w : 0.f;
        }
        d2a[j >> 1][(j & 1) * 2 + 0] = pack_bf16(d[0], d[1]);
        d2a[j >> 1][(j & 1) * 2 + 1] = pack_bf16(d[2], d[3]);
      }
      // H1 and dH2 rows to shared memory for the weight gradients
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int col = j * 8 + 2 * t4;
        *reinterpret_cast<uint32_t*>(sm + L::H1 + swz<64>(rlo, col)) = h1a[j >> 1][(j & 1) * 2];
        *reinterpret_cast<uint32_t*>(sm + L::H1 + swz<64>(rhi, col)) = h1a[j >> 1][(j & 1) * 2 + 1];
        *reinterpret_cast<uint32_t*>(sm + L::DH2 + swz<64>(rlo, col)) = d2a[j >> 1][(j & 1) * 2];
        *reinterpret_cast<uint32_t*>(sm + L::DH2 + swz<64>(rhi, col)) = d2a[j >> 1][(j & 1) * 2 + 1];
      }
      // dL/dz1 = (dz2 W2) [z1 > 0]
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          uint32_t bb[4];
          ldsm4t(bb, sW2 + swz<64>(kk * 16 + (lane & 15), q * 16 + (lane >> 4) * 8));
          mma(acc[2 * q], d2a[kk], bb[0], bb[1]);
          mma(acc[2 * q + 1], d2a[kk], bb[2], bb[3]);
        }
      }
      uint32_t d1a[4][4];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float2 hl = unpack_bf16(h1a[j >> 1][(j & 1) * 2]);
        const float2 hh = unpack_bf16(h1a[j >> 1][(j & 1) * 2 + 1]);
        const uint32_t lo = pack_bf16(hl.x > 0.f ? acc[j][0] : 0.f, hl.y > 0.f ? acc[j][1] : 0.f);
        const uint32_t hi = pack_bf16(hh.x > 0.f ? acc[j][2] : 0.f, hh.y > 0.f ? acc[j][3] : 0.f);
        d1a[j >> 1][(j & 1) * 2] = lo;
        d1a[j >> 1][(j & 1) * 2 + 1] = hi;
        const int col = j * 8 + 2 * t4;
        *reinterpret_cast<uint32_t*>(sm + L::DH1 + swz<64>(rlo, col)) = lo;
        *reinterpret_cast<uint32_t*>(sm + L::DH1 + swz<64>(rhi, col)) = hi;
      }
      // dL/dy = dz1 W1 (FP32 to shared memory), 32 columns at a time
#pragma unroll
      for (int nc = 0; nc < NTY; nc += 4) {
        float a4[4][4];
#pragma unroll
        for (int j = 0; j < 4; ++j) a4[j][0] = a4[j][1] = a4[j][2] = a4[j][3] = 0.f;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            if (nc + 2 * q < NTY) {
              uint32_t bb[4];
              ldsm4t(bb, sW1 + swz<K>(kk * 16 + (lane & 15), (nc + 2 * q) * 8 + (lane >> 4) * 8));
              mma(a4[2 * q], d1a[kk], bb[0], bb[1]);
              mma(a4[2 * q + 1], d1a[kk], bb[2], bb[3]);
            }
          }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (nc + j < NTY) {
            const int col = (nc + j) * 8 + 2 * t4;
            *reinterpret_cast<float2*>(dys + rlo * L::DYS + col) = make_float2(a4[j][0], a4[j][1]);
            *reinterpret_cast<float2*>(dys + rhi * L::DYS + col) = make_float2(a4[j][2], a4[j][3]);
          }
        }
      }
      __syncthreads();
      SRN_PHASE(4);

      // ---- dW2 += dz2^T H1 and dW1 += dz1^T Y over the tile's 128 points
      {
        const int mt = warp & 3, nb2 = (warp >> 2) * 32, nb1 = (warp >> 2) * (K / 2);
#pragma unroll 2
        for (int ks = 0; ks < T / 16; ++ks) {
          const int arow = ks * 16 + (lane & 7) + ((lane >> 4) << 3);
          const int acol = mt * 16 + ((lane >> 3) & 1) * 8;
          uint32_t a[4];
          ldsm4t(a, sDH2 + swz<64>(arow, acol));
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            uint32_t bb[4];
            ldsm4t(bb, sH1 + swz<64>(ks * 16 + (lane & 15), nb2 + q * 16 + (lane >> 4) * 8));
            mma(dw2[2 * q], a, bb[0], bb[1]);
            mma(dw2[2 * q + 1], a, bb[2], bb[3]);
          }
          ldsm4t(a, sDH1 + swz<64>(arow, acol));
          if constexpr (NW1 >= 2) {
#pragma unroll
            for (int q = 0; q < NW1 / 2; ++q) {
              uint32_t bb[4];
              ldsm4t(bb, sY + swz<K>(ks * 16 + (lane & 15), nb1 + q * 16 + (lane >> 4) * 8));
              mma(dw1[2 * q], a, bb[0], bb[1]);
              mma(dw1[2 * q + 1], a, bb[2], bb[3]);
            }
          } else {
            uint32_t bb[2];
            ldsm2t(bb, sY + swz<K>(ks * 16 + (lane & 15), nb1));
            mma(dw1[0], a, bb[0], bb[1]);
          }
        }
      }

      __syncthreads();  // Y..DH1 become the scatter scratch
      SRN_PHASE(5);

      // ---- scatter dL/dy into the gradient grids (adjoint of Eq. 2).  Warp w owns
      //      grids w, w+8, ...: it counting-sorts the tile's points by their cell in
      //      the grid's box (integer shared-memory atomics), sums each cell's eight
      //      corner contributions with plain FMAs, then adds every box node into the
      //      float32 gradient grid with one float2 atomic.  Points whose cell falls
      //      outside a usable box add their corners directly.
      {
        unsigned char* scr = sm + L::SCR + warp * L::SCR_WARP;
        float* cs = reinterpret_cast<float*>(scr);                       // [capc][8C]
        int* cnt = reinterpret_cast<int*>(scr + capc * 32 * C);          // [capc + 1]
        unsigned short* perm = reinterpret_cast<unsigned short*>(cnt + capc + 1);  // [T]
        float* wts = reinterpret_cast<float*>(scr + L::SCR_WARP - T * 12 - T * 2);  // [T][3]
        short* cid = reinterpret_cast<short*>(scr + L::SCR_WARP - T * 2);          // [T]
        float* dFb = gr.dF + (int64_t)b * gr.sF;
        for (int i = warp; i < M; i += NT / 32) {
          const TileBox bx = boxes[i];
          float* dFi = dFb + i * gsz;
          const bool boxed = (bx.flags & BOX_SCATTER) != 0;
          const int cx = bx.n[0] - 1, cy = bx.n[1] - 1;
          int rk[T / 32];
          // (a) cell of each point in the box (or a direct scatter)
#pragma unroll
          for (int j = 0; j < T / 32; ++j) {
            const int p = lane + 32 * j;
            rk[j] = -1;
            short id = -1;
            if (p < np) {
              const float4 pt = reinterpret_cast<const float4*>(xs)[p];
              float ux, uy, uz;
              affine(gs + 12 * i, pt.x, pt.y, pt.z, ux, uy, uz);
              const Cell c = make_cell(ux, uy, uz, R);
              float g0, g1 = 0.f;
              if (C == 2) {
                const float2 g = *reinterpret_cast<const float2*>(dys + p * L::DYS + 2 * i);
                g0 = g.x; g1 = g.y;
              } else {
                g0 = dys[p * L::DYS + i];
              }
              if (c.inside && (g0 != 0.f || g1 != 0.f)) {
                const int lx = c.cx - bx.lo[0], ly = c.cy - bx.lo[1], lz = c.cz - bx.lo[2];
                if (boxed && lx >= 0 && ly >= 0 && lz >= 0 && lx < cx && ly < cy && lz < bx.n[2] - 1) {
                  id = (short)((lz * cy + ly) * cx + lx);
                  wts[3 * p] = c.wx; wts[3 * p + 1] = c.wy; wts[3 * p + 2] = c.wz;
                } else {
                  scatter_f32(dFi, c, R, C, g0, g1);
                }
              }
            }
            if (p < T) cid[p] = id;
          }
          if (!boxed) continue;  // warp-uniform
          // (b) counting sort of the points by cell
          for (int l = lane; l <= bx.cells; l += 32) cnt[l] = 0;
          __syncwarp();
#pragma unroll
          for (int j = 0; j < T / 32; ++j) {
            const int id = cid[lane + 32 * j];
            if (id >= 0) rk[j] = atomicAdd(cnt + id, 1);
          }
          __syncwarp();
          {
            const int per = (bx.cells + 31) / 32;
            const int l0 = lane * per;
            int run = 0;
            for (int l = l0; l < min(l0 + per, bx.cells); ++l) run += cnt[l];
            int incl = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
              const int v = __shfl_up_sync(0xffffffffu, incl, o);
              if (lane >= o) incl += v;
            }
            int acc = incl - run;
            __syncwarp();
            for (int l = l0; l < min(l0 + per, bx.cells); ++l) {
              const int v = cnt[l];
              cnt[l] = acc;
              acc += v;
            }
            if (lane == 31) cnt[bx.cells] = incl;
          }
          __syncwarp();
#pragma unroll
          for (int j = 0; j < T / 32; ++j) {
            const int p = lane + 32 * j;
            if (rk[j] >= 0) perm[cnt[cid[p]] + rk[j]] = (unsigned short)p;
          }
          __syncwarp();
          // (c) per cell: the eight corner sums of its points
          for (int l = lane; l < bx.cells; l += 32) {
            float a[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) a[k] = 0.f;
            for (int s = cnt[l]; s < cnt[l + 1]; ++s) {
              const int p = perm[s];
              const float wx = wts[3 * p], wy = wts[3 * p + 1], wz = wts[3 * p + 2];
              const float ax = 1.f - wx, ay = 1.f - wy, az = 1.f - wz;
              const float w[8] = {az * ay * ax, az * ay * wx, az * wy * ax, az * wy * wx,
                                  wz * ay * ax, wz * ay * wx, wz * wy * ax, wz * wy * wx};
              if (C == 2) {
                const float2 g = *reinterpret_cast<const float2*>(dys + p * L::DYS + 2 * i);
#pragma unroll
                for (int k = 0; k < 8; ++k) { a[2 * k] = fmaf(w[k], g.x, a[2 * k]); a[2 * k + 1] = fmaf(w[k], g.y, a[2 * k + 1]); }
              } else {
                const float g = dys[p * L::DYS + i];
#pragma unroll
                for (int k = 0; k < 8; ++k) a[k] = fmaf(w[k], g, a[k]);
              }
            }
            float* o = cs + l * 8 * C;
            if (C == 2) {
#pragma unroll
              for (int k = 0; k < 4; ++k)
                reinterpret_cast<float4*>(o)[k] = make_float4(a[4 * k], a[4 * k + 1], a[4 * k + 2], a[4 * k + 3]);
            } else {
#pragma unroll
              for (int k = 0; k < 2; ++k)
                reinterpret_cast<float4*>(o)[k] = make_float4(a[4 * k], a[4 * k + 1], a[4 * k + 2], a[4 * k + 3]);
            }
          }
          __syncwarp();
          // (d) every node of the box gathers the corner sums of its (up to) 8 cells
          const int rows = bx.n[1] * bx.n[2];
          for (int r = lane; r < rows; r += 32) {
            const int qz = r / bx.n[1], qy = r - qz * bx.n[1];
            const int64_t g0 = ((int64_t)(bx.lo[2] + qz) * R + (bx.lo[1] + qy)) * R + bx.lo[0];
            for (int qx = 0; qx < bx.n[0]; ++qx) {
              float v0 = 0.f, v1 = 0.f;
#pragma unroll
              for (int k = 0; k < 8; ++k) {
                const int ex = qx - (k & 1), ey = qy - ((k >> 1) & 1), ez = qz - (k >> 2);
                if (ex >= 0 && ey >= 0 && ez >= 0 && ex < cx && ey < cy && ez < bx.n[2] - 1) {
                  const float* s = cs + ((ez * cy + ey) * cx + ex) * 8 * C + k * C;
                  v0 += s[0];
                  if (C == 2) v1 += s[1];
                }
              }
              if (v0 != 0.f || v1 != 0.f) {
                if (C == 2) atomicAdd(reinterpret_cast<float2*>(dFi) + g0 + qx, make_float2(v0, v1));
                else atomicAdd(dFi + g0 + qx, v0);
              }
            }
          }
          __syncwarp();
        }
      }
      __syncthreads();
      SRN_PHASE(6);
    }
  }
  if constexpr (TRAIN) {
    if (cur >= 0) flush(cur);
  }
  SRN_PHASE(7);
}

template <int K, int MODE>
cudaError_t launch_k(const Launch& L, const Model& md, const Grads& gr, const Bricks& br,
                     const TrainWs& ws, const float* xyz, const float* target, float* out) {
  const int smem = Lay<K>::BYTES;
  auto kern = k_query_bf16<K, MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int grid = L.num_sms;
  if (!br.dev) {
    int total = 0;
    for (int b = 0; b < br.n; ++b) total += (int)((br.off[b + 1] - br.off[b] + T - 1) / T);
    if (total == 0) return cudaSuccess;
    grid = total < L.num_sms ? total : L.num_sms;
  }
  kern<<<grid, NT, smem, L.stream>>>(md, gr, br, ws, xyz, target, out);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_mode(const Launch& L, const Model& md, const Grads& gr, const Bricks& br,
                        const TrainWs& ws, const float* xyz, const float* target, float* out) {
  switch (md.K) {
    case 16: return launch_k<16, MODE>(L, md, gr, br, ws, xyz, target, out);
    case 32: return launch_k<32, MODE>(L, md, gr, br, ws, xyz, target, out);
    case 64: return launch_k<64, MODE>(L, md, gr, br, ws, xyz, target, out);
    case 128: return launch_k<128, MODE>(L, md, gr, br, ws, xyz, target, out);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_query_bf16(const Launch& L, QueryMode mode, const Model& md, const Grads& gr,
                              const Bricks& br, const TrainWs& ws, const float* xyz,
                              const float* target, float* out) {
  switch (mode) {
    case kForward: return launch_mode<kForward>(L, md, gr, br, ws, xyz, target, out);
    case kTrain: return launch_mode<kTrain>(L, md, gr, br, ws, xyz, target, out);
    default: return launch_mode<kTrainDensity>(L, md, gr, br, ws, xyz, target, out);
  }
}

}  // namespace srn
