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
  static constexpr int BYTES = DET + kMaxGrids * 4;
};

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

    // ---- points (and targets) of the tile
    if (tid < T) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (tid < np) {
        const float* q = xyz + 3 * (p0 + tid);
        v.x = q[0]; v.y = q[1]; v.z = q[2];
        if (TRAIN) v.w = target[p0 + tid];
      }
      reinterpret_cast<float4*>(xs)[tid] = v;
    }
    __syncthreads();

    // ---- encode: Eq. 1 and Eq. 2 for (point p, every other grid)
    const __nv_bfloat16* Fb = md.F16 + (int64_t)b * md.sF;
    const int64_t gsz = (int64_t)R * R * R * C;
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
        if (valid && c.inside) trilinear_bf16(Fb + i * gsz, c, R, C, f0, f1);
        if (C == 2)
          *reinterpret_cast<uint32_t*>(sm + L::Y + swz<K>(p, 2 * i)) = pack_bf16(f0, f1);
        else
          *reinterpret_cast<__nv_bfloat16*>(sm + L::Y + swz<K>(p, i)) = __float2bfloat16_rn(f0);
        if (DENS && valid) rho += dets[i] * flat_top(ux, uy, uz, md.p);
      }
      if (DENS) rhos[gsub * T + p] = rho;
    }
    __syncthreads();
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

      // ---- scatter dL/dy into the gradient grids (adjoint of Eq. 2)
      {
        const int p = (warp & 3) * 32 + lane, gsub = warp >> 2;
        if (p < np) {
          const float4 pt = reinterpret_cast<const float4*>(xs)[p];
          float* dFb = gr.dF + (int64_t)b * gr.sF;
          for (int i = gsub; i < M; i += 2) {
            float ux, uy, uz;
            affine(gs + 12 * i, pt.x, pt.y, pt.z, ux, uy, uz);
            const Cell c = make_cell(ux, uy, uz, R);
            if (!c.inside) continue;
            float g0, g1 = 0.f;
            if (C == 2) {
              const float2 g = *reinterpret_cast<const float2*>(dys + p * L::DYS + 2 * i);
              g0 = g.x; g1 = g.y;
            } else {
              g0 = dys[p * L::DYS + i];
            }
            if (g0 == 0.f && g1 == 0.f) continue;
            scatter_f32(dFb + i * gsz, c, R, C, g0, g1);
          }
        }
      }
      __syncthreads();
    }
  }
  if constexpr (TRAIN) {
    if (cur >= 0) flush(cur);
  }
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
