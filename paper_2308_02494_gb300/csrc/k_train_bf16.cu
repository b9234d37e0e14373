// BF16 training pass over all bricks: three kernels, each shaped for its own bound.
//
//  k_enc   encoder (Eq. 1-3) over the same tiles as k_scat, as (tile, group of 32
//          grids) units, two CTAs per SM: each unit's node boxes of the BF16 grids
//          are staged in shared memory as float32 (one column per lane), the corners
//          read and blended as packed f32x2.  Writes the features Y [N][K] (bf16).
//          rho of Eq. 7 is a pass of its own (k_density_rho).
//  k_mlp   decoder forward and backward for K < 128 on the tensor cores (mma.sync
//          m16n8k16, BF16 operands, FP32 accumulation): L_rec partial sums,
//          h(x) = (f - v)^2, dW1/dW2/dw3 accumulated in registers per CTA and flushed
//          once, and dL/dy written point-major as bf16 (dY [N][M][C], like Y).
//          K = 128 runs on tcgen05 instead (k_mlp_tc.cu).
//  k_scat  adjoint of Eq. 2.  A tile is up to tile_points (<= 1024) points of one brick
//          lying in one aligned Morton range of the sampler's bins (a small
//          axis-aligned block of the brick), listed by k_unit_starts / k_tile_list.
//          Two CTAs per SM take (tile, group of 32 grids) units.  Lane l of a warp
//          takes grid l of the group: the block, mapped through the grid's Eq. 1,
//          bounds a node box that the tile's level keeps within shared memory, and the
//          warp adds one point's eight corners into 32 grids' boxes at once, as 32-bit
//          fixed-point integers (a power-of-two scale per grid and tile from a bound on
//          its largest |dL/dy|: for K = 128 the decoder's maxima per 128 points) with
//          shared-memory integer reductions, one bank per lane.
//          Each box node then goes into the float32 gradient grid with one atomic.
//          Points outside their tile's box (rounding at its faces; a batch that is not
//          Morton-sorted) add their corners directly.
#include "enc_ops.cuh"
#include "kernels.h"
#include <algorithm>
#include <climits>
#include <cmath>
#include <type_traits>

namespace srn {
namespace {

template <typename Tv>
__device__ __forceinline__ Tv warp_sum(Tv v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int ET = 128;   // points per decoder tile (k_mlp, k_mlp_tc)

// =============================================================================== k_mlp
constexpr int T = 128;
constexpr int NT = 256;

template <int K>
struct MlpLay {
  static constexpr int DYS = K + 2;                    // dL/dy row pitch (floats)
  static constexpr int W1 = 0;                         // [64][K] bf16 swizzled
  static constexpr int W2 = W1 + 64 * K * 2;           // [64][64] bf16
  static constexpr int Y = W2 + 64 * 64 * 2;           // [T][K] bf16 features
  static constexpr int H1 = Y + T * K * 2;             // [T][64] bf16 ReLU(z1)
  static constexpr int DH2 = H1 + T * 64 * 2;          // [T][64] bf16 dL/dz2
  static constexpr int DH1 = DH2 + T * 64 * 2;         // [T][64] bf16 dL/dz1
  static constexpr int DY = DH1 + T * 64 * 2;          // [T][DYS] f32 dL/dy
  static constexpr int W3 = DY + T * DYS * 4;          // [64] f32
  static constexpr int V = W3 + 64 * 4;                // [T] f32 targets (or dL/df)
  static constexpr int BYTES = V + T * 4;
};

template <int K>
__global__ void __launch_bounds__(NT, 1)
k_mlp(Model md, Grads gr, Bricks brp, TrainWs ws, const float* __restrict__ target) {
  constexpr int NW1 = K / 16;
  constexpr int NTY = K / 8;
  using L = MlpLay<K>;
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ TileMap tm;
  __shared__ Bricks br;
  load_bricks(brp, br);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g8 = lane >> 2, t4 = lane & 3;
  const int M = md.M, C = md.C;
  if (tid == 0) build_tile_map(br, T, tm);
  __syncthreads();
  const int total = tm.first[br.n];
  const int per = (total + gridDim.x - 1) / gridDim.x;
  const int tb = blockIdx.x * per, te = min(total, tb + per);
  float* w3s = reinterpret_cast<float*>(sm + L::W3);
  float* vs = reinterpret_cast<float*>(sm + L::V);
  float* dys = reinterpret_cast<float*>(sm + L::DY);
  const uint32_t sW1 = su32(sm + L::W1), sW2 = su32(sm + L::W2), sY = su32(sm + L::Y);
  const uint32_t sH1 = su32(sm + L::H1), sDH2 = su32(sm + L::DH2), sDH1 = su32(sm + L::DH1);

  float dw1[NW1][4], dw2[4][4], dw3[8][2];
  double sum_r2 = 0.0;
#pragma unroll
  for (int i = 0; i < NW1; ++i) dw1[i][0] = dw1[i][1] = dw1[i][2] = dw1[i][3] = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) dw2[i][0] = dw2[i][1] = dw2[i][2] = dw2[i][3] = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) dw3[i][0] = dw3[i][1] = 0.f;

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
    const double s = warp_sum(sum_r2);
    if (lane == 0) atomicAdd(ws.acc + b * kAccPerBrick + ACC_SUM_R2, s);
    sum_r2 = 0.0;
  };

  int cur = -1;
  float span = 0.f, vmin = 0.f, inv_n = 0.f;
  for (int tile = tb; tile < te; ++tile) {
    const int b = brick_of_tile(tm, br.n, tile, cur);
    if (b != cur) {
      if (cur >= 0) flush(cur);
      __syncthreads();
      cur = b;
      const uint4* w1 = reinterpret_cast<const uint4*>(md.W1h + (int64_t)b * md.sW1);
      for (int c = tid; c < 64 * K / 8; c += NT)
        *reinterpret_cast<uint4*>(sm + L::W1 + swz<K>(c / (K / 8), (c % (K / 8)) * 8)) = w1[c];
      const uint4* w2 = reinterpret_cast<const uint4*>(md.W2h + (int64_t)b * md.sW2);
      for (int c = tid; c < 64 * 8; c += NT)
        *reinterpret_cast<uint4*>(sm + L::W2 + swz<64>(c / 8, (c % 8) * 8)) = w2[c];
      if (tid < 64) w3s[tid] = md.w3[(int64_t)b * md.sw3 + tid];
      vmin = md.range[2 * b];
      span = md.range[2 * b + 1] - vmin;
      inv_n = 1.f / (float)(br.off[b + 1] - br.off[b]);
      __syncthreads();
    }
    const int64_t p0 = br.off[b] + (int64_t)(tile - tm.first[b]) * T;
    const int np = (int)min((int64_t)T, br.off[b + 1] - p0);
    // ---- the tile's features (16-byte asynchronous copies; rows past np zero-filled)
    for (int c = tid; c < T * (K / 8); c += NT) {
      const int row = c / (K / 8), ch = c % (K / 8);
      const int valid = row < np;
      const __nv_bfloat16* src = ws.Y + (valid ? (p0 + row) * K + ch * 8 : 0);
      cp_async16(sY + swz<K>(row, ch * 8), src, valid ? 16 : 0);
    }
    if (tid < T) vs[tid] = tid < np ? target[p0 + tid] : 0.f;
    cp_async_wait_all();
    __syncthreads();

    // ---- decoder forward: rows r0..r0+15 of this warp
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
    uint32_t h1a[4][4];
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
    float dmlo, dmhi;
    if (ws.upstream) {  // caller-supplied dL/df: dL/dm = dL/df (max - min)
      dmlo = rlo < np ? vs[rlo] * span : 0.f;
      dmhi = rhi < np ? vs[rhi] * span : 0.f;
    } else {  // L_rec: dL/dm = 2 (f - v) (max - min) / N
      const float elo = rlo < np ? fmaf(mlo, span, vmin) - vs[rlo] : 0.f;
      const float ehi = rhi < np ? fmaf(mhi, span, vmin) - vs[rhi] : 0.f;
      if (t4 == 0) {
        sum_r2 += (double)elo * elo + (double)ehi * ehi;
        if (rlo < np) ws.herr[p0 + rlo] = elo * elo;
        if (rhi < np) ws.herr[p0 + rhi] = ehi * ehi;
      }
      dmlo = 2.f * elo * span * inv_n;
      dmhi = 2.f * ehi * span * inv_n;
    }
    // ---- decoder backward
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
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int col = j * 8 + 2 * t4;
      *reinterpret_cast<uint32_t*>(sm + L::H1 + swz<64>(rlo, col)) = h1a[j >> 1][(j & 1) * 2];
      *reinterpret_cast<uint32_t*>(sm + L::H1 + swz<64>(rhi, col)) = h1a[j >> 1][(j & 1) * 2 + 1];
      *reinterpret_cast<uint32_t*>(sm + L::DH2 + swz<64>(rlo, col)) = d2a[j >> 1][(j & 1) * 2];
      *reinterpret_cast<uint32_t*>(sm + L::DH2 + swz<64>(rhi, col)) = d2a[j >> 1][(j & 1) * 2 + 1];
    }
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
    // ---- dW2 += dz2^T H1 and dW1 += dz1^T Y over the tile
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
    // ---- dL/dy to global memory, point-major bf16: dY[p][i][c]
    for (int idx = tid; idx < M * T; idx += NT) {
      const int p = idx / M, i = idx % M;
      if (p < np) {
        const int64_t o = (p0 + p) * M + i;
        if (C == 2) {
          const float2 g = *reinterpret_cast<const float2*>(dys + p * L::DYS + 2 * i);
          reinterpret_cast<uint32_t*>(ws.dY)[o] = pack_bf16(g.x, g.y);
        } else {
          ws.dY[o] = __float2bfloat16_rn(dys[p * L::DYS + i]);
        }
      }
    }
    __syncthreads();
  }
  if (cur >= 0) flush(cur);
}

// =============================================================================== k_scat
constexpr int ST = kMaxTilePoints;   // Morton-consecutive points per tile (at most)
constexpr int SNT = 512;        // threads of k_enc (two CTAs per SM)
constexpr int SNW = SNT / 32;
constexpr int SCT = 256;        // threads of k_scat (two CTAs per SM)
constexpr int SCW = SCT / 32;

// Head of k_scat's dynamic shared memory; the unit's fixed-point node boxes follow it,
// [node][channel][32 columns] int32 (see ScatMap).
struct ScatHead {
  float4 xs[ST];               // the tile's points
  uint2 box[32];               // node box of the tile's block per grid of the unit: lo | nodes per axis (bytes)
  uint32_t gmax[32];           // largest |dL/dy| of the tile per grid of the unit (bf16 bits)
  ScatTile tile, tnext;         // this unit's tile, and the next unit's (taken one ahead)
  int grp, gnext;               // their column groups
};

// Thread -> grid, column group and point group of a unit of k_scat or k_enc (unit_map).
// A grid group's boxes are stored node by node with one column per lane, so the 32
// shared-memory accesses of a warp instruction fall in distinct banks.
struct ScatMap {
  int g, grp, pg, npg;
};
// The units of k_scat and k_enc are (tile, column group): with M >= 32 a CTA of NW
// warps takes the 32 grids of group grp and its warps split the tile's points; with
// M < 32 (one group) lane l takes grid l mod M and a warp 32/M points at a time.
template <int NW>
__device__ __forceinline__ ScatMap unit_map(int M, int grp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  ScatMap m;
  if (M >= 32) {
    m.grp = grp;
    m.g = grp * 32 + lane;
    m.pg = warp;
    m.npg = NW;
  } else {
    m.grp = 0;
    m.g = lane % M;
    m.pg = warp * (32 / M) + lane / M;
    m.npg = NW * (32 / M);
  }
  return m;
}

// Power-of-two scale of one grid's fixed-point sums over a tile of np points whose
// largest |dL/dy| has bf16 bits mb: every product w g scale stays below 2^B <= 2^22 in
// magnitude (so kMagic rounds it exactly) and every node's sum below np 2^B <= 2^30
// (each point adds at most |g| to a node).  inv = 1 / scale exactly.
__device__ __forceinline__ float fixed_scale(uint32_t mb, int np, float& inv) {
  const int lognp = 32 - __clz(max(np - 1, 1));   // ceil(log2 np)
  const int B = min(22, 30 - lognp);
  const int ef = (int)((mb >> 7) & 0xffu);          // biased exponent: max|g| < 2^(ef - 126)
  const int sb = min(B + 253 - ef, 250);            // scale = 2^(sb - 127) <= 2^(B + 126 - ef)
  inv = __int_as_float((254 - sb) << 23);
  return __int_as_float(sb << 23);
}
__device__ __forceinline__ int32_t fixed_pt(float w, float gs) {
  return __float_as_int(fmaf(w, gs, kMagic)) - kMagicBits;
}
template <int OFF>
__device__ __forceinline__ void red_s32(uint32_t a, int32_t v) {
  asm volatile("red.shared.add.u32 [%0+%2], %1;" ::"r"(a), "r"(v), "n"(OFF));
}
// The two x-neighbour corners (weights wa at x, wb at x + 1) of one (y, z) corner pair.
template <int C>
__device__ __forceinline__ void red_pair(uint32_t a, float wa, float wb, float gs0, float gs1) {
  red_s32<0>(a, fixed_pt(wa, gs0));
  red_s32<C * 128>(a, fixed_pt(wb, gs0));
  if constexpr (C == 2) {
    red_s32<128>(a, fixed_pt(wa, gs1));
    red_s32<C * 128 + 128>(a, fixed_pt(wb, gs1));
  }
}

// The 8 corners x C channels of one (point, grid) whose cell lies in the box: corner
// (i, j, k) of the cell at a0 (+ i node, + j oy, + k oz) gets round(Wx_i Wy_j Wz_k g scale)
// for each channel g of dL/dy (bf16 bits d), the products formed channel pairs at a time
// as ((g scale) Wz_k) Wy_j, and the Wx_i factor fused into the rounding FMA.
template <int C>
__device__ __forceinline__ void red_cell(uint32_t a0, uint32_t oy, uint32_t oz, float wx, float wy, float wz,
                                         uint32_t d, float scale) {
  if constexpr (C == 2) {
    const unsigned long long one = f2_bits(1.f, 1.f), mm = f2_bits(kMagic, kMagic);
    const unsigned long long wx2 = f2_bits(wx, wx), wy2 = f2_bits(wy, wy), wz2 = f2_bits(wz, wz);
    unsigned long long ax2, ay2, az2;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(ax2) : "l"(one), "l"(wx2));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(ay2) : "l"(one), "l"(wy2));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(az2) : "l"(one), "l"(wz2));
    const unsigned long long gs = mul2(bf2_bits(d), f2_bits(scale, scale));
    const unsigned long long z0 = mul2(az2, gs), z1 = mul2(wz2, gs);
    const unsigned long long yz[4] = {mul2(ay2, z0), mul2(wy2, z0), mul2(ay2, z1), mul2(wy2, z1)};
    const uint32_t a[4] = {a0, a0 + oy, a0 + oz, a0 + oy + oz};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const unsigned long long va = fma2(ax2, yz[j], mm), vb = fma2(wx2, yz[j], mm);
      red_s32<0>(a[j], (int32_t)(uint32_t)va - kMagicBits);
      red_s32<128>(a[j], (int32_t)(uint32_t)(va >> 32) - kMagicBits);
      red_s32<256>(a[j], (int32_t)(uint32_t)vb - kMagicBits);
      red_s32<384>(a[j], (int32_t)(uint32_t)(vb >> 32) - kMagicBits);
    }
  } else {
    const float ax = 1.f - wx, ay = 1.f - wy, az = 1.f - wz;
    const float zy0 = az * ay, zy1 = az * wy, zy2 = wz * ay, zy3 = wz * wy;
    const float gs0 = __uint_as_float(d << 16) * scale;
    red_pair<C>(a0, zy0 * ax, zy0 * wx, gs0, 0.f);
    red_pair<C>(a0 + oy, zy1 * ax, zy1 * wx, gs0, 0.f);
    red_pair<C>(a0 + oz, zy2 * ax, zy2 * wx, gs0, 0.f);
    red_pair<C>(a0 + oy + oz, zy3 * ax, zy3 * wx, gs0, 0.f);
  }
}

// dL/dy of point p (global index) for grid g: C bf16 values in the low bits.
template <int C>
__device__ __forceinline__ uint32_t dy_bits(const __nv_bfloat16* dY, int64_t p, int M, int g) {
  if constexpr (C == 2) return __ldg(reinterpret_cast<const unsigned int*>(dY) + p * M + g);
  else return (uint32_t)__ldg(reinterpret_cast<const unsigned short*>(dY) + p * M + g);
}

// First point of every Morton unit (2 x 2 x 2 bins) that starts a run of that unit in
// each brick's batch; the other entries keep the -1 they were cleared to.
__global__ void k_unit_starts(Bricks brp, const float* __restrict__ xyz, int32_t* __restrict__ ustart) {
  __shared__ Bricks br;
  load_bricks(brp, br);
  __syncthreads();
  const int b = blockIdx.y;
  const int64_t o = br.off[b], n = br.off[b + 1] - o;
  int32_t* us = ustart + (int64_t)b * (kUnits + 1);
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const float* q = xyz + 3 * (o + p);
    const uint32_t u = morton_bin(q[0], q[1], q[2]) >> 3;
    if (p == 0 || (morton_bin(q[-3], q[-2], q[-1]) >> 3) != u) us[u] = (int32_t)p;
  }
}

// One CTA per brick.  The brick's largest tile level lmax is the largest L <= lcap whose
// block, mapped through any of the brick's grids, has a node box of at most capn nodes:
// per grid axis, the image's extent in cells plus the box margin, one partial cell at
// each end and the node past the last cell bound tile_box's count (0 when even one unit
// is too large; such grids add their corners directly).  Units without a recorded start
// take the next recorded one (a suffix minimum; for a sorted batch this is exact, for any
// batch the starts become non-decreasing from 0 to n, so the tiles below always partition
// the brick's points).  Every unit then belongs to the largest aligned range of 2^L units
// (L <= lmax) holding at most tp (<= ST) points; each such range becomes ceil(points / tp)
// tiles of consecutive points.
__global__ void __launch_bounds__(1024) k_tile_list(Bricks brp, TrainWs ws, Model md, int capn, int lcap,
                                                    int tp) {
  constexpr int UPT = kUnits / 1024;
  __shared__ Bricks br;
  __shared__ int32_t st[kUnits + 1];
  __shared__ int32_t wred[32];
  __shared__ int32_t gbase;
  __shared__ int32_t s_lv;
  if (threadIdx.x == 0) s_lv = lcap;
  load_bricks(brp, br);
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < md.M) {
    const float* g = md.G + (int64_t)b * md.sG + 12 * tid;
    const float hs = 0.5f * (float)(md.R - 1) * (2.f / (float)(1 << kUnitBits));   // cells per unit
    int lv = 0;
    for (int L = lcap; L > 0; --L) {
      const float ext[3] = {(float)(1 << ((L + 2) / 3)), (float)(1 << ((L + 1) / 3)), (float)(1 << (L / 3))};
      int nodes = 1;
      for (int d = 0; d < 3; ++d) {
        const float e = (fabsf(g[4 * d]) * ext[0] + fabsf(g[4 * d + 1]) * ext[1] + fabsf(g[4 * d + 2]) * ext[2]) * hs;
        nodes *= min((int)ceilf(e + 0.01f) + 2, md.R);
      }
      if (nodes <= capn) { lv = L; break; }
    }
    atomicMin(&s_lv, lv);
  }
  __syncthreads();
  const int lmax = s_lv;
  const int64_t o = br.off[b];
  const int32_t n = (int32_t)(br.off[b + 1] - o);
  const int32_t* us = ws.ustart + (int64_t)b * (kUnits + 1);
  int32_t loc[UPT];
  {
    int32_t m = INT_MAX;
#pragma unroll
    for (int k = UPT - 1; k >= 0; --k) {
      // a batch from the sampler: unit u starts where its first bin starts
      const int32_t v = ws.bin_start ? (int32_t)ws.bin_start[(int64_t)b * kSortBins + ((tid * UPT + k) << 3)]
                                     : us[tid * UPT + k];
      if (v >= 0) m = min(m, v);
      loc[k] = m;
    }
    int32_t incl = loc[0];   // suffix minimum over lanes >= lane
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int32_t y = __shfl_down_sync(0xffffffffu, incl, d);
      if (lane + d < 32) incl = min(incl, y);
    }
    if (lane == 0) wred[warp] = incl;
    __syncthreads();
    int32_t after = n;
    for (int q = warp + 1; q < 32; ++q) after = min(after, wred[q]);
    const int32_t next = __shfl_down_sync(0xffffffffu, incl, 1);
    const int32_t excl = lane < 31 ? min(next, after) : after;
#pragma unroll
    for (int k = 0; k < UPT; ++k) st[tid * UPT + k] = min(loc[k], excl);
    // the first point always opens a tile: in a batch that is not sorted, later points
    // of its unit may have overwritten its recorded start
    if (tid == 0) { st[0] = 0; st[kUnits] = n; }
  }
  __syncthreads();
  int nt[UPT], lv[UPT];
  int tot = 0;
#pragma unroll
  for (int k = 0; k < UPT; ++k) {
    const int u = tid * UPT + k;
    int L = 0;
    for (int l = lmax; l > 0; --l) {
      const int a = u & ~((1 << l) - 1);
      if (st[a + (1 << l)] - st[a] <= tp) { L = l; break; }
    }
    lv[k] = L;
    nt[k] = 0;
    if ((u & ((1 << L) - 1)) == 0) nt[k] = (st[u + (1 << L)] - st[u] + tp - 1) / tp;
    tot += nt[k];
  }
  int incl = tot;   // block-wide exclusive scan of the tile counts
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += y;
  }
  __syncthreads();
  if (lane == 31) wred[warp] = incl;
  __syncthreads();
  int base = incl - tot, all = 0;
  for (int q = 0; q < 32; ++q) {
    if (q < warp) base += wred[q];
    all += wred[q];
  }
  if (tid == 0) gbase = atomicAdd(ws.tile_ctr, all);
  __syncthreads();
  int idx = gbase + base;
#pragma unroll
  for (int k = 0; k < UPT; ++k) {
    const int u = tid * UPT + k;
    const int c = nt[k] ? st[u + (1 << lv[k])] - st[u] : 0;
    for (int t = 0; t < nt[k]; ++t, ++idx) {
      ScatTile T;
      T.start = o + st[u] + (int64_t)t * c / nt[k];
      T.count = (int32_t)((int64_t)(t + 1) * c / nt[k] - (int64_t)t * c / nt[k]);
      T.code = (uint32_t)b << 20 | (uint32_t)lv[k] << 16 | (uint32_t)u;
      ws.tiles[idx] = T;
    }
  }
}

// Node box of the tile's block (units [u0, u0 + 2^L)) in grid g, padded by a small
// margin in s against rounding; returned as bytes lo[3] | n[3] (n = 0: no point of the
// block is inside the grid).
__device__ uint2 tile_box(uint32_t code, const float* __restrict__ g, int R) {
  const int L = (code >> 16) & 15;
  const uint32_t u0 = code & 0xffffu;
  const int ext[3] = {1 << ((L + 2) / 3), 1 << ((L + 1) / 3), 1 << (L / 3)};
  const uint32_t uc[3] = {compact3(u0), compact3(u0 >> 1), compact3(u0 >> 2)};
  const float unit = 2.f / (float)(1 << kUnitBits);
  float lo[3], hi[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    lo[d] = -1.f + unit * (float)uc[d];
    hi[d] = -1.f + unit * (float)(uc[d] + ext[d]);
  }
  return block_box(lo, hi, g, R);
}

// Two CTAs of 8 warps per SM, each on its own units, so that one CTA's barriers and
// flushes overlap the other's reductions.  At most 96 registers: with them a CTA of the
// density pass (8 warps x 64) fits beside the scatter's 16 warps in one SM's register file.
template <int C, bool EVEN_R>
__global__ void __maxnreg__(96)
k_scat(Model md, Grads gr, Bricks brp, TrainWs ws, const float* __restrict__ xyz, int capn) {
  extern __shared__ __align__(16) unsigned char smraw[];
  ScatHead& h = *reinterpret_cast<ScatHead*>(smraw);
  int32_t* acc = reinterpret_cast<int32_t*>(smraw + sizeof(ScatHead));
  __shared__ Bricks br;
  __shared__ TileMap dtm;   // the decoder's 128-point tiles (ws.gmax_blk)
  load_bricks(brp, br);
  if (threadIdx.x == 0) build_tile_map(br, 128, dtm);
  const int tid = threadIdx.x, lane = tid & 31;
  const int M = md.M, R = md.R;
  const int ngrp = M >= 32 ? M >> 5 : 1;
  const int gper = M >= 32 ? 32 : M;             // grids of a unit
  constexpr int kNode = C * 32;                  // words of one node of a column group
  constexpr uint32_t kNodeBytes = kNode * 4;
  {  // the boxes start zeroed; every flush leaves them zeroed again
    uint4* a4 = reinterpret_cast<uint4*>(acc);
    for (int q = tid; q < capn * kNode / 4; q += SCT) a4[q] = make_uint4(0u, 0u, 0u, 0u);
  }
  const int nunits = ws.tile_ctr[0] * ngrp;
  const int64_t gsz = (int64_t)R * R * R * C;
  int32_t* col = acc + lane;                     // this thread's column
  const uint32_t col_s = su32(col);
  constexpr uint32_t kNz = C == 2 ? 0x7fff7fffu : 0x7fffu;    // nonzero dL/dy
  bool first = true;
  for (;;) {
    // units are taken in list order (brick by brick, Morton order inside a brick, the
    // groups of a tile one after the other), so the CTAs on the GPU at one time work on
    // neighbouring blocks of one brick; each CTA takes its next unit one ahead and asks
    // L2 for that tile's dL/dy rows (contiguous)
    if (tid == 0) {
      auto take = [&](int& grp) {
        const int t = atomicAdd(ws.tile_ctr + 1, 1);
        ScatTile T;
        T.start = 0; T.count = -1; T.code = 0;
        grp = 0;
        if (t < nunits) { T = ws.tiles[t / ngrp]; grp = t % ngrp; }
        return T;
      };
      if (first) h.tile = take(h.grp);
      else { h.tile = h.tnext; h.grp = h.gnext; }
      if (h.tile.count < 0) { h.tnext = h.tile; h.gnext = 0; }
      else h.tnext = take(h.gnext);
      if (h.tnext.count > 0) {
        const char* rows = reinterpret_cast<const char*>(ws.dY + h.tnext.start * md.K);
        const uint32_t bytes = (uint32_t)h.tnext.count * (uint32_t)md.K * 2u;   // a multiple of 16
        for (uint32_t o = 0; o < bytes; o += 65536u)
          asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(rows + o), "r"(min(65536u, bytes - o))
                       : "memory");
      }
    }
    first = false;
    __syncthreads();   // also: the previous tile's flush has finished with h
    const ScatTile T = h.tile;
    if (T.count < 0) break;
    const ScatMap mp = unit_map<SCW>(M, h.grp);
    const int g0u = mp.grp * 32;                  // the unit's first grid (M >= 32)
    const int b = (int)(T.code >> 20);
    const int64_t p0 = T.start;
    const int np = T.count;
    const float* Gb = md.G + (int64_t)b * md.sG;
    const int lvl = (int)((T.code >> 16) & 15u);
    bool mine_in = true;   // every point of this thread lies in the tile's block
    for (int p = tid; p < np; p += SCT) {
      const float x = xyz[3 * (p0 + p)], y = xyz[3 * (p0 + p) + 1], z = xyz[3 * (p0 + p) + 2];
      h.xs[p] = make_float4(x, y, z, 0.f);
      mine_in &= (((morton_bin(x, y, z) >> 3) ^ (T.code & 0xffffu)) >> lvl) == 0u;
    }
    if (tid < gper) {
      const int g = g0u + tid;
      h.box[tid] = tile_box(T.code, Gb + 12 * g, R);
      uint32_t mb = 0u;
      if (ws.gmax_blk) {   // the decoder's maxima of the 128-point tiles overlapping this tile
        const int64_t lp = p0 - br.off[b];
        const int d0 = dtm.first[b] + (int)(lp / 128), d1 = dtm.first[b] + (int)((lp + np - 1) / 128);
        for (int d = d0; d <= d1; ++d) mb = max(mb, (uint32_t)ws.gmax_blk[(int64_t)d * M + g]);
      }
      h.gmax[tid] = mb;
    }
    // the block's boxes bound the points only if all of them lie in the block (always,
    // for a Morton-sorted batch); otherwise points outside a box add their corners directly
    const bool in_block = __syncthreads_and(mine_in) != 0;
    if (!ws.gmax_blk) {  // largest |dL/dy| of every grid over the tile (eight loads in flight; the
                         // rows were prefetched into L2 while the previous tile ran)
      uint32_t mx = 0u;
      for (int p = mp.pg; p < np; p += 8 * mp.npg) {
        uint32_t d[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int q = p + u * mp.npg;
          d[u] = q < np ? dy_bits<C>(ws.dY, p0 + q, M, mp.g) & kNz : 0u;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) mx = C == 2 ? __vmaxu2(mx, d[u]) : max(mx, d[u]);
      }
      if (C == 2) mx = max(mx & 0xffffu, mx >> 16);
      if (mx) atomicMax(h.gmax + (mp.g - g0u), mx);
    }
    __syncthreads();
    const uint2 bx = h.box[mp.g - g0u];
    const int nxb = (int)(bx.y & 0xffu), nyb = (int)((bx.y >> 8) & 0xffu), nzb = (int)((bx.y >> 16) & 0xffu);
    const int lox = (int)(bx.x & 0xffu), loy = (int)((bx.x >> 8) & 0xffu), loz = (int)((bx.x >> 16) & 0xffu);
    const int nodes = nxb * nyb * nzb;
    const bool boxed = nodes > 0 && nodes <= capn;
    const uint32_t mb = h.gmax[mp.g - g0u];
    float inv;
    const float scale = fixed_scale(mb, np, inv);
    float* dFi = gr.dF + (int64_t)b * gr.sF + mp.g * gsz;
    if (mb != 0u && (nodes > 0 || !in_block)) {
      float gi[12];
      {
        const float4* g4 = reinterpret_cast<const float4*>(Gb + 12 * mp.g);
        const float4 a = __ldg(g4), c = __ldg(g4 + 1), d = __ldg(g4 + 2);
        gi[0] = a.x; gi[1] = a.y; gi[2] = a.z; gi[3] = a.w; gi[4] = c.x; gi[5] = c.y;
        gi[6] = c.z; gi[7] = c.w; gi[8] = d.x; gi[9] = d.y; gi[10] = d.z; gi[11] = d.w;
      }
      const uint32_t oy = (uint32_t)nxb * kNodeBytes, oz = (uint32_t)(nxb * nyb) * kNodeBytes;
      const float hs = 0.5f * (float)(R - 1);
      const float ct = hs - 0.5f + kMagic;   // an integer when R is even (axis_cell)
      const unsigned long long hs2 = f2_bits(hs, hs), ct2 = f2_bits(ct, ct), mm2 = f2_bits(kMagic, kMagic);
      const int32_t mlox = kMagicBits + lox, mloy = kMagicBits + loy, mloz = kMagicBits + loz;
      // dL/dy of the next SU points is requested while the current SU are processed
      constexpr int SU = 4;
      uint32_t dn[SU];
      // this lane's dL/dy of the tile's first point; point q's is q * M entries on
      // (C bf16 per entry)
      using DyT = std::conditional_t<C == 2, unsigned int, unsigned short>;
      const DyT* dyl = reinterpret_cast<const DyT*>(ws.dY) + p0 * M + mp.g;
      auto load_next = [&](int p) {
#pragma unroll
        for (int u = 0; u < SU; ++u) {
          const int q = p + u * mp.npg;
          dn[u] = q < np ? (uint32_t)__ldg(dyl + q * M) : 0u;
        }
      };
      load_next(mp.pg);
      for (int p = mp.pg; p < np; p += SU * mp.npg) {
        uint32_t dc[SU];
#pragma unroll
        for (int u = 0; u < SU; ++u) dc[u] = dn[u];
        load_next(p + SU * mp.npg);
        // the cells and weights of all SU points first, without branches, so that their
        // dependency chains overlap; then the reductions point by point
        uint32_t ad[SU];            // box address of the cell's first corner; ~0u: not in the box
        float wxs[SU], wys[SU], wzs[SU];
        uint32_t live = 0u;         // bit u: nonzero dL/dy, cell not in the box (the direct path)
#pragma unroll
        for (int u = 0; u < SU; ++u) {
          const int q = p + u * mp.npg;
          const float4 x = h.xs[q < np ? q : p];
          float ux, uy, uz;
          affine(gi, x.x, x.y, x.z, ux, uy, uz);
          // Eq. 2's set-up as make_cell computes it; for points inside the grid s lies in
          // [0, R-1] already (the rounding of fmaf is monotone), so no clamp is needed
          // (with R odd the cell is floor(s): it differs from min(floor(s), R-2) only at
          // s = R-1, whose cell R-1 is never in a box and takes the exact path below)
          const bool nz = (dc[u] & kNz) != 0u;
          unsigned lx, ly, lz;   // cell relative to the box
          if constexpr (EVEN_R) {
            int32_t tx, ty;   // x and y as one packed pair
            axis_cell2(f2_bits(ux, uy), hs2, ct2, mm2, tx, ty, wxs[u], wys[u]);
            lx = (unsigned)(tx - mlox);
            ly = (unsigned)(ty - mloy);
            lz = (unsigned)(axis_cell(uz, hs, ct, wzs[u]) - mloz);
          } else {
            const float sx = fmaf(ux, hs, hs), sy = fmaf(uy, hs, hs), sz = fmaf(uz, hs, hs);
            const int cx = (int)sx, cy = (int)sy, cz = (int)sz;
            wxs[u] = sx - (float)cx; wys[u] = sy - (float)cy; wzs[u] = sz - (float)cz;
            lx = (unsigned)(cx - lox); ly = (unsigned)(cy - loy); lz = (unsigned)(cz - loz);
          }
          bool inbox = boxed && lx < (unsigned)(nxb - 1) && ly < (unsigned)(nyb - 1) && lz < (unsigned)(nzb - 1);
          // With R even a cell in the box means the point is inside the grid (Eq. 2's
          // mask): the box's cells lie in [0, R-2], and beyond a face the cell on that
          // axis is -1 or R-1.  With R odd the cell is a truncation: test the mask.
          if constexpr (!EVEN_R) inbox = inbox && (fabsf(ux) <= 1.f) & (fabsf(uy) <= 1.f) & (fabsf(uz) <= 1.f);
          ad[u] = nz && inbox ? col_s + ((lz * (unsigned)nyb + ly) * (unsigned)nxb + lx) * kNodeBytes : ~0u;
          live |= (uint32_t)(nz && !inbox) << u;
        }
#pragma unroll
        for (int u = 0; u < SU; ++u) {
          if (ad[u] != ~0u) {
            red_cell<C>(ad[u], oy, oz, wxs[u], wys[u], wzs[u], dc[u], scale);
          } else if (live & (1u << u)) {   // outside the tile's box (rounding at its faces, or an unsorted batch)
            const float4 x = h.xs[p + u * mp.npg];
            float ux, uy, uz;
            affine(gi, x.x, x.y, x.z, ux, uy, uz);
            const Cell c = make_cell(ux, uy, uz, R);
            const uint32_t d = dc[u];
            if (c.inside)
              scatter_point(dFi, c, R, C, __uint_as_float(d << 16), C == 2 ? __uint_as_float(d & 0xffff0000u) : 0.f);
          }
        }
      }
    }
    __syncthreads();
    // flush: every nonzero node of the grid's box into the float32 gradient grid with one
    // atomic, summing the grid's columns (M < 32) and clearing them for the next tile
    if (boxed && mb != 0u && (M >= 32 || lane < M)) {
      const int step = M >= 32 ? mp.npg : SCW;   // M < 32: lanes >= M idle, warps split the nodes
      const int n0 = M >= 32 ? mp.pg : (tid >> 5);
      int qz = n0 / (nxb * nyb), qr = n0 - qz * nxb * nyb;
      int qy = qr / nxb, qx = qr - qy * nxb;
      for (int n = n0; n < nodes; n += step) {
        int32_t s0 = 0, s1 = 0;
        int32_t* q = acc + n * kNode + lane;   // column lane = grid g's first
        for (int sub = 0; sub < (M >= 32 ? 1 : 32 / M); ++sub) {
          int32_t* qs = q + sub * M;
          s0 += qs[0];
          qs[0] = 0;
          if (C == 2) { s1 += qs[32]; qs[32] = 0; }
        }
        if (s0 | s1) {
          const int node = ((loz + qz) * R + (loy + qy)) * R + lox + qx;   // < R^3 <= 2^18
          if (C == 2) atomicAdd(reinterpret_cast<float2*>(dFi) + node, make_float2((float)s0 * inv, (float)s1 * inv));
          else atomicAdd(dFi + node, (float)s0 * inv);
        }
        qx += step;
        while (qx >= nxb) {
          qx -= nxb;
          if (++qy == nyb) { qy = 0; ++qz; }
        }
      }
    }
  }
}

// =============================================================================== k_enc
// Encoder (Eq. 1-3) on the scatter's tiles, as (tile, group of 32 grids) units, two CTAs
// of 16 warps per SM.  Lane l of a warp takes grid l of the unit's group (ScatMap).
// Each grid's node box of the tile's block is staged in shared memory as the float32
// values of its BF16 nodes (C per entry), node by node with one column per lane, so
// the eight corner reads of a warp fall in distinct banks and the warp's features of
// one point form one coalesced store of Y.  Points outside their box (rounding at its
// faces; an unsorted batch) and grids whose box does not fit read the corners from
// global memory.  The feature density of Eq. 7 is a pass of its own (k_density_rho).
struct EncHead {
  float4 xs[ST];                // the tile's points
  uint2 box[32];                // node box of the tile's block per grid of the unit (as in the scatter)
  float gs[kMaxGrids * 12];     // the brick's transforms
  ScatTile tile;
  int grp;
};
template <int C, bool EVEN_R>
__global__ void __launch_bounds__(SNT, 2)
k_enc(Model md, Bricks brp, TrainWs ws, const float* __restrict__ xyz, int capn) {
  using E = EncNode<C>;
  using SE = EncSNode<C>;
  extern __shared__ __align__(16) unsigned char smraw[];
  EncHead& h = *reinterpret_cast<EncHead*>(smraw);
  SE* boxes = reinterpret_cast<SE*>(smraw + sizeof(EncHead));   // [capn][32 columns]
  __shared__ Bricks br;
  load_bricks(brp, br);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int M = md.M, R = md.R;
  const int ngrp = M >= 32 ? M >> 5 : 1;
  const int gper = M >= 32 ? 32 : M;             // grids of a unit
  const int nunits = ws.tile_ctr[0] * ngrp;
  const int64_t gsz = (int64_t)R * R * R * C;
  SE* col = boxes + lane;                        // this thread's column
  const float hs = 0.5f * (float)(R - 1);
  // staging: every lane fills its own column, the warps split the nodes
  const int n0 = warp, nstep = SNW;
  int cur = -1;
  for (;;) {
    if (tid == 0) {
      const int t = atomicAdd(ws.tile_ctr + 2, 1);
      ScatTile T;
      T.start = 0; T.count = -1; T.code = 0;
      h.grp = 0;
      if (t < nunits) { T = ws.tiles[t / ngrp]; h.grp = t % ngrp; }
      h.tile = T;
    }
    __syncthreads();   // also: the previous unit is done with h and the boxes
    const ScatTile T = h.tile;
    if (T.count < 0) break;
    const ScatMap mp = unit_map<SNW>(M, h.grp);
    const int g0u = mp.grp * 32;                  // the unit's first grid (M >= 32)
    const int b = (int)(T.code >> 20);
    const float* Gb = md.G + (int64_t)b * md.sG;
    if (b != cur) {
      cur = b;
      for (int c = tid; c < M * 12; c += SNT) h.gs[c] = Gb[c];
    }
    const int64_t p0 = T.start;
    const int np = T.count;
    for (int p = tid; p < np; p += SNT)
      h.xs[p] = make_float4(xyz[3 * (p0 + p)], xyz[3 * (p0 + p) + 1], xyz[3 * (p0 + p) + 2], 0.f);
    if (tid < gper) h.box[tid] = tile_box(T.code, Gb + 12 * (g0u + tid), R);
    __syncthreads();
    const EncBox eb = enc_box<C>(h.box[mp.g - g0u], capn, su32(col));
    const E* Fg = reinterpret_cast<const E*>(md.F16 + (int64_t)b * md.sF + mp.g * gsz);
    if (eb.boxed) enc_stage<C>(eb, Fg, R, col, n0, nstep);
    float gi[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) gi[j] = h.gs[12 * mp.g + j];
    __syncthreads();
    const float ct = hs - 0.5f + kMagic;   // an integer when R is even (axis_cell)
    E* Yt = reinterpret_cast<E*>(ws.Y) + p0 * M + mp.g;
    const __nv_bfloat16* Fi = md.F16 + (int64_t)b * md.sF + mp.g * gsz;
#pragma unroll 2
    for (int p = mp.pg; p < np; p += mp.npg) {
      const float4 x = h.xs[p];
      Yt[p * M] = (E)encode_point<C, EVEN_R>(gi, x.x, x.y, x.z, eb, hs, ct, R, Fi);
    }
  }
}

// =============================================================================== k_rec_dg
// dL/dG through the features (SRN_REC_DG), from the decoder's dL/dy: per point and
// grid, dL/du = (R-1)/2 sum_c dL/dy_c de_c/ds (Eq. 2 differentiated inside the cell,
// on the BF16 features the forward pass read), then dL/dA_i += dL/du x^T and
// dL/dt_i += dL/du.  Thread (grid tid % M, point group tid / M) sums its points in
// float32; the block reduces the groups in float64 and adds them per brick.
constexpr int RT = 128;   // points per tile
constexpr int RNT = 256;

template <int C>
__global__ void __launch_bounds__(RNT) k_rec_dg(Model md, Bricks brp, TrainWs ws, const float* __restrict__ xyz) {
  __shared__ Bricks br;
  __shared__ TileMap tm;
  __shared__ float4 sx[RT];
  __shared__ float sg[kMaxGrids * 12];
  __shared__ double red[RNT];
  load_bricks(brp, br);
  const int tid = threadIdx.x, M = md.M, R = md.R;
  const int npg = RNT / M, gi = tid % M, pg = tid / M;   // M divides RNT (M = K / C, a power of two)
  if (tid == 0) build_tile_map(br, RT, tm);
  __syncthreads();
  const int total = tm.first[br.n];
  const int per = (total + gridDim.x - 1) / gridDim.x;
  const int tb = blockIdx.x * per, te = min(total, tb + per);
  const int64_t gsz = (int64_t)R * R * R * C;
  const float hs = 0.5f * (float)(R - 1);
  float acc[12];
#pragma unroll
  for (int j = 0; j < 12; ++j) acc[j] = 0.f;
  auto flush = [&](int b) {
    for (int j = 0; j < 12; ++j) {
      red[tid] = (double)acc[j];
      acc[j] = 0.f;
      __syncthreads();
      if (pg == 0) {
        double t = 0.0;
        for (int q = 0; q < npg; ++q) t += red[q * M + gi];
        atomicAdd(ws.rsum + ((int64_t)b * M + gi) * 12 + j, t);
      }
      __syncthreads();
    }
  };
  int cur = -1;
  for (int tile = tb; tile < te; ++tile) {
    const int b = brick_of_tile(tm, br.n, tile, cur);
    if (b != cur) {
      if (cur >= 0) flush(cur);
      cur = b;
      for (int k = tid; k < M * 12; k += RNT) sg[k] = md.G[(int64_t)b * md.sG + k];
    }
    const int64_t p0 = br.off[b] + (int64_t)(tile - tm.first[b]) * RT;
    const int np = (int)min((int64_t)RT, br.off[b + 1] - p0);
    if (tid < RT) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (tid < np) v = make_float4(xyz[3 * (p0 + tid)], xyz[3 * (p0 + tid) + 1], xyz[3 * (p0 + tid) + 2], 0.f);
      sx[tid] = v;
    }
    __syncthreads();
    const float* g = sg + 12 * gi;
    const __nv_bfloat16* Fi = md.F16 + (int64_t)b * md.sF + gi * gsz;
    for (int p = pg; p < np; p += npg) {
      const float4 x = sx[p];
      float ux, uy, uz;
      affine(g, x.x, x.y, x.z, ux, uy, uz);
      const Cell c = make_cell(ux, uy, uz, R);
      if (!c.inside) continue;
      float g0, g1 = 0.f;
      if (C == 2) {
        const float2 d = unpack_bf16(__ldg(reinterpret_cast<const unsigned int*>(ws.dY) + (p0 + p) * M + gi));
        g0 = d.x;
        g1 = d.y;
      } else {
        g0 = __bfloat162float(ws.dY[(p0 + p) * M + gi]);
      }
      const int64_t nb = ((int64_t)c.cz * R + c.cy) * R + c.cx;
      float a[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int64_t n = nb + (k & 1) + ((k & 2) ? R : 0) + ((k & 4) ? (int64_t)R * R : 0);
        if (C == 2) {
          const float2 f = node2(Fi, n);
          a[k] = fmaf(g0, f.x, g1 * f.y);
        } else {
          a[k] = g0 * node1(Fi, n);
        }
      }
      float du[3];
      trilinear_ds(a, c.wx, c.wy, c.wz, du[0], du[1], du[2]);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const float q = du[d] * hs;
        acc[4 * d] = fmaf(q, x.x, acc[4 * d]);
        acc[4 * d + 1] = fmaf(q, x.y, acc[4 * d + 1]);
        acc[4 * d + 2] = fmaf(q, x.z, acc[4 * d + 2]);
        acc[4 * d + 3] += q;
      }
    }
    __syncthreads();
  }
  if (cur >= 0) flush(cur);
}

int occupancy(const void* kern, int threads, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem) != cudaSuccess || n < 1) n = 1;
  return n;
}

// Dynamic shared memory of k_scat for boxes of capn nodes (one column group), and the
// largest capn with which two of its CTAs and one CTA of the density pass fit on an SM.
size_t scat_smem(int M, int C, int capn) {
  (void)M;
  return sizeof(ScatHead) + (size_t)capn * C * 128;
}
int scat_capn(int M, int C) {
  int dev = 0, optin = 0, per_sm = 0, stat = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, (const void*)k_scat<2, true>) == cudaSuccess) stat = (int)fa.sharedSizeBytes;
  (void)M;
  // two CTAs (1 KB reserved for each) and room for one CTA of the density pass that may
  // run beside them (its reserve included)
  const long long block = std::min<long long>(optin, ((long long)per_sm - 2 * 1024 - kDensityCtaSmem) / 2);
  const long long room = block - stat - (long long)sizeof(ScatHead);
  return room > 0 ? (int)(room / ((long long)C * 128)) : 0;
}

// The same for k_enc, at two CTAs per SM.
size_t enc_smem(int M, int C, int capn) {
  (void)M;
  return sizeof(EncHead) + (size_t)capn * 32 * (C == 2 ? 8 : 4);
}
int enc_capn(int M, int C) {
  int dev = 0, per_sm = 0, stat = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, (const void*)k_enc<2, true>) == cudaSuccess) stat = (int)fa.sharedSizeBytes;
  (void)M;
  const long long room = (long long)per_sm / 2 - 1024 - stat - (long long)sizeof(EncHead);
  return room > 0 ? (int)(room / ((long long)32 * (C == 2 ? 8 : 4))) : 0;
}

template <int K>
cudaError_t launch_train_k(const Launch& L, bool dens, const Model& md, const Grads& gr, const Bricks& br,
                           const TrainWs& ws, const float* xyz, const float* target, const Tuning& tn,
                           const KernelMark* mark, const SideStream* side) {
  auto mark_start = [&](int k) { if (mark && mark->which == k) cudaEventRecord(mark->start, L.stream); };
  auto mark_stop = [&](int k) { if (mark && mark->which == k) cudaEventRecord(mark->stop, L.stream); };
  int tiles = 0;
  for (int b = 0; b < br.n; ++b) tiles += (int)((br.off[b + 1] - br.off[b] + ET - 1) / ET);
  if (tiles == 0) return cudaSuccess;
  cudaError_t e;
  {  // scatter tiles: aligned Morton blocks of each brick's points
    int64_t nmax = 0;
    for (int b = 0; b < br.n; ++b) nmax = std::max<int64_t>(nmax, br.off[b + 1] - br.off[b]);
    if (nmax > INT32_MAX) return cudaErrorInvalidValue;
    if ((e = cudaMemsetAsync(ws.tile_ctr, 0, 3 * sizeof(int32_t), L.stream)) != cudaSuccess) return e;
    if (!ws.bin_start) {   // else the sampler's histogram gives the unit starts
      if ((e = cudaMemsetAsync(ws.ustart, 0xff, sizeof(int32_t) * (kUnits + 1) * br.n, L.stream)) != cudaSuccess)
        return e;
      const int bx = (int)std::min<int64_t>((nmax + 255) / 256, 4 * L.num_sms / std::max(1, br.n) + 1);
      k_unit_starts<<<dim3(bx, br.n), 256, 0, L.stream>>>(br, xyz, ws.ustart);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int cap = std::min(scat_capn(md.M, md.C), enc_capn(md.M, md.C));   // both kernels' boxes fit
    if (cap < 8) return cudaErrorInvalidConfiguration;
    if (tn.tile_points < kMinTilePoints || tn.tile_points > ST || tn.tile_level < 0 || tn.tile_level > kMaxTileLevel)
      return cudaErrorInvalidValue;
    k_tile_list<<<br.n, 1024, 0, L.stream>>>(br, ws, md, cap, tn.tile_level, tn.tile_points);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  {
    const int capn = enc_capn(md.M, md.C);
    const size_t smem = enc_smem(md.M, md.C, capn);
    const bool even = (md.R & 1) == 0;
    const void* kern = md.C == 2 ? (even ? (const void*)k_enc<2, true> : (const void*)k_enc<2, false>)
                                 : (even ? (const void*)k_enc<1, true> : (const void*)k_enc<1, false>);
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return e;
    const int grid = L.num_sms * occupancy(kern, SNT, smem);
    mark_start(0);
    void* args[] = {(void*)&md, (void*)&br, (void*)&ws, (void*)&xyz, (void*)&capn};
    if ((e = cudaLaunchKernel(kern, dim3(grid), dim3(SNT), args, smem, L.stream)) != cudaSuccess) return e;
    if (dens && side) {   // rho beside the decoder
      if ((e = cudaEventRecord(side->enc_done, L.stream)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(side->stream, side->enc_done, 0)) != cudaSuccess) return e;
      if ((e = launch_density_rho(Launch{side->stream, L.num_sms}, md, br, ws, xyz)) != cudaSuccess) return e;
    } else if (dens && (e = launch_density_rho(L, md, br, ws, xyz)) != cudaSuccess) {
      return e;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    mark_stop(0);
  }
  if constexpr (K == 128) {   // tcgen05 decoder
    mark_start(1);
    if ((e = launch_mlp_tc(L, md, gr, br, ws, target)) != cudaSuccess) return e;
    mark_stop(1);
  } else {
    const int smem = MlpLay<K>::BYTES;
    if ((e = cudaFuncSetAttribute(k_mlp<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
      return e;
    const int grid = std::min(tiles, L.num_sms);
    mark_start(1);
    k_mlp<K><<<grid, NT, smem, L.stream>>>(md, gr, br, ws, target);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    mark_stop(1);
  }
  if (dens && side) {   // the other two density passes beside the scatter, after the decoder
    // CTAs taking tiles from a counter, tn.density_ctas per SM (default two): one fits
    // beside the scatter's two CTAs (registers and the shared memory scat_capn leaves),
    // the other starts as the scatter's CTAs finish and leaves room for the Adam of F and
    // the decoder, which the training step runs beside this pass's tail (measured: 3.43 ms
    // per step against 3.48 with four CTAs per SM, whose registers fill the SM)
    const int ctas = std::min(std::max(tn.density_ctas, 1), kMaxDensityCtas);
    if ((e = cudaEventRecord(side->fork, L.stream)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(side->stream, side->fork, 0)) != cudaSuccess) return e;
    if ((e = launch_density(Launch{side->stream, L.num_sms}, md, br, ws, xyz, ws.eps, ctas)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(side->join, side->stream)) != cudaSuccess) return e;
  }
  {
    const int capn = scat_capn(md.M, md.C);
    if (capn < 8) return cudaErrorInvalidConfiguration;
    const size_t smem = scat_smem(md.M, md.C, capn);
    const bool even = (md.R & 1) == 0;
    const void* kern = md.C == 2 ? (even ? (const void*)k_scat<2, true> : (const void*)k_scat<2, false>)
                                 : (even ? (const void*)k_scat<1, true> : (const void*)k_scat<1, false>);
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return e;
    const int grid = L.num_sms * occupancy(kern, SCT, smem);
    mark_start(2);
    void* args[] = {(void*)&md, (void*)&gr, (void*)&br, (void*)&ws, (void*)&xyz, (void*)&capn};
    if ((e = cudaLaunchKernel(kern, dim3(grid), dim3(SCT), args, smem, L.stream)) != cudaSuccess) return e;
    mark_stop(2);
  }
  if (ws.rec_dg) {
    const int grid = std::min((int)((br.off[br.n] + RT - 1) / RT), 2 * L.num_sms);
    if (md.C == 2) k_rec_dg<2><<<grid, RNT, 0, L.stream>>>(md, br, ws, xyz);
    else k_rec_dg<1><<<grid, RNT, 0, L.stream>>>(md, br, ws, xyz);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (dens && side && !side->defer_join && (e = cudaStreamWaitEvent(L.stream, side->join, 0)) != cudaSuccess)
    return e;
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_train_bf16(const Launch& L, bool dens, const Model& md, const Grads& gr, const Bricks& br,
                              const TrainWs& ws, const float* xyz, const float* target, const Tuning& tn,
                              const KernelMark* mark, const SideStream* side) {
  switch (md.K) {
    case 16: return launch_train_k<16>(L, dens, md, gr, br, ws, xyz, target, tn, mark, side);
    case 32: return launch_train_k<32>(L, dens, md, gr, br, ws, xyz, target, tn, mark, side);
    case 64: return launch_train_k<64>(L, dens, md, gr, br, ws, xyz, target, tn, mark, side);
    case 128: return launch_train_k<128>(L, dens, md, gr, br, ws, xyz, target, tn, mark, side);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace srn
