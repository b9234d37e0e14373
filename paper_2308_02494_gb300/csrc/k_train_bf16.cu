// BF16 training pass over all bricks: three kernels, each shaped for its own bound.
//
//  k_enc   encoder (Eq. 1-3) and the feature density of Eq. 7.  Low register count,
//          several CTAs per SM to hide the latency of the corner gathers (L1/L2
//          resident BF16 grids).  Writes the features Y [N][K] (bf16) and rho [N].
//  k_mlp   decoder forward and backward for K < 128 on the tensor cores (mma.sync
//          m16n8k16, BF16 operands, FP32 accumulation): L_rec partial sums,
//          h(x) = (f - v)^2, dW1/dW2/dw3 accumulated in registers per CTA and flushed
//          once, and dL/dy written grid-major as bf16 (dY [M][N][C]) for the scatter.
//          K = 128 runs on tcgen05 instead (k_mlp_tc.cu).
//  k_scat  adjoint of Eq. 2.  A tile is up to 1024 points of one brick lying in one
//          aligned Morton range of the sampler's bins (a small axis-aligned block of
//          the brick), listed by k_unit_starts / k_tile_list.  The CTA takes the grids
//          one at a time: the tile's block, mapped through the grid's Eq. 1, bounds
//          the node box; the CTA counting-sorts the tile's points by their cell in that
//          box (integer shared-memory atomics, a block-wide scan), sums each cell's
//          eight corner contributions with plain FMAs into corner-major per-cell sums,
//          and lets every node of the box gather its (up to) eight cells and add the
//          total into the float32 gradient grid with one float2 atomic.  When the box
//          exceeds the shared-memory capacity the tile falls back to the exact box of
//          its points, of each half, of each 256-point chunk, then to adding each
//          point's corners directly; so do single points outside their tile's block
//          (a batch that is not Morton-sorted is correct, only slower).
#include "bf16_ops.cuh"
#include "kernels.h"
#include <algorithm>
#include <climits>
#include <cmath>

namespace srn {
namespace {

template <typename Tv>
__device__ __forceinline__ Tv warp_sum(Tv v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// =============================================================================== k_enc
constexpr int ET = 128;
constexpr int ENT = 256;

template <int K, bool DENS>
__global__ void __launch_bounds__(ENT, 4)
k_enc(Model md, Bricks brp, TrainWs ws, const float* __restrict__ xyz) {
  __shared__ TileMap tm;
  __shared__ Bricks br;
  __shared__ float4 xs[ET];
  __shared__ __align__(16) float gs[kMaxGrids * 12];
  __shared__ float dets[kMaxGrids];
  __shared__ float rhos[2][ET];
  __shared__ uint32_t ys[ET][K / 2 + 1];   // bf16 pairs; odd row pitch: conflict-free column writes
  load_bricks(brp, br);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int M = md.M, C = md.C, R = md.R;
  if (tid == 0) build_tile_map(br, ET, tm);
  __syncthreads();
  const int total = tm.first[br.n];
  const int per = (total + gridDim.x - 1) / gridDim.x;
  const int tb = blockIdx.x * per, te = min(total, tb + per);
  double sum_rho = 0.0;
  int cur = -1;
  auto flush = [&](int b) {
    if (!DENS) return;
    double s = warp_sum(sum_rho);
    if (lane == 0) atomicAdd(ws.acc + b * kAccPerBrick + ACC_SUM_RHO, s);
    sum_rho = 0.0;
  };
  uint32_t* Y32 = reinterpret_cast<uint32_t*>(ws.Y);
  for (int tile = tb; tile < te; ++tile) {
    const int b = brick_of_tile(tm, br.n, tile, cur);
    if (b != cur) {
      if (cur >= 0) flush(cur);
      __syncthreads();
      cur = b;
      const float* G = md.G + (int64_t)b * md.sG;
      for (int c = tid; c < M * 12; c += ENT) gs[c] = G[c];
      if (tid < M) dets[tid] = det3(G + 12 * tid);
      __syncthreads();
    }
    const int64_t p0 = br.off[b] + (int64_t)(tile - tm.first[b]) * ET;
    const int np = (int)min((int64_t)ET, br.off[b + 1] - p0);
    if (tid < ET) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (tid < np) v = make_float4(xyz[3 * (p0 + tid)], xyz[3 * (p0 + tid) + 1], xyz[3 * (p0 + tid) + 2], 0.f);
      xs[tid] = v;
    }
    __syncthreads();
    {
      const __nv_bfloat16* Fb = md.F16 + (int64_t)b * md.sF;
      const int64_t gsz = (int64_t)R * R * R * C;
      const int p = (warp & 3) * 32 + lane, gsub = warp >> 2;
      const float4 pt = xs[p];
      const bool valid = p < np;
      float rho = 0.f;
#pragma unroll 4
      for (int i = gsub; i < M; i += 2) {
        float ux, uy, uz;
        {
          const float4* g4 = reinterpret_cast<const float4*>(gs + 12 * i);
          const float4 a = g4[0], c = g4[1], d = g4[2];
          ux = fmaf(a.x, pt.x, fmaf(a.y, pt.y, fmaf(a.z, pt.z, a.w)));
          uy = fmaf(c.x, pt.x, fmaf(c.y, pt.y, fmaf(c.z, pt.z, c.w)));
          uz = fmaf(d.x, pt.x, fmaf(d.y, pt.y, fmaf(d.z, pt.z, d.w)));
        }
        const Cell c = make_cell(ux, uy, uz, R);
        float f0 = 0.f, f1 = 0.f;
        if (valid && c.inside) trilinear_bf16_any(Fb + i * gsz, c, R, C, f0, f1);
        if (C == 2) ys[p][i] = pack_bf16(f0, f1);
        else reinterpret_cast<__nv_bfloat16*>(ys[p])[i] = __float2bfloat16_rn(f0);
        if (DENS && valid) rho += dets[i] * flat_top(ux, uy, uz, md.p);
      }
      if (DENS) rhos[gsub][p] = rho;
    }
    __syncthreads();
    for (int idx = tid; idx < np * (K / 2); idx += ENT) {
      const int p = idx / (K / 2), w = idx % (K / 2);
      Y32[(p0 + p) * (K / 2) + w] = ys[p][w];
    }
    if (DENS && tid < np) {
      const float r = rhos[0][tid] + rhos[1][tid];
      ws.rho[p0 + tid] = r;
      sum_rho += (double)r;
    }
    __syncthreads();
  }
  if (cur >= 0) flush(cur);
}

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
  const int64_t ntot = br.off[br.n];
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
    // ---- dL/dy to global memory, grid-major bf16: dY[i][p][c]
    for (int idx = tid; idx < M * T; idx += NT) {
      const int i = idx / T, p = idx % T;
      if (p < np) {
        const int64_t o = (int64_t)i * ntot + p0 + p;
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
constexpr int ST = 1024;        // Morton-consecutive points per scatter tile
constexpr int SNT = 256;
constexpr int PPT = ST / SNT;   // points per thread (point tid + 256 j belongs to chunk j)
constexpr int CCAP = 512;       // cells of a usable box
constexpr int NCAP = 1024;      // nodes of a usable box

// Shared memory of k_scat (dynamic): per-point data, the counting sort, per-cell
// corner sums (corner-major, conflict-free) and the carried partial sums.
struct ScatSmem {
  float cs[16 * CCAP];         // per-cell corner sums: corner k, cell l, channel e at (k CCAP + l) C + e
  float pl[16 * SNT];          // chunk t's last partial sums (its cell goes on past the chunk): (k SNT + t) C + e
  uint2 tbox[kMaxGrids];       // the tile's node box in every grid (lo and node counts, bytes)
  float4 wg[ST];               // per point: grid coordinates s (Eq. 2), then, for the points of a
                               // box pass, the cell weights; .w holds dL/dy (bf16 x 2 bits)
  int cnt[CCAP + 1];           // cell counts, then starts; all zero between passes
  alignas(16) unsigned short perm[ST];    // point indices ordered by cell
  alignas(16) unsigned short pcell[ST];    // the cell of each sorted position
  int red[2][SNT / 32][6];     // block min/max scratch (alternating between calls)
  int wsum[SNT / 32];          // block scan scratch
};

struct Box {
  int lo[3], n[3];   // first node and nodes per axis of the box
  int ncells;
  bool ok;
};

// Exact node box of the cells in [mn, mx] (per axis, cell coordinates), reduced over
// the block; empty when no point was inside the grid.  Consecutive calls alternate
// between two scratch rows (`parity`), so one barrier per call suffices: a row is
// rewritten only after every thread has passed the barrier of the call in between.
__device__ __forceinline__ Box block_box(ScatSmem& s, int (&mn)[3], int (&mx)[3], unsigned& parity) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int (*red)[6] = s.red[parity & 1u];
  ++parity;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    mn[d] = __reduce_min_sync(0xffffffffu, mn[d]);
    mx[d] = __reduce_max_sync(0xffffffffu, mx[d]);
  }
  if (lane == 0)
    for (int d = 0; d < 3; ++d) { red[warp][d] = mn[d]; red[warp][3 + d] = mx[d]; }
  __syncthreads();
  Box bx;
  for (int d = 0; d < 3; ++d) {
    int lo = red[0][d], hi = red[0][3 + d];
    for (int q = 1; q < SNT / 32; ++q) { lo = min(lo, red[q][d]); hi = max(hi, red[q][3 + d]); }
    bx.lo[d] = lo;
    bx.n[d] = hi >= lo ? hi - lo + 2 : 0;
  }
  bx.ncells = bx.n[0] ? (bx.n[0] - 1) * (bx.n[1] - 1) * (bx.n[2] - 1) : 0;
  bx.ok = bx.ncells > 0 && bx.ncells <= CCAP && bx.n[0] * bx.n[1] * bx.n[2] <= NCAP;
  return bx;
}

// Adds the eight corner weights of one point (wg entry v) times its dL/dy into a.
template <int C>
__device__ __forceinline__ void add_corners(float (&a)[8][C], const float4 v) {
  const float wx = v.x, wy = v.y, wz = v.z, ax = 1.f - wx, ay = 1.f - wy, az = 1.f - wz;
  const float zy[4] = {az * ay, az * wy, wz * ay, wz * wy};
  const float2 g = unpack_bf16(__float_as_uint(v.w));
  const float ge[2] = {g.x, g.y};
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float wt = zy[k >> 1] * ((k & 1) ? wx : ax);
#pragma unroll
    for (int e = 0; e < C; ++e) a[k][e] = fmaf(wt, ge[e], a[k][e]);
  }
}

// Counting sort of the points with id >= 0 by cell (each already holds its rank rk
// among its cell's points, taken with an atomic on s.cnt), per-cell corner sums, node
// gather and one atomic per nonzero node of the box.  Leaves s.cnt zero.  The corner sums are balanced over threads: thread t sums the sorted
// positions 4t..4t+3 run by run.  A run that is a whole cell is stored as the cell's
// sum; the chunk's last run, when its cell goes on into the next chunk, is parked in
// pl[.][t]; the chunk's first run, when its cell began in an earlier chunk, is that
// cell's last piece, and this thread adds the parked pieces of the cell's earlier
// chunks to it and stores the sum.
// Corner k's C sums of cell l (a float2 when C = 2) in the layouts of ScatSmem.
template <int C>
__device__ __forceinline__ void put_sums(float* base, int k, int l, int cap, const float (&a)[8][C]) {
  if (C == 2) *reinterpret_cast<float2*>(base + ((k * cap + l) << 1)) = make_float2(a[k][0], a[k][C - 1]);
  else base[k * cap + l] = a[k][0];
}
template <int C>
__device__ __forceinline__ void add_sums(const float* base, int k, int l, int cap, float (&a)[8][C]) {
  if (C == 2) {
    const float2 v = *reinterpret_cast<const float2*>(base + ((k * cap + l) << 1));
    a[k][0] += v.x;
    a[k][C - 1] += v.y;
  } else {
    a[k][0] += base[k * cap + l];
  }
}

template <int C>
__device__ void box_pass(ScatSmem& s, const Box& bx, float* dFi, int R, const short (&id)[PPT],
                         const int (&rk)[PPT]) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ncx = bx.n[0] - 1, ncy = bx.n[1] - 1, ncz = bx.n[2] - 1, ncells = bx.ncells;
  {  // cells without points must read as zero in the gather
    const int n4 = (ncells * C + 3) >> 2;   // float4 per corner row
    for (int l = tid; l < n4; l += SNT)
#pragma unroll
      for (int k = 0; k < 8; ++k) reinterpret_cast<float4*>(s.cs + k * CCAP * C)[l] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();   // the callers took every point's rank in its cell (s.cnt) before
  {  // block-wide exclusive scan, two consecutive cells per thread
    const int l0 = 2 * tid;
    const int c0 = l0 < ncells ? s.cnt[l0] : 0, c1 = l0 + 1 < ncells ? s.cnt[l0 + 1] : 0;
    const int run = c0 + c1;
    int incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) s.wsum[warp] = incl;
    __syncthreads();
    int base = 0;
    for (int q = 0; q < warp; ++q) base += s.wsum[q];
    const int ex = base + incl - run;
    if (l0 < ncells) s.cnt[l0] = ex;
    if (l0 + 1 < ncells) s.cnt[l0 + 1] = ex + c0;
    if (tid == SNT - 1) s.cnt[ncells] = base + incl;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < PPT; ++j)
    if (rk[j] >= 0) {
      const int pos = s.cnt[id[j]] + rk[j];
      s.perm[pos] = (unsigned short)(tid + SNT * j);
      s.pcell[pos] = (unsigned short)id[j];
    }
  __syncthreads();
  const int n_act = s.cnt[ncells];
  const int q0 = 4 * tid;
  int head_cell = -1, head_from = 0;   // the chunk's first run, when its cell began in an earlier chunk
  if (q0 < n_act) {
    const int nq = min(4, n_act - q0);
    const uint2 pp = *reinterpret_cast<const uint2*>(s.perm + q0);
    const uint2 pc = *reinterpret_cast<const uint2*>(s.pcell + q0);
    const int idx[4] = {(int)(pp.x & 0xffffu), (int)(pp.x >> 16), (int)(pp.y & 0xffffu), (int)(pp.y >> 16)};
    const int cel[4] = {(int)(pc.x & 0xffffu), (int)(pc.x >> 16), (int)(pc.y & 0xffffu), (int)(pc.y >> 16)};
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = u < nq ? s.wg[idx[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int start0 = s.cnt[cel[0]];
    float a[8][C];
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int e = 0; e < C; ++e) a[k][e] = 0.f;
    int cur = cel[0];
    bool first = true;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (u < nq) {
        if (u > 0 && cel[u] != cur) {   // cell cur ended inside the chunk
          if (first && start0 < q0) head_cell = cur;
#pragma unroll
          for (int k = 0; k < 8; ++k) put_sums<C>(s.cs, k, cur, CCAP, a);
#pragma unroll
          for (int k = 0; k < 8; ++k)
#pragma unroll
            for (int e = 0; e < C; ++e) a[k][e] = 0.f;
          cur = cel[u];
          first = false;
        }
        add_corners<C>(a, v[u]);
      }
    }
    if (s.cnt[cur + 1] > q0 + 4) {   // the last run goes on into the next chunk
#pragma unroll
      for (int k = 0; k < 8; ++k) put_sums<C>(s.pl, k, tid, SNT, a);
    } else {
      if (first && start0 < q0) head_cell = cur;
#pragma unroll
      for (int k = 0; k < 8; ++k) put_sums<C>(s.cs, k, cur, CCAP, a);
    }
    head_from = start0 >> 2;
  }
  __syncthreads();
  if (head_cell >= 0) {   // last piece of a cell spanning chunks head_from .. tid
    float acc[8][C], acc2[8][C];   // two chunks per iteration: independent loads in flight
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int e = 0; e < C; ++e) { acc[k][e] = 0.f; acc2[k][e] = 0.f; }
#pragma unroll
    for (int k = 0; k < 8; ++k) add_sums<C>(s.cs, k, head_cell, CCAP, acc);
    int j = head_from;
    for (; j + 1 < tid; j += 2)
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        add_sums<C>(s.pl, k, j, SNT, acc);
        add_sums<C>(s.pl, k, j + 1, SNT, acc2);
      }
    if (j < tid)
#pragma unroll
      for (int k = 0; k < 8; ++k) add_sums<C>(s.pl, k, j, SNT, acc);
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int e = 0; e < C; ++e) acc[k][e] += acc2[k][e];
#pragma unroll
    for (int k = 0; k < 8; ++k) put_sums<C>(s.cs, k, head_cell, CCAP, acc);
  }
  __syncthreads();
  for (int l = tid; l <= ncells; l += SNT) s.cnt[l] = 0;   // ready for the next pass
  const int nodes = bx.n[0] * bx.n[1] * bx.n[2];
  const float inv_x = 1.f / (float)bx.n[0], inv_xy = 1.f / (float)(bx.n[0] * bx.n[1]);
  const int sy = ncx, sz = ncx * ncy;   // cell index strides
  for (int q = tid; q < nodes; q += SNT) {
    const int qz = (int)(((float)q + 0.5f) * inv_xy);
    const int rxy = q - qz * bx.n[0] * bx.n[1];
    const int qy = (int)(((float)rxy + 0.5f) * inv_x);
    const int qx = rxy - qy * bx.n[0];
    // node (qx, qy, qz) is corner k = (dx, dy, dz) of cell (qx - dx, qy - dy, qz - dz)
    const int l0 = (qz * ncy + qy) * ncx + qx;
    const bool x0 = qx < ncx, x1 = qx > 0, y0 = qy < ncy, y1 = qy > 0, z0 = qz < ncz, z1 = qz > 0;
    float v[C];
#pragma unroll
    for (int e = 0; e < C; ++e) v[e] = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const bool in = ((k & 1) ? x1 : x0) && ((k & 2) ? y1 : y0) && ((k & 4) ? z1 : z0);
      if (in) {
        const int l = l0 - ((k & 1) ? 1 : 0) - ((k & 2) ? sy : 0) - ((k & 4) ? sz : 0);
        if (C == 2) {
          const float2 w = *reinterpret_cast<const float2*>(s.cs + ((k * CCAP + l) << 1));
          v[0] += w.x;
          v[C - 1] += w.y;
        } else {
          v[0] += s.cs[k * CCAP + l];
        }
      }
    }
    const int64_t g = ((int64_t)(bx.lo[2] + qz) * R + (bx.lo[1] + qy)) * R + bx.lo[0] + qx;
    if (C == 2) {
      if (v[0] != 0.f || v[C - 1] != 0.f)
        atomicAdd(reinterpret_cast<float2*>(dFi) + g, make_float2(v[0], v[C - 1]));
    } else {
      if (v[0] != 0.f) atomicAdd(dFi + g, v[0]);
    }
  }
  __syncthreads();
}

// Cell of a point from its grid coordinates (the clamped s of Eq. 2).
__device__ __forceinline__ void cell_of(const float4 w, int R, int& cx, int& cy, int& cz) {
  cx = min((int)w.x, R - 2);
  cy = min((int)w.y, R - 2);
  cz = min((int)w.z, R - 2);
}

// Box pass over this thread's points whose chunk j is in the mask jm (bit j), read from
// s.wg.  Returns false, having changed nothing, when their box does not fit in shared
// memory; otherwise replaces their grid coordinates in s.wg by cell weights and runs
// the pass.
template <int C>
__device__ bool masked_pass(ScatSmem& s, unsigned jm, float* dFi, int R, unsigned& parity) {
  int mn[3] = {1 << 20, 1 << 20, 1 << 20}, mx[3] = {-1, -1, -1};
#pragma unroll
  for (int j = 0; j < PPT; ++j)
    if ((jm >> j) & 1u) {
      const float4 w = s.wg[threadIdx.x + SNT * j];
      if (__float_as_uint(w.w) & 0x7fff7fffu) {
        int cx, cy, cz;
        cell_of(w, R, cx, cy, cz);
        mn[0] = min(mn[0], cx); mn[1] = min(mn[1], cy); mn[2] = min(mn[2], cz);
        mx[0] = max(mx[0], cx); mx[1] = max(mx[1], cy); mx[2] = max(mx[2], cz);
      }
    }
  const Box bx = block_box(s, mn, mx, parity);   // block-uniform
  if (bx.n[0] == 0) return true;
  if (!bx.ok) return false;
  short id[PPT];
  int rk[PPT];
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    id[j] = -1;
    rk[j] = -1;
    if ((jm >> j) & 1u) {
      const int p = threadIdx.x + SNT * j;
      const float4 w = s.wg[p];
      if (__float_as_uint(w.w) & 0x7fff7fffu) {
        int cx, cy, cz;
        cell_of(w, R, cx, cy, cz);
        id[j] = (short)(((cz - bx.lo[2]) * (bx.n[1] - 1) + (cy - bx.lo[1])) * (bx.n[0] - 1) + (cx - bx.lo[0]));
        s.wg[p] = make_float4(w.x - (float)cx, w.y - (float)cy, w.z - (float)cz, w.w);
        rk[j] = atomicAdd(s.cnt + id[j], 1);
      }
    }
  }
  box_pass<C>(s, bx, dFi, R, id, rk);
  return true;
}

// Largest Morton level (a range of 2^L units) whose block keeps the node box of a
// grid with R nodes per axis, mapped without distortion, within 80% of the capacities.
int scat_lmax(int R) {
  const double cells_per_unit = (double)(R - 1) / (double)(1 << kUnitBits);
  for (int L = 5; L > 0; --L) {
    const int ext[3] = {1 << ((L + 2) / 3), 1 << ((L + 1) / 3), 1 << (L / 3)};
    int64_t cells = 1, nodes = 1;
    for (int d = 0; d < 3; ++d) {
      const int c = (int)std::ceil(ext[d] * cells_per_unit) + 1;
      cells *= c;
      nodes *= c + 1;
    }
    if (cells <= CCAP * 4 / 5 && nodes <= NCAP * 4 / 5) return L;
  }
  return 0;
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

// One CTA per brick.  Units without a recorded start take the next recorded one (a
// suffix minimum; for a sorted batch this is exact, for any batch the starts become
// non-decreasing from 0 to n, so the tiles below always partition the brick's points).  Every unit
// then belongs to the largest aligned range of 2^L units (L <= lmax) holding at most ST
// points; each such range becomes ceil(points / ST) tiles of consecutive points.
__global__ void __launch_bounds__(1024) k_tile_list(Bricks brp, TrainWs ws, int lmax) {
  constexpr int UPT = kUnits / 1024;
  __shared__ Bricks br;
  __shared__ int32_t st[kUnits + 1];
  __shared__ int32_t wred[32];
  __shared__ int32_t gbase;
  load_bricks(brp, br);
  __syncthreads();
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t o = br.off[b];
  const int32_t n = (int32_t)(br.off[b + 1] - o);
  const int32_t* us = ws.ustart + (int64_t)b * (kUnits + 1);
  int32_t loc[UPT];
  {
    int32_t m = INT_MAX;
#pragma unroll
    for (int k = UPT - 1; k >= 0; --k) {
      const int32_t v = us[tid * UPT + k];
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
      if (st[a + (1 << l)] - st[a] <= ST) { L = l; break; }
    }
    lv[k] = L;
    nt[k] = 0;
    if ((u & ((1 << L) - 1)) == 0) nt[k] = (st[u + (1 << L)] - st[u] + ST - 1) / ST;
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
  const float h = 0.5f * (float)(R - 1);
  uint32_t blo = 0, bn = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float umin = __ldg(g + 4 * d + 3), umax = umin;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float a = __ldg(g + 4 * d + k);
      const float p = a * lo[k], q = a * hi[k];
      umin += fminf(p, q);
      umax += fmaxf(p, q);
    }
    if (umax < -1.f || umin > 1.f) return make_uint2(0u, 0u);
    const float s0 = fminf(fmaxf(fmaf(umin, h, h) - 1e-3f, 0.f), (float)(R - 1));
    const float s1 = fminf(fmaxf(fmaf(umax, h, h) + 1e-3f, 0.f), (float)(R - 1));
    const int c0 = min((int)s0, R - 2), c1 = min((int)s1, R - 2);
    blo |= (uint32_t)c0 << (8 * d);
    bn |= (uint32_t)(c1 - c0 + 2) << (8 * d);
  }
  return make_uint2(blo, bn);
}

template <int C>
__global__ void __launch_bounds__(SNT, 3)
k_scat(Model md, Grads gr, Bricks brp, TrainWs ws, const float* __restrict__ xyz) {
  extern __shared__ __align__(16) unsigned char smraw[];
  ScatSmem& s = *reinterpret_cast<ScatSmem*>(smraw);
  __shared__ Bricks br;
  __shared__ ScatTile cur_tile;
  load_bricks(brp, br);
  const int tid = threadIdx.x;
  const int M = md.M, R = md.R;
  for (int l = tid; l <= CCAP; l += SNT) s.cnt[l] = 0;
  const int ntiles = ws.tile_ctr[0];
  const int64_t ntot = br.off[br.n];
  const int64_t gsz = (int64_t)R * R * R * C;
  unsigned parity = 0;
  for (;;) {
    // tiles are taken in list order (brick by brick, Morton order inside a brick), so
    // the CTAs on the GPU at one time work on neighbouring blocks of one brick
    if (tid == 0) {
      const int t = atomicAdd(ws.tile_ctr + 1, 1);
      ScatTile T;
      T.start = 0; T.count = -1; T.code = 0;
      if (t < ntiles) T = ws.tiles[t];
      cur_tile = T;
    }
    __syncthreads();
    const ScatTile T = cur_tile;
    if (T.count < 0) break;
    const int b = (int)(T.code >> 20);
    const int64_t p0 = T.start;
    const int np = T.count;
    const float* Gb = md.G + (int64_t)b * md.sG;
    for (int i = tid; i < M; i += SNT) s.tbox[i] = tile_box(T.code, Gb + 12 * i, R);
    float px[PPT], py[PPT], pz[PPT];   // this thread's points (tid + 256 j), kept in registers
    bool mine_in = true;               // every point of this thread lies in the tile's block
    const int lvl = (int)((T.code >> 16) & 15u);
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const int p = tid + SNT * j;
      px[j] = py[j] = pz[j] = 0.f;
      if (p < np) {
        px[j] = xyz[3 * (p0 + p)]; py[j] = xyz[3 * (p0 + p) + 1]; pz[j] = xyz[3 * (p0 + p) + 2];
        mine_in &= (((morton_bin(px[j], py[j], pz[j]) >> 3) ^ (T.code & 0xffffu)) >> lvl) == 0u;
      }
    }
    const unsigned act = (1u << ((np + SNT - 1) / SNT)) - 1u;   // chunks holding points
    // dL/dy of grid i is loaded one grid ahead, so its latency hides behind grid i-1
    uint32_t dyn[PPT];
    auto load_dy = [&](int i) {
#pragma unroll
      for (int j = 0; j < PPT; ++j) {
        const int p = tid + SNT * j;
        dyn[j] = 0u;
        if (p < np) {
          if (C == 2) dyn[j] = __ldg(reinterpret_cast<const unsigned int*>(ws.dY) + (int64_t)i * ntot + p0 + p);
          else dyn[j] = (uint32_t)__bfloat16_as_ushort(ws.dY[(int64_t)i * ntot + p0 + p]);
        }
      }
    };
    load_dy(0);
    // s.tbox; the block's boxes bound the points only if all of them lie in the block
    // (always, for a Morton-sorted batch)
    const bool in_block = __syncthreads_and(mine_in) != 0;
    for (int i = 0; i < M; ++i) {
      uint32_t dcur[PPT];
#pragma unroll
      for (int j = 0; j < PPT; ++j) dcur[j] = dyn[j];
      if (i + 1 < M) load_dy(i + 1);
      const uint2 tb = s.tbox[i];
      if (in_block && tb.y == 0u) continue;   // the block lies outside grid i
      float gi[12];
      {
        const float4* g4 = reinterpret_cast<const float4*>(Gb + 12 * i);
        const float4 a = __ldg(g4), c = __ldg(g4 + 1), d = __ldg(g4 + 2);
        gi[0] = a.x; gi[1] = a.y; gi[2] = a.z; gi[3] = a.w; gi[4] = c.x; gi[5] = c.y;
        gi[6] = c.z; gi[7] = c.w; gi[8] = d.x; gi[9] = d.y; gi[10] = d.z; gi[11] = d.w;
      }
      float* dFi = gr.dF + (int64_t)b * gr.sF + i * gsz;
      Box bx;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        bx.lo[d] = (int)((tb.x >> (8 * d)) & 0xffu);
        bx.n[d] = (int)((tb.y >> (8 * d)) & 0xffu);
      }
      bx.ncells = (bx.n[0] - 1) * (bx.n[1] - 1) * (bx.n[2] - 1);
      bx.ok = in_block && bx.ncells <= CCAP && bx.n[0] * bx.n[1] * bx.n[2] <= NCAP;
      if (bx.ok) {   // block-uniform
        short id[PPT];
        int rk[PPT];
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
          const int p = tid + SNT * j;
          id[j] = -1;
          rk[j] = -1;
          if (p < np) {
            float ux, uy, uz;
            affine(gi, px[j], py[j], pz[j], ux, uy, uz);
            const Cell c = make_cell(ux, uy, uz, R);
            if (c.inside && (dcur[j] & 0x7fff7fffu)) {
              const int lx = c.cx - bx.lo[0], ly = c.cy - bx.lo[1], lz = c.cz - bx.lo[2];
              if (lx >= 0 && ly >= 0 && lz >= 0 && lx < bx.n[0] - 1 && ly < bx.n[1] - 1 && lz < bx.n[2] - 1) {
                id[j] = (short)((lz * (bx.n[1] - 1) + ly) * (bx.n[0] - 1) + lx);
                s.wg[p] = make_float4(c.wx, c.wy, c.wz, __uint_as_float(dcur[j]));
                rk[j] = atomicAdd(s.cnt + id[j], 1);
              } else {   // outside the block's box (rounding at its faces): add the corners directly
                const float2 g = unpack_bf16(dcur[j]);
                scatter_point(dFi, c, R, C, g.x, g.y);
              }
            }
          }
        }
        box_pass<C>(s, bx, dFi, R, id, rk);
        continue;
      }
      // the block's box is too large, or does not bound the points: exact boxes of the
      // points, of each half, of each 256-point chunk, else the chunk's points add their
      // corners directly
#pragma unroll
      for (int j = 0; j < PPT; ++j) {
        const int p = tid + SNT * j;
        if (!((act >> j) & 1u)) continue;
        float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
        if (p < np) {
          float ux, uy, uz;
          affine(gi, px[j], py[j], pz[j], ux, uy, uz);
          const Cell c = make_cell(ux, uy, uz, R);
          w = make_float4((float)c.cx + c.wx, (float)c.cy + c.wy, (float)c.cz + c.wz,
                          __uint_as_float(c.inside ? dcur[j] : 0u));
        }
        s.wg[p] = w;
      }
      if (masked_pass<C>(s, act, dFi, R, parity)) continue;
#pragma unroll
      for (int h = 0; h < PPT / 2; ++h) {
        const unsigned hm = (3u << (2 * h)) & act;
        if (!hm) continue;
        if (hm != act && masked_pass<C>(s, hm, dFi, R, parity)) continue;
#pragma unroll
        for (int c = 2 * h; c < 2 * h + 2; ++c) {
          const unsigned cm = 1u << c;
          if (!(act & cm)) continue;
          if (cm != hm && masked_pass<C>(s, cm, dFi, R, parity)) continue;
          const float4 w = s.wg[tid + SNT * c];
          if (__float_as_uint(w.w) & 0x7fff7fffu) {
            Cell cl;
            cell_of(w, R, cl.cx, cl.cy, cl.cz);
            cl.wx = w.x - (float)cl.cx; cl.wy = w.y - (float)cl.cy; cl.wz = w.z - (float)cl.cz;
            const float2 g = unpack_bf16(__float_as_uint(w.w));
            scatter_point(dFi, cl, R, C, g.x, g.y);
          }
        }
      }
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
  const int64_t ntot = br.off[br.n];
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
        const float2 d = unpack_bf16(__ldg(reinterpret_cast<const unsigned int*>(ws.dY) + (int64_t)gi * ntot + p0 + p));
        g0 = d.x;
        g1 = d.y;
      } else {
        g0 = __bfloat162float(ws.dY[(int64_t)gi * ntot + p0 + p]);
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

template <int K>
cudaError_t launch_train_k(const Launch& L, bool dens, const Model& md, const Grads& gr, const Bricks& br,
                           const TrainWs& ws, const float* xyz, const float* target, const KernelMark* mark) {
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
    if ((e = cudaMemsetAsync(ws.ustart, 0xff, sizeof(int32_t) * (kUnits + 1) * br.n, L.stream)) != cudaSuccess)
      return e;
    if ((e = cudaMemsetAsync(ws.tile_ctr, 0, 2 * sizeof(int32_t), L.stream)) != cudaSuccess) return e;
    const int bx = (int)std::min<int64_t>((nmax + 255) / 256, 4 * L.num_sms / std::max(1, br.n) + 1);
    k_unit_starts<<<dim3(bx, br.n), 256, 0, L.stream>>>(br, xyz, ws.ustart);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_tile_list<<<br.n, 1024, 0, L.stream>>>(br, ws, scat_lmax(md.R));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  {
    const void* kern = dens ? (const void*)k_enc<K, true> : (const void*)k_enc<K, false>;
    const int grid = std::min(tiles, L.num_sms * occupancy(kern, ENT, 0));
    mark_start(0);
    if (dens) k_enc<K, true><<<grid, ENT, 0, L.stream>>>(md, br, ws, xyz);
    else k_enc<K, false><<<grid, ENT, 0, L.stream>>>(md, br, ws, xyz);
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
  {
    const size_t smem = sizeof(ScatSmem);
    mark_start(2);
    if (md.C == 2) {
      if ((e = cudaFuncSetAttribute(k_scat<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
      const int grid = L.num_sms * occupancy((const void*)k_scat<2>, SNT, smem);
      k_scat<2><<<grid, SNT, smem, L.stream>>>(md, gr, br, ws, xyz);
    } else {
      if ((e = cudaFuncSetAttribute(k_scat<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
      const int grid = L.num_sms * occupancy((const void*)k_scat<1>, SNT, smem);
      k_scat<1><<<grid, SNT, smem, L.stream>>>(md, gr, br, ws, xyz);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    mark_stop(2);
  }
  if (ws.rec_dg) {
    const int grid = std::min((int)((br.off[br.n] + RT - 1) / RT), 2 * L.num_sms);
    if (md.C == 2) k_rec_dg<2><<<grid, RNT, 0, L.stream>>>(md, br, ws, xyz);
    else k_rec_dg<1><<<grid, RNT, 0, L.stream>>>(md, br, ws, xyz);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_train_bf16(const Launch& L, bool dens, const Model& md, const Grads& gr, const Bricks& br,
                              const TrainWs& ws, const float* xyz, const float* target, const KernelMark* mark) {
  switch (md.K) {
    case 16: return launch_train_k<16>(L, dens, md, gr, br, ws, xyz, target, mark);
    case 32: return launch_train_k<32>(L, dens, md, gr, br, ws, xyz, target, mark);
    case 64: return launch_train_k<64>(L, dens, md, gr, br, ws, xyz, target, mark);
    case 128: return launch_train_k<128>(L, dens, md, gr, br, ws, xyz, target, mark);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace srn
