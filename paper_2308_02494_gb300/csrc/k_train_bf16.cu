// BF16 training pass over all bricks: three kernels, each shaped for its own bound.
//
//  k_enc   encoder (Eq. 1-3) and the feature density of Eq. 7.  Low register count,
//          several CTAs per SM to hide the latency of the corner gathers (L1/L2
//          resident BF16 grids).  Writes the features Y [N][K] (bf16) and rho [N].
//  k_mlp   decoder forward and backward on the tensor cores (mma.sync m16n8k16,
//          BF16 operands, FP32 accumulation): L_rec partial sums, h(x) = (f - v)^2,
//          dW1/dW2/dw3 accumulated in registers per CTA and flushed once, and
//          dL/dy written grid-major as bf16 (dY [M][N][C]) for the scatter.
//  k_scat  adjoint of Eq. 2.  A tile is 1024 Morton-consecutive points of one brick.
//          The CTA takes the grids one at a time: it counting-sorts the tile's points
//          by their cell in the grid's node box (integer shared-memory atomics, a
//          block-wide scan), sums each cell's eight corner contributions with plain
//          FMAs into corner-major per-cell sums, and lets every node of the box gather
//          its (up to) eight cells and add the total into the float32 gradient grid
//          with one float2 atomic.  The box is the exact bounding box of the cells the
//          tile's points occupy in that grid; when it exceeds the shared-memory
//          capacity the tile falls back to a box per 256-point chunk, then to adding
//          each point's corners directly.
#include "bf16_ops.cuh"
#include "kernels.h"
#include <algorithm>

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
  __shared__ float gs[kMaxGrids * 12];
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
#pragma unroll 2
      for (int i = gsub; i < M; i += 2) {
        float ux, uy, uz;
        affine(gs + 12 * i, pt.x, pt.y, pt.z, ux, uy, uz);
        const Cell c = make_cell(ux, uy, uz, R);
        float f0 = 0.f, f1 = 0.f;
        if (valid && c.inside) trilinear_bf16(Fb + i * gsz, c, R, C, f0, f1);
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
// corner sums (corner-major, conflict-free), the tile's points and transforms.
struct ScatSmem {
  float cs[16][CCAP];          // corner k, channel e -> cs[k*C + e][cell]
  float4 wg[ST];               // wx, wy, wz and dL/dy (bf16 x 2 bits) of each point
  int cnt[CCAP + 1];           // cell counts, then starts
  unsigned short perm[ST];     // point indices ordered by cell
  float gs[kMaxGrids * 12];    // this brick's transforms
  int red[SNT / 32][6];        // block min/max scratch
  int wsum[SNT / 32];          // block scan scratch
};

struct Box {
  int lo[3], n[3];   // first node and nodes per axis of the box
  int ncells;
  bool ok;
};

// Exact node box of the cells in [mn, mx] (per axis, cell coordinates), reduced over
// the block; empty when no point was inside the grid.
__device__ __forceinline__ Box block_box(ScatSmem& s, int (&mn)[3], int (&mx)[3]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    mn[d] = __reduce_min_sync(0xffffffffu, mn[d]);
    mx[d] = __reduce_max_sync(0xffffffffu, mx[d]);
  }
  if (lane == 0)
    for (int d = 0; d < 3; ++d) { s.red[warp][d] = mn[d]; s.red[warp][3 + d] = mx[d]; }
  __syncthreads();
  Box bx;
  for (int d = 0; d < 3; ++d) {
    int lo = s.red[0][d], hi = s.red[0][3 + d];
    for (int q = 1; q < SNT / 32; ++q) { lo = min(lo, s.red[q][d]); hi = max(hi, s.red[q][3 + d]); }
    bx.lo[d] = lo;
    bx.n[d] = hi >= lo ? hi - lo + 2 : 0;
  }
  __syncthreads();
  bx.ncells = bx.n[0] ? (bx.n[0] - 1) * (bx.n[1] - 1) * (bx.n[2] - 1) : 0;
  bx.ok = bx.ncells > 0 && bx.ncells <= CCAP && bx.n[0] * bx.n[1] * bx.n[2] <= NCAP;
  return bx;
}

// Counting sort of the points with cid >= 0 by cell, per-cell corner sums, node gather
// and one atomic per nonzero node of the box.  `mine` marks the points this thread
// registered (the ones it owns among those whose cid was written).
template <int C>
__device__ void box_pass(ScatSmem& s, const Box& bx, float* dFi, int R, const short (&id)[PPT]) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ncx = bx.n[0] - 1, ncy = bx.n[1] - 1, ncz = bx.n[2] - 1, ncells = bx.ncells;
  for (int l = tid; l <= ncells; l += SNT) s.cnt[l] = 0;
  __syncthreads();
  int rk[PPT];
#pragma unroll
  for (int j = 0; j < PPT; ++j) rk[j] = id[j] >= 0 ? atomicAdd(s.cnt + id[j], 1) : -1;
  __syncthreads();
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
    if (rk[j] >= 0) s.perm[s.cnt[id[j]] + rk[j]] = (unsigned short)(tid + SNT * j);
  __syncthreads();
  for (int l = tid; l < ncells; l += SNT) {
    float a[8][C];
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int e = 0; e < C; ++e) a[k][e] = 0.f;
    const int s1 = s.cnt[l + 1];
    for (int q0 = s.cnt[l]; q0 < s1; q0 += 4) {  // four points' loads in flight at a time
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = q0 + u < s1 ? s.wg[s.perm[q0 + u]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float wx = v[u].x, wy = v[u].y, wz = v[u].z, ax = 1.f - wx, ay = 1.f - wy, az = 1.f - wz;
        const float wt[8] = {az * ay * ax, az * ay * wx, az * wy * ax, az * wy * wx,
                             wz * ay * ax, wz * ay * wx, wz * wy * ax, wz * wy * wx};
        const float2 g = unpack_bf16(__float_as_uint(v[u].w));   // zero for the padding slots
        const float ge[2] = {g.x, g.y};
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
          for (int e = 0; e < C; ++e) a[k][e] = fmaf(wt[k], ge[e], a[k][e]);
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int e = 0; e < C; ++e) s.cs[k * C + e][l] = a[k][e];
  }
  __syncthreads();
  const int nodes = bx.n[0] * bx.n[1] * bx.n[2];
  const float inv_x = 1.f / (float)bx.n[0], inv_xy = 1.f / (float)(bx.n[0] * bx.n[1]);
  for (int q = tid; q < nodes; q += SNT) {
    const int qz = (int)(((float)q + 0.5f) * inv_xy);
    const int rxy = q - qz * bx.n[0] * bx.n[1];
    const int qy = (int)(((float)rxy + 0.5f) * inv_x);
    const int qx = rxy - qy * bx.n[0];
    float v[C];
#pragma unroll
    for (int e = 0; e < C; ++e) v[e] = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int ex = qx - (k & 1), ey = qy - ((k >> 1) & 1), ez = qz - (k >> 2);
      if (ex >= 0 && ey >= 0 && ez >= 0 && ex < ncx && ey < ncy && ez < ncz) {
        const int l = (ez * ncy + ey) * ncx + ex;
#pragma unroll
        for (int e = 0; e < C; ++e) v[e] += s.cs[k * C + e][l];
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

template <int C>
__global__ void __launch_bounds__(SNT, 3)
k_scat(Model md, Grads gr, Bricks brp, TileSizes ts, TrainWs ws, const float* __restrict__ xyz) {
  extern __shared__ __align__(16) unsigned char smraw[];
  ScatSmem& s = *reinterpret_cast<ScatSmem*>(smraw);
  __shared__ TileMap tm;
  __shared__ Bricks br;
  load_bricks(brp, br);
  const int tid = threadIdx.x;
  const int M = md.M, R = md.R;
  if (tid == 0) build_tile_map_sized(br, ts, tm);
  __syncthreads();
  const int total = tm.first[br.n];
  const int per = (total + gridDim.x - 1) / gridDim.x;
  const int tb = blockIdx.x * per, te = min(total, tb + per);
  const int64_t ntot = br.off[br.n];
  const int64_t gsz = (int64_t)R * R * R * C;
  int cur = -1;
  for (int tile = tb; tile < te; ++tile) {
    const int b = brick_of_tile(tm, br.n, tile, cur);
    if (b != cur) {
      __syncthreads();
      cur = b;
      for (int c = tid; c < M * 12; c += SNT) s.gs[c] = md.G[(int64_t)b * md.sG + c];
    }
    const int tsz = ts.t[b];
    const int64_t p0 = br.off[b] + (int64_t)(tile - tm.first[b]) * tsz;
    const int np = (int)min((int64_t)tsz, br.off[b + 1] - p0);
    float px[PPT], py[PPT], pz[PPT];   // this thread's points (tid + 256 j), kept in registers
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const int p = tid + SNT * j;
      px[j] = py[j] = pz[j] = 0.f;
      if (p < np) { px[j] = xyz[3 * (p0 + p)]; py[j] = xyz[3 * (p0 + p) + 1]; pz[j] = xyz[3 * (p0 + p) + 2]; }
    }
    __syncthreads();
    for (int i = 0; i < M; ++i) {
      const float* gi = s.gs + 12 * i;
      float* dFi = gr.dF + (int64_t)b * gr.sF + i * gsz;
      const uint32_t* dY32 = reinterpret_cast<const uint32_t*>(ws.dY) + (int64_t)i * ntot + p0;
      const __nv_bfloat16* dY16 = ws.dY + (int64_t)i * ntot + p0;
      // the thread's points: cell, weights and dL/dy, and the cells' bounds
      Cell cl[PPT];
      float g0[PPT], g1[PPT];
      bool on[PPT];
      int mn[3] = {1 << 20, 1 << 20, 1 << 20}, mx[3] = {-1, -1, -1};
#pragma unroll
      for (int j = 0; j < PPT; ++j) {
        const int p = tid + SNT * j;
        on[j] = false;
        g0[j] = g1[j] = 0.f;
        if (p < np) {
          float ux, uy, uz;
          affine(gi, px[j], py[j], pz[j], ux, uy, uz);
          cl[j] = make_cell(ux, uy, uz, R);
          if (cl[j].inside) {
            if (C == 2) {
              const float2 g = unpack_bf16(dY32[p]);
              g0[j] = g.x; g1[j] = g.y;
            } else {
              g0[j] = __bfloat162float(dY16[p]);
            }
            on[j] = g0[j] != 0.f || g1[j] != 0.f;
          }
          if (on[j]) {
            mn[0] = min(mn[0], cl[j].cx); mn[1] = min(mn[1], cl[j].cy); mn[2] = min(mn[2], cl[j].cz);
            mx[0] = max(mx[0], cl[j].cx); mx[1] = max(mx[1], cl[j].cy); mx[2] = max(mx[2], cl[j].cz);
          }
        }
      }
      Box bx = block_box(s, mn, mx);
      if (bx.n[0] == 0) continue;   // block-uniform: no contribution to grid i
      if (bx.ok) {
        short id[PPT];
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
          id[j] = -1;
          if (on[j]) {
            const int p = tid + SNT * j;
            id[j] = (short)(((cl[j].cz - bx.lo[2]) * (bx.n[1] - 1) + (cl[j].cy - bx.lo[1])) * (bx.n[0] - 1) +
                            (cl[j].cx - bx.lo[0]));
            s.wg[p] = make_float4(cl[j].wx, cl[j].wy, cl[j].wz, __uint_as_float(pack_bf16(g0[j], g1[j])));
          }
        }
        box_pass<C>(s, bx, dFi, R, id);
        continue;
      }
      // the tile's box is too large: a box per 256-point chunk (point j of every thread)
#pragma unroll
      for (int c = 0; c < PPT; ++c) {
        int cmn[3] = {1 << 20, 1 << 20, 1 << 20}, cmx[3] = {-1, -1, -1};
        if (on[c]) {
          cmn[0] = cmx[0] = cl[c].cx; cmn[1] = cmx[1] = cl[c].cy; cmn[2] = cmx[2] = cl[c].cz;
        }
        const Box cb = block_box(s, cmn, cmx);
        if (cb.n[0] == 0) continue;
        if (cb.ok) {
          short id[PPT];
#pragma unroll
          for (int j = 0; j < PPT; ++j) id[j] = -1;
          if (on[c]) {
            const int p = tid + SNT * c;
            id[c] = (short)(((cl[c].cz - cb.lo[2]) * (cb.n[1] - 1) + (cl[c].cy - cb.lo[1])) * (cb.n[0] - 1) +
                            (cl[c].cx - cb.lo[0]));
            s.wg[p] = make_float4(cl[c].wx, cl[c].wy, cl[c].wz, __uint_as_float(pack_bf16(g0[c], g1[c])));
          }
          box_pass<C>(s, cb, dFi, R, id);
        } else if (on[c]) {
          scatter_point(dFi, cl[c], R, C, g0[c], g1[c]);
        }
      }
    }
    __syncthreads();
  }
}

int occupancy(const void* kern, int threads, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem) != cudaSuccess || n < 1) n = 1;
  return n;
}

template <int K>
cudaError_t launch_train_k(const Launch& L, bool dens, const Model& md, const Grads& gr, const Bricks& br,
                           const TrainWs& ws, const float* xyz, const float* target) {
  int tiles = 0;
  for (int b = 0; b < br.n; ++b) tiles += (int)((br.off[b + 1] - br.off[b] + ET - 1) / ET);
  if (tiles == 0) return cudaSuccess;
  cudaError_t e;
  {
    const void* kern = dens ? (const void*)k_enc<K, true> : (const void*)k_enc<K, false>;
    const int grid = std::min(tiles, L.num_sms * occupancy(kern, ENT, 0));
    if (dens) k_enc<K, true><<<grid, ENT, 0, L.stream>>>(md, br, ws, xyz);
    else k_enc<K, false><<<grid, ENT, 0, L.stream>>>(md, br, ws, xyz);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  {
    const int smem = MlpLay<K>::BYTES;
    if ((e = cudaFuncSetAttribute(k_mlp<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
      return e;
    const int grid = std::min(tiles, L.num_sms);
    k_mlp<K><<<grid, NT, smem, L.stream>>>(md, gr, br, ws, target);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  {
    const size_t smem = sizeof(ScatSmem);
    // per-brick tile size: the largest power of two <= ST whose expected cell count in
    // a grid (tile points x cells per point) stays near 128, so boxes fit in most tiles
    TileSizes ts{};
    int stiles = 0;
    const double cells = (double)(md.R - 1) * (md.R - 1) * (md.R - 1);
    for (int b = 0; b < br.n; ++b) {
      const int64_t nb = br.off[b + 1] - br.off[b];
      int t = ST;
      while (t > 128 && (double)t * cells > 128.0 * (double)(nb > 0 ? nb : 1)) t >>= 1;
      ts.t[b] = t;
      stiles += (int)((nb + t - 1) / t);
    }
    if (md.C == 2) {
      if ((e = cudaFuncSetAttribute(k_scat<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
      const int grid = std::min(stiles, L.num_sms * occupancy((const void*)k_scat<2>, SNT, smem));
      k_scat<2><<<grid, SNT, smem, L.stream>>>(md, gr, br, ts, ws, xyz);
    } else {
      if ((e = cudaFuncSetAttribute(k_scat<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
      const int grid = std::min(stiles, L.num_sms * occupancy((const void*)k_scat<1>, SNT, smem));
      k_scat<1><<<grid, SNT, smem, L.stream>>>(md, gr, br, ts, ws, xyz);
    }
    return cudaGetLastError();
  }
}

}  // namespace

cudaError_t launch_train_bf16(const Launch& L, bool dens, const Model& md, const Grads& gr, const Bricks& br,
                              const TrainWs& ws, const float* xyz, const float* target) {
  switch (md.K) {
    case 16: return launch_train_k<16>(L, dens, md, gr, br, ws, xyz, target);
    case 32: return launch_train_k<32>(L, dens, md, gr, br, ws, xyz, target);
    case 64: return launch_train_k<64>(L, dens, md, gr, br, ws, xyz, target);
    case 128: return launch_train_k<128>(L, dens, md, gr, br, ws, xyz, target);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace srn
