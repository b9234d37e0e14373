// FP32 fused point-query kernel: the same computation as the BF16 kernel (encoder
// Eq. 1-3, decoder Sec. 4.1.2, L_rec backward, Eq. 7 density) entirely in float32,
// with the decoder on the SIMT pipes.  It is the full-precision reference path:
// 64-point tiles, 256 threads, every matrix product a register-blocked loop over
// shared memory.
#include "common.cuh"
#include "kernels.h"

namespace srn {
namespace {

constexpr int T = 64;
constexpr int NT = 256;

__device__ __forceinline__ void trilinear_f32(const float* Fi, const Cell& c, int R, int C,
                                              float& o0, float& o1) {
  const int64_t b = ((int64_t)c.cz * R + c.cy) * R + c.cx;
  const int64_t sy = R, sz = (int64_t)R * R;
  const float ax = 1.f - c.wx, ay = 1.f - c.wy, az = 1.f - c.wz;
  if (C == 2) {
    const float2* F = reinterpret_cast<const float2*>(Fi);
    const float2 v0 = __ldg(F + b), v1 = __ldg(F + b + 1), v2 = __ldg(F + b + sy), v3 = __ldg(F + b + sy + 1);
    const float2 v4 = __ldg(F + b + sz), v5 = __ldg(F + b + sz + 1), v6 = __ldg(F + b + sz + sy),
                 v7 = __ldg(F + b + sz + sy + 1);
    o0 = az * (ay * (ax * v0.x + c.wx * v1.x) + c.wy * (ax * v2.x + c.wx * v3.x)) +
         c.wz * (ay * (ax * v4.x + c.wx * v5.x) + c.wy * (ax * v6.x + c.wx * v7.x));
    o1 = az * (ay * (ax * v0.y + c.wx * v1.y) + c.wy * (ax * v2.y + c.wx * v3.y)) +
         c.wz * (ay * (ax * v4.y + c.wx * v5.y) + c.wy * (ax * v6.y + c.wx * v7.y));
  } else {
    const float v0 = __ldg(Fi + b), v1 = __ldg(Fi + b + 1), v2 = __ldg(Fi + b + sy), v3 = __ldg(Fi + b + sy + 1);
    const float v4 = __ldg(Fi + b + sz), v5 = __ldg(Fi + b + sz + 1), v6 = __ldg(Fi + b + sz + sy),
                v7 = __ldg(Fi + b + sz + sy + 1);
    o0 = az * (ay * (ax * v0 + c.wx * v1) + c.wy * (ax * v2 + c.wx * v3)) +
         c.wz * (ay * (ax * v4 + c.wx * v5) + c.wy * (ax * v6 + c.wx * v7));
    o1 = 0.f;
  }
}

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
  static constexpr int KP = K + 1, HP = 65;
  static constexpr int W1 = 0;                   // [64][KP]
  static constexpr int W2 = W1 + 64 * KP;        // [64][HP]
  static constexpr int Y = W2 + 64 * HP;         // [T][KP]
  static constexpr int H1 = Y + T * KP;          // [T][HP]
  static constexpr int D2 = H1 + T * HP;         // [T][HP]
  static constexpr int D1 = D2 + T * HP;         // [T][HP]
  static constexpr int DY = D1 + T * HP;         // [T][KP]
  static constexpr int W3 = DY + T * KP;         // [64]
  static constexpr int X = (W3 + 64 + 3) / 4 * 4;  // [T] float4
  static constexpr int RHO = X + 4 * T;          // [4][T]
  static constexpr int G = RHO + 4 * T;          // [M][12]
  static constexpr int DET = G + kMaxGrids * 12; // [M]
  static constexpr int RG = DET + kMaxGrids;     // [M][12] dL/dG through the features (rec_dg)
  static constexpr int FLOATS = RG + kMaxGrids * 12;
};

template <int K, int MODE>
__global__ void __launch_bounds__(NT, 1)
k_query_f32(Model md, Grads gr, Bricks brp, TrainWs ws, const float* __restrict__ xyz,
            const float* __restrict__ target, float* __restrict__ out) {
  constexpr bool TRAIN = MODE >= kTrain;
  constexpr bool DENS = MODE == kTrainDensity;
  constexpr int NC1 = K / 16;  // feature columns per thread
  using L = Lay<K>;
  extern __shared__ __align__(128) float smf[];
  __shared__ TileMap tm;
  __shared__ Bricks br;
  load_bricks(brp, br);
  float* W1s = smf + L::W1;
  float* W2s = smf + L::W2;
  float* Ys = smf + L::Y;
  float* H1s = smf + L::H1;
  float* D2s = smf + L::D2;
  float* D1s = smf + L::D1;
  float* DYs = smf + L::DY;
  float* w3s = smf + L::W3;
  float4* xs = reinterpret_cast<float4*>(smf + L::X);
  float* rhos = smf + L::RHO;
  float* gs = smf + L::G;
  float* dets = smf + L::DET;
  float* rgs = smf + L::RG;

  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int M = md.M, C = md.C, R = md.R;
  if (TRAIN && ws.rec_dg)
    for (int c = tid; c < M * 12; c += NT) rgs[c] = 0.f;
  if (tid == 0) build_tile_map(br, T, tm);
  __syncthreads();
  const int total = tm.first[br.n];
  const int per = (total + gridDim.x - 1) / gridDim.x;
  const int tb = blockIdx.x * per, te = min(total, tb + per);

  float dw1[4][NC1], dw2[4][4], dw3[4];
  double sum_r2 = 0.0, sum_rho = 0.0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
#pragma unroll
    for (int c = 0; c < NC1; ++c) dw1[r][c] = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) dw2[r][c] = 0.f;
    dw3[r] = 0.f;
  }

  auto flush = [&](int b) {
    float* gW1 = gr.dW1 + (int64_t)b * gr.sW1;
    float* gW2 = gr.dW2 + (int64_t)b * gr.sW2;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
      for (int c = 0; c < NC1; ++c) { atomicAdd(gW1 + (4 * ty + r) * K + tx + 16 * c, dw1[r][c]); dw1[r][c] = 0.f; }
#pragma unroll
      for (int c = 0; c < 4; ++c) { atomicAdd(gW2 + (4 * ty + r) * 64 + tx + 16 * c, dw2[r][c]); dw2[r][c] = 0.f; }
      atomicAdd(gr.dw3 + (int64_t)b * gr.sw3 + tx + 16 * r, dw3[r]);
      dw3[r] = 0.f;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      sum_r2 += __shfl_xor_sync(0xffffffffu, sum_r2, o);
      sum_rho += __shfl_xor_sync(0xffffffffu, sum_rho, o);
    }
    if ((tid & 31) == 0) {
      atomicAdd(ws.acc + b * kAccPerBrick + ACC_SUM_R2, sum_r2);
      if (DENS) atomicAdd(ws.acc + b * kAccPerBrick + ACC_SUM_RHO, sum_rho);
    }
    sum_r2 = 0.0;
    sum_rho = 0.0;
    if (ws.rec_dg)
      for (int c = tid; c < M * 12; c += NT) {
        atomicAdd(ws.rsum + (int64_t)b * M * 12 + c, (double)rgs[c]);
        rgs[c] = 0.f;
      }
  };

  int cur = -1;
  float span = 0.f, vmin = 0.f, inv_n = 0.f;
  for (int tile = tb; tile < te; ++tile) {
    const int b = brick_of_tile(tm, br.n, tile, cur);
    if (b != cur) {
      if (TRAIN && cur >= 0) flush(cur);
      __syncthreads();
      cur = b;
      const float* W1 = md.W1f + (int64_t)b * md.sW1;
      for (int c = tid; c < 64 * K; c += NT) W1s[(c / K) * L::KP + c % K] = W1[c];
      const float* W2 = md.W2f + (int64_t)b * md.sW2;
      for (int c = tid; c < 64 * 64; c += NT) W2s[(c / 64) * L::HP + c % 64] = W2[c];
      if (tid < 64) w3s[tid] = md.w3[(int64_t)b * md.sw3 + tid];
      const float* G = md.G + (int64_t)b * md.sG;
      for (int c = tid; c < M * 12; c += NT) gs[c] = G[c];
      if (tid < M) dets[tid] = det3(G + 12 * tid);
      vmin = md.range[2 * b];
      span = md.range[2 * b + 1] - vmin;
      inv_n = 1.f / (float)(br.off[b + 1] - br.off[b]);
      __syncthreads();
    }
    const int64_t p0 = br.off[b] + (int64_t)(tile - tm.first[b]) * T;
    const int np = (int)min((int64_t)T, br.off[b + 1] - p0);
    if (tid < T) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (tid < np) {
        const float* q = xyz + 3 * (p0 + tid);
        v.x = q[0]; v.y = q[1]; v.z = q[2];
        if (TRAIN) v.w = target[p0 + tid];
      }
      xs[tid] = v;
    }
    __syncthreads();

    // ---- encode (Eq. 1-3): point p, grids gsub, gsub+4, ...
    const float* Fb = md.F32 + (int64_t)b * md.sF;
    const int64_t gsz = (int64_t)R * R * R * C;
    {
      const int p = tid & (T - 1), gsub = tid / T;
      const float4 pt = xs[p];
      const bool valid = p < np;
      float rho = 0.f;
      for (int i = gsub; i < M; i += 4) {
        float ux, uy, uz;
        affine(gs + 12 * i, pt.x, pt.y, pt.z, ux, uy, uz);
        const Cell c = make_cell(ux, uy, uz, R);
        float f0 = 0.f, f1 = 0.f;
        if (valid && c.inside) trilinear_f32(Fb + i * gsz, c, R, C, f0, f1);
        Ys[p * L::KP + i * C] = f0;
        if (C == 2) Ys[p * L::KP + i * C + 1] = f1;
        if (DENS && valid) rho += dets[i] * flat_top(ux, uy, uz, md.p);
      }
      if (DENS) rhos[gsub * T + p] = rho;
    }
    __syncthreads();
    if (DENS && tid < np) {
      const float r = (rhos[tid] + rhos[T + tid]) + (rhos[2 * T + tid] + rhos[3 * T + tid]);
      ws.rho[p0 + tid] = r;
      sum_rho += (double)r;
    }

    // ---- z1 = Y W1^T, H1 = ReLU(z1): rows 4ty+r, columns tx+16c
    float z[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) z[r][0] = z[r][1] = z[r][2] = z[r][3] = 0.f;
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
      float y[4], w[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) y[r] = Ys[(4 * ty + r) * L::KP + k];
#pragma unroll
      for (int c = 0; c < 4; ++c) w[c] = W1s[(tx + 16 * c) * L::KP + k];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) z[r][c] = fmaf(y[r], w[c], z[r][c]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) H1s[(4 * ty + r) * L::HP + tx + 16 * c] = fmaxf(z[r][c], 0.f);
    __syncthreads();

    // ---- z2 = H1 W2^T
#pragma unroll
    for (int r = 0; r < 4; ++r) z[r][0] = z[r][1] = z[r][2] = z[r][3] = 0.f;
#pragma unroll 4
    for (int k = 0; k < 64; ++k) {
      float h[4], w[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) h[r] = H1s[(4 * ty + r) * L::HP + k];
#pragma unroll
      for (int c = 0; c < 4; ++c) w[c] = W2s[(tx + 16 * c) * L::HP + k];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) z[r][c] = fmaf(h[r], w[c], z[r][c]);
    }
    // ---- m = ReLU(z2) w3, reduced over the 16 threads sharing rows
    float m[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      float s = 0.f;
#pragma unroll
      for (int c = 0; c < 4; ++c) s = fmaf(fmaxf(z[r][c], 0.f), w3s[tx + 16 * c], s);
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      s += __shfl_xor_sync(0xffffffffu, s, 4);
      s += __shfl_xor_sync(0xffffffffu, s, 8);
      m[r] = s;
    }
    if constexpr (!TRAIN) {
      if (tx == 0) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (4 * ty + r < np) out[p0 + 4 * ty + r] = fmaf(m[r], span, vmin);
      }
      __syncthreads();
      continue;
    } else {
      float dm[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int p = 4 * ty + r;
        if (ws.upstream) {  // caller-supplied dL/df: dL/dm = dL/df (max - min)
          dm[r] = p < np ? xs[p].w * span : 0.f;
          continue;
        }
        const float e = p < np ? fmaf(m[r], span, vmin) - xs[p].w : 0.f;
        if (tx == 0 && p < np) {
          sum_r2 += (double)e * e;
          ws.herr[p0 + p] = e * e;
        }
        dm[r] = 2.f * e * span * inv_n;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float w = w3s[tx + 16 * c];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          dw3[c] = fmaf(dm[r], fmaxf(z[r][c], 0.f), dw3[c]);
          D2s[(4 * ty + r) * L::HP + tx + 16 * c] = z[r][c] > 0.f ? dm[r] * w : 0.f;
        }
      }
      __syncthreads();
      // ---- dz1 = (dz2 W2) [z1 > 0]  and  dW2 += dz2^T H1
#pragma unroll
      for (int r = 0; r < 4; ++r) z[r][0] = z[r][1] = z[r][2] = z[r][3] = 0.f;
#pragma unroll 4
      for (int k = 0; k < 64; ++k) {
        float d[4], w[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) d[r] = D2s[(4 * ty + r) * L::HP + k];
#pragma unroll
        for (int c = 0; c < 4; ++c) w[c] = W2s[k * L::HP + tx + 16 * c];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) z[r][c] = fmaf(d[r], w[c], z[r][c]);
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int idx = (4 * ty + r) * L::HP + tx + 16 * c;
          D1s[idx] = H1s[idx] > 0.f ? z[r][c] : 0.f;
        }
#pragma unroll 4
      for (int p = 0; p < T; ++p) {
        float d[4], h[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) d[r] = D2s[p * L::HP + 4 * ty + r];
#pragma unroll
        for (int c = 0; c < 4; ++c) h[c] = H1s[p * L::HP + tx + 16 * c];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) dw2[r][c] = fmaf(d[r], h[c], dw2[r][c]);
      }
      __syncthreads();
      // ---- dW1 += dz1^T Y  and  dy = dz1 W1
#pragma unroll 4
      for (int p = 0; p < T; ++p) {
        float d[4], y[NC1];
#pragma unroll
        for (int r = 0; r < 4; ++r) d[r] = D1s[p * L::HP + 4 * ty + r];
#pragma unroll
        for (int c = 0; c < NC1; ++c) y[c] = Ys[p * L::KP + tx + 16 * c];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < NC1; ++c) dw1[r][c] = fmaf(d[r], y[c], dw1[r][c]);
      }
      {
        float dy[4][NC1];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < NC1; ++c) dy[r][c] = 0.f;
#pragma unroll 4
        for (int j = 0; j < 64; ++j) {
          float d[4], w[NC1];
#pragma unroll
          for (int r = 0; r < 4; ++r) d[r] = D1s[(4 * ty + r) * L::HP + j];
#pragma unroll
          for (int c = 0; c < NC1; ++c) w[c] = W1s[j * L::KP + tx + 16 * c];
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < NC1; ++c) dy[r][c] = fmaf(d[r], w[c], dy[r][c]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < NC1; ++c) DYs[(4 * ty + r) * L::KP + tx + 16 * c] = dy[r][c];
      }
      __syncthreads();
      // ---- scatter dL/dy into the gradient grids (adjoint of Eq. 2)
      {
        const int p = tid & (T - 1), gsub = tid / T;
        if (p < np) {
          const float4 pt = xs[p];
          float* dFb = gr.dF + (int64_t)b * gr.sF;
          for (int i = gsub; i < M; i += 4) {
            float ux, uy, uz;
            affine(gs + 12 * i, pt.x, pt.y, pt.z, ux, uy, uz);
            const Cell c = make_cell(ux, uy, uz, R);
            if (!c.inside) continue;
            const float g0 = DYs[p * L::KP + i * C];
            const float g1 = C == 2 ? DYs[p * L::KP + i * C + 1] : 0.f;
            if (g0 == 0.f && g1 == 0.f) continue;
            scatter_f32(dFb + i * gsz, c, R, C, g0, g1);
          }
        }
      }
      // ---- dL/dG through the features (SRN_REC_DG): dL/du = (R-1)/2 sum_c dL/dy_c de_c/ds
      // (Eq. 2 differentiated in the cell), then dL/dA_i += dL/du x^T, dL/dt_i += dL/du;
      // each warp (32 points, one grid at a time) adds its sums into the block's rgs
      if (ws.rec_dg) {
        const int p = tid & (T - 1), gsub = tid / T;
        const float4 pt = xs[p];
        const float hs = 0.5f * (float)(R - 1);
        for (int i = gsub; i < M; i += 4) {
          float du[3] = {0.f, 0.f, 0.f};
          if (p < np) {
            float ux, uy, uz;
            affine(gs + 12 * i, pt.x, pt.y, pt.z, ux, uy, uz);
            const Cell c = make_cell(ux, uy, uz, R);
            if (c.inside) {
              const float g0 = DYs[p * L::KP + i * C];
              const float g1 = C == 2 ? DYs[p * L::KP + i * C + 1] : 0.f;
              const float* Fi = Fb + i * gsz;
              const int64_t nb = ((int64_t)c.cz * R + c.cy) * R + c.cx;
              float a[8];
#pragma unroll
              for (int k = 0; k < 8; ++k) {
                const int64_t n = nb + (k & 1) + ((k & 2) ? R : 0) + ((k & 4) ? (int64_t)R * R : 0);
                if (C == 2) {
                  const float2 f = __ldg(reinterpret_cast<const float2*>(Fi) + n);
                  a[k] = fmaf(g0, f.x, g1 * f.y);
                } else {
                  a[k] = g0 * __ldg(Fi + n);
                }
              }
              trilinear_ds(a, c.wx, c.wy, c.wz, du[0], du[1], du[2]);
#pragma unroll
              for (int d = 0; d < 3; ++d) du[d] *= hs;
            }
          }
          float v[12];
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            v[4 * d] = du[d] * pt.x; v[4 * d + 1] = du[d] * pt.y; v[4 * d + 2] = du[d] * pt.z; v[4 * d + 3] = du[d];
          }
#pragma unroll
          for (int j = 0; j < 12; ++j)
#pragma unroll
            for (int o = 16; o; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
          if ((tid & 31) == 0)
#pragma unroll
            for (int j = 0; j < 12; ++j) atomicAdd(rgs + 12 * i + j, v[j]);
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
  const int smem = Lay<K>::FLOATS * 4;
  auto kern = k_query_f32<K, MODE>;
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

cudaError_t launch_query_fp32(const Launch& L, QueryMode mode, const Model& md, const Grads& gr,
                              const Bricks& br, const TrainWs& ws, const float* xyz,
                              const float* target, float* out) {
  switch (mode) {
    case kForward: return launch_mode<kForward>(L, md, gr, br, ws, xyz, target, out);
    case kTrain: return launch_mode<kTrain>(L, md, gr, br, ws, xyz, target, out);
    default: return launch_mode<kTrainDensity>(L, md, gr, br, ws, xyz, target, out);
  }
}

}  // namespace srn
