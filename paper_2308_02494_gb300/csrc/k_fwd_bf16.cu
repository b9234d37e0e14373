// BF16 forward query f(x) = d(e(x)) (Eq. 1-3 and Sec. 4.1.2) for srn_forward and the
// renderer.  Persistent CTAs walk contiguous ranges of 128-point tiles over all
// bricks; per tile, thread (point, half of the grids) evaluates Eq. 1 in registers
// and Eq. 2 by eight corner loads of the BF16 grid, the features go to shared memory
// (BF16, swizzled), and warp w runs the two hidden layers for rows 16w..16w+15 on the
// tensor cores (m16n8k16, FP32 accumulate) and the 64 -> 1 output layer in FP32.
#include "bf16_ops.cuh"
#include "kernels.h"

namespace srn {
namespace {

constexpr int T = 128;
constexpr int NT = 256;

template <int K>
struct FwdLay {
  static constexpr int W1 = 0;                       // [64][K] bf16 swizzled
  static constexpr int W2 = W1 + 64 * K * 2;         // [64][64] bf16
  static constexpr int Y = W2 + 64 * 64 * 2;         // [T][K] bf16
  static constexpr int W3 = Y + T * K * 2;           // [64] f32
  static constexpr int X = W3 + 64 * 4;              // [T] float4
  static constexpr int G = X + T * 16;               // [M][12] f32
  static constexpr int BYTES = G + kMaxGrids * 12 * 4;
};

template <int K>
__global__ void __launch_bounds__(NT, 3)
k_fwd_bf16(Model md, Bricks brp, const float* __restrict__ xyz, float* __restrict__ out) {
  using L = FwdLay<K>;
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
  const uint32_t sW1 = su32(sm + L::W1), sW2 = su32(sm + L::W2), sY = su32(sm + L::Y);

  int cur = -1;
  float span = 0.f, vmin = 0.f;
  for (int tile = tb; tile < te; ++tile) {
    const int b = brick_of_tile(tm, br.n, tile, cur);
    if (b != cur) {
      __syncthreads();
      cur = b;
      const uint4* w1 = reinterpret_cast<const uint4*>(md.W1h + (int64_t)b * md.sW1);
      for (int c = tid; c < 64 * K / 8; c += NT)
        *reinterpret_cast<uint4*>(sm + L::W1 + swz<K>(c / (K / 8), (c % (K / 8)) * 8)) = w1[c];
      const uint4* w2 = reinterpret_cast<const uint4*>(md.W2h + (int64_t)b * md.sW2);
      for (int c = tid; c < 64 * 8; c += NT)
        *reinterpret_cast<uint4*>(sm + L::W2 + swz<64>(c / 8, (c % 8) * 8)) = w2[c];
      if (tid < 64) w3s[tid] = md.w3[(int64_t)b * md.sw3 + tid];
      for (int c = tid; c < M * 12; c += NT) gs[c] = md.G[(int64_t)b * md.sG + c];
      vmin = md.range[2 * b];
      span = md.range[2 * b + 1] - vmin;
      __syncthreads();
    }
    const int64_t p0 = br.off[b] + (int64_t)(tile - tm.first[b]) * T;
    const int np = (int)min((int64_t)T, br.off[b + 1] - p0);
    if (tid < T) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (tid < np) {
        const float* q = xyz + 3 * (p0 + tid);
        v.x = q[0]; v.y = q[1]; v.z = q[2];
      }
      reinterpret_cast<float4*>(xs)[tid] = v;
    }
    __syncthreads();
    {  // encode
      const __nv_bfloat16* Fb = md.F16 + (int64_t)b * md.sF;
      const int64_t gsz = (int64_t)R * R * R * C;
      const int p = (warp & 3) * 32 + lane, gsub = warp >> 2;
      const float4 pt = reinterpret_cast<const float4*>(xs)[p];
      const bool valid = p < np;
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
        if (C == 2)
          *reinterpret_cast<uint32_t*>(sm + L::Y + swz<K>(p, 2 * i)) = pack_bf16(f0, f1);
        else
          *reinterpret_cast<__nv_bfloat16*>(sm + L::Y + swz<K>(p, i)) = __float2bfloat16_rn(f0);
      }
    }
    __syncthreads();
    {  // decoder
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
      const int rlo = r0 + g8, rhi = rlo + 8;
      if (t4 == 0) {
        if (rlo < np) out[p0 + rlo] = fmaf(mlo, span, vmin);
        if (rhi < np) out[p0 + rhi] = fmaf(mhi, span, vmin);
      }
    }
    __syncthreads();
  }
}

template <int K>
cudaError_t launch_k(const Launch& L, const Model& md, const Bricks& br, const float* xyz, float* out) {
  const int smem = FwdLay<K>::BYTES;
  auto kern = k_fwd_bf16<K>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int grid = 3 * L.num_sms;
  if (!br.dev) {
    int total = 0;
    for (int b = 0; b < br.n; ++b) total += (int)((br.off[b + 1] - br.off[b] + T - 1) / T);
    if (total == 0) return cudaSuccess;
    grid = total < grid ? total : grid;
  }
  kern<<<grid, NT, smem, L.stream>>>(md, br, xyz, out);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_forward_bf16(const Launch& L, const Model& md, const Bricks& br, const float* xyz,
                                float* out) {
  switch (md.K) {
    case 16: return launch_k<16>(L, md, br, xyz, out);
    case 32: return launch_k<32>(L, md, br, xyz, out);
    case 64: return launch_k<64>(L, md, br, xyz, out);
    case 128: return launch_k<128>(L, md, br, xyz, out);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace srn
