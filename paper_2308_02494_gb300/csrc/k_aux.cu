// libsrn kernels around the fused query:
//   * the density loss: rho per point (Eq. 7) for the BF16 pass, passes 2 and 3
//     (Eq. 8, Eq. 9 and dL_den/dG) and the per-brick finalisation (losses, dG from
//     the float64 sums);
//   * Adam (Sec. 6) over the flat parameter buffer, plus the BF16 shadow refresh;
//   * the batch sampler (Philox4x32-10, then a counting sort by 32^3 Morton bin);
//   * the ground-truth lookup v(x) of Sec. 4.3.1 (trilinear in a float32 volume).
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace srn {
namespace {

__device__ __forceinline__ int brick_of_point(const Bricks& br, int64_t g) {
  int lo = 0, hi = br.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (br.off[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename Tv>
__device__ __forceinline__ Tv warp_sum(Tv v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------ density pass 1
// rho(x) = sum_i det(A_i) exp(-sum_d u_d^2p) (Eq. 7) per point and its sum S per brick,
// one thread per point over the grids; for the BF16 training pass, which runs it on the
// second stream beside the decoder (it needs only the points and the transforms).
// Tiles of RHP points come from a counter; the float32 terms of a point are summed in
// float32, the points of a brick in float64.
constexpr int RHT = 256;   // threads; one CTA fits beside two decoder CTAs (at most 56 registers)
constexpr int RHP = 2 * RHT;   // points per tile: two per thread, interleaved for latency

// exp(-sum_d u_d^2p) of Eq. 7 for p = 10, the x and y axes as a packed pair (ux, uy)
__device__ __forceinline__ float flat_top_p10(f2_t uxy, float uz) {
  const f2_t s2 = f2_mul(uxy, uxy);
  f2_t q = f2_mul(s2, s2);
  q = f2_mul(q, q);
  q = f2_mul(q, q);
  const f2_t p20 = f2_mul(f2_mul(q, s2), s2);
  const float z2 = uz * uz;
  float pz = z2 * z2;
  pz = pz * pz;
  pz = pz * pz;
  const float ssum = fmaf(pz * z2, z2, f2_lo(p20) + f2_hi(p20));
  return ssum <= 87.f ? __expf(-ssum) : 0.f;
}

template <bool P10>
__global__ void __maxnreg__(56)
k_density_rho(Model md, Bricks brp, TrainWs ws, const float* __restrict__ xyz) {
  __shared__ Bricks br;
  __shared__ TileMap tm;
  __shared__ __align__(16) float sg[kMaxGrids * 12];
  __shared__ float sdet[kMaxGrids];
  __shared__ double red[RHT / 32];
  __shared__ int s_tile;
  load_bricks(brp, br);
  const int tid = threadIdx.x, lane = tid & 31, M = md.M;
  if (tid == 0) build_tile_map(br, RHP, tm);
  __syncthreads();
  const int total = tm.first[br.n];
  double sum = 0.0;
  int cur = -1;
  auto flush = [&](int b) {   // block-uniform
    const double w = warp_sum(sum);
    if (lane == 0) red[tid >> 5] = w;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int q = 0; q < RHT / 32; ++q) t += red[q];
      atomicAdd(ws.acc + b * kAccPerBrick + ACC_SUM_RHO, t);
    }
    sum = 0.0;
  };
  for (;;) {
    if (tid == 0) s_tile = atomicAdd(ws.tile_ctr + 4, 1);
    __syncthreads();
    const int tile = s_tile;
    if (tile >= total) break;
    const int b = brick_of_tile(tm, br.n, tile, cur);
    if (b != cur) {
      if (cur >= 0) flush(cur);
      cur = b;
      // each grid's map staged as the column pairs of its x and y rows, then its z row:
      // [g0 g4 | g1 g5 | g2 g6 | g3 g7 | g8 g9 g10 g11] (g the row-major 3 x 4 map)
      const float* G = md.G + (int64_t)b * md.sG;
      for (int k = tid; k < M * 12; k += RHT) {
        const int i = k / 12, j = k - 12 * i;
        sg[k] = G[12 * i + (j < 8 ? (j >> 1) + 4 * (j & 1) : j)];
      }
      for (int i = tid; i < M; i += RHT) sdet[i] = det3(G + 12 * i);
      __syncthreads();
    }
    const int64_t pa = br.off[b] + (int64_t)(tile - tm.first[b]) * RHP + tid, pb = pa + RHT;
    const bool va = pa < br.off[b + 1], vb = pb < br.off[b + 1];
    const float xa = va ? xyz[3 * pa] : 0.f, ya = va ? xyz[3 * pa + 1] : 0.f, za = va ? xyz[3 * pa + 2] : 0.f;
    const float xb = vb ? xyz[3 * pb] : 0.f, yb = vb ? xyz[3 * pb + 1] : 0.f, zb = vb ? xyz[3 * pb + 2] : 0.f;
    float ra = 0.f, rb = 0.f;
    if constexpr (P10) {   // Eq. 1's x and y rows as packed pairs: the point's coordinates doubled once
      const f2_t xxa = f2_pack(xa, xa), yya = f2_pack(ya, ya), zza = f2_pack(za, za);
      const f2_t xxb = f2_pack(xb, xb), yyb = f2_pack(yb, yb), zzb = f2_pack(zb, zb);
#pragma unroll 2
      for (int i = 0; i < M; ++i) {
        const ulonglong2 ab = *reinterpret_cast<const ulonglong2*>(sg + 12 * i);
        const ulonglong2 cd = *reinterpret_cast<const ulonglong2*>(sg + 12 * i + 4);
        const float4 z = *reinterpret_cast<const float4*>(sg + 12 * i + 8);
        const float det = sdet[i];
        ra = fmaf(det, flat_top_p10(f2_fma(ab.x, xxa, f2_fma(ab.y, yya, f2_fma(cd.x, zza, cd.y))),
                                    fmaf(z.x, xa, fmaf(z.y, ya, fmaf(z.z, za, z.w)))), ra);
        rb = fmaf(det, flat_top_p10(f2_fma(ab.x, xxb, f2_fma(ab.y, yyb, f2_fma(cd.x, zzb, cd.y))),
                                    fmaf(z.x, xb, fmaf(z.y, yb, fmaf(z.z, zb, z.w)))), rb);
      }
    } else {
#pragma unroll 2
      for (int i = 0; i < M; ++i) {
        const float4* g4 = reinterpret_cast<const float4*>(sg + 12 * i);
        const float4 a = g4[0], c = g4[1], d = g4[2];   // (g0 g4 g1 g5), (g2 g6 g3 g7), (g8 .. g11)
        const float det = sdet[i];
        ra = fmaf(det, flat_top(fmaf(a.x, xa, fmaf(a.z, ya, fmaf(c.x, za, c.z))),
                                           fmaf(a.y, xa, fmaf(a.w, ya, fmaf(c.y, za, c.w))),
                                           fmaf(d.x, xa, fmaf(d.y, ya, fmaf(d.z, za, d.w))), md.p), ra);
        rb = fmaf(det, flat_top(fmaf(a.x, xb, fmaf(a.z, yb, fmaf(c.x, zb, c.z))),
                                           fmaf(a.y, xb, fmaf(a.w, yb, fmaf(c.y, zb, c.w))),
                                           fmaf(d.x, xb, fmaf(d.y, yb, fmaf(d.z, zb, d.w))), md.p), rb);
      }
    }
    if (va) { ws.rho[pa] = ra; sum += (double)ra; }
    if (vb) { ws.rho[pb] = rb; sum += (double)rb; }
    __syncthreads();
  }
  if (cur >= 0) flush(cur);
}

// ------------------------------------------------------------ density pass 2
// Per point: rho_s = rho/S, k = hbar/(h+eps), rho* = exp(k log(rho_s+eps)) (held
// constant), g = dL/drho_s = -rho*/(N (rho_s+eps)).  Sums per brick:
// c = sum g rho_s (needed by dL/drho = (g - c)/S) and L_den = mean rho* (k-1) log(rho_s+eps).
// Per-point scalar chain of Eq. 8 in float32 (the terms whose rho* is not negligible
// have |k log(rho_s + eps)| of order one, where float32 exp/log are accurate to a
// few ulp); each thread sums its few points in float32, every sum across threads is
// carried in float64.
struct PointDensity {
  float rs, k, lr, star, g;
};
__device__ __forceinline__ PointDensity point_density(float rho, float h, float invS, float hbar,
                                                      float eps, float n) {
  PointDensity d;
  d.rs = rho * invS;
  d.k = hbar / (h + eps);
  d.lr = logf(d.rs + eps);
  d.star = expf(d.k * d.lr);
  d.g = -d.star / (n * (d.rs + eps));
  return d;
}

constexpr int ST = 256;   // points per tile of the scalar pass

__global__ void __launch_bounds__(ST) k_density_scalar(Bricks br, TrainWs ws, float eps) {
  __shared__ TileMap tm;
  __shared__ double red[2][ST / 32];
  const int tid = threadIdx.x;
  if (tid == 0) build_tile_map(br, ST, tm);
  __syncthreads();
  const int total = tm.first[br.n];
  const int per = (total + gridDim.x - 1) / gridDim.x;
  const int tb = blockIdx.x * per, te = min(total, tb + per);
  float c_acc = 0.f, l_acc = 0.f;   // this thread's few points in float32; float64 across
  int cur = -1;
  float invS = 0.f, hbar = 0.f, n = 1.f;
  auto flush = [&](int b) {
    double cd = warp_sum((double)c_acc);
    double ld = warp_sum((double)l_acc) / (double)n;
    if ((tid & 31) == 0) { red[0][tid >> 5] = cd; red[1][tid >> 5] = ld; }
    __syncthreads();
    if (tid == 0) {
      double c = 0.0, l = 0.0;
      for (int w = 0; w < ST / 32; ++w) { c += red[0][w]; l += red[1][w]; }
      atomicAdd(ws.acc + b * kAccPerBrick + ACC_C, c);
      atomicAdd(ws.acc + b * kAccPerBrick + ACC_LDEN, l);
    }
    __syncthreads();
    c_acc = 0.f;
    l_acc = 0.f;
  };
  for (int tile = tb; tile < te; ++tile) {
    const int b = brick_of_tile(tm, br.n, tile, cur);
    if (b != cur) {
      if (cur >= 0) flush(cur);
      cur = b;
      const double nb = (double)(br.off[b + 1] - br.off[b]);
      n = (float)nb;
      invS = (float)(1.0 / ws.acc[b * kAccPerBrick + ACC_SUM_RHO]);
      hbar = (float)(ws.acc[b * kAccPerBrick + ACC_SUM_R2] / nb);
    }
    const int64_t p = br.off[b] + (int64_t)(tile - tm.first[b]) * ST + tid;
    if (p < br.off[b + 1] && !(ws.sched && !ws.sched[b].den_on)) {
      const PointDensity d = point_density(ws.rho[p], ws.herr[p], invS, hbar, eps, n);
      c_acc = fmaf(d.g, d.rs, c_acc);
      l_acc = fmaf(d.star * (d.k - 1.f), d.lr, l_acc);
    }
  }
  if (cur >= 0) flush(cur);
}

// ------------------------------------------------------------ density pass 3
// dL/drho_n = q_n = (g_n - c)/S.  For grid i, with E = exp(-sum_d u_d^2p) and
// e_d = 2p u_d^(2p-1): dL/dA_i = det_i (A_i^{-T} sum q E - sum q E e x^T),
// dL/dt_i = -det_i sum q E e.  This pass accumulates, per brick and grid, the 13
// sums  sum qE,  sum qE e_d,  sum qE e_d x_e  (float32 per thread, float64 across).
constexpr int DT = 128;   // points per tile
constexpr int DNT = 256;  // threads

static_assert(sizeof(TileMap) + DT * 2 * sizeof(float4) + kMaxGrids * 12 * sizeof(float) +
                  DNT * sizeof(double) + 1024 <= kDensityCtaSmem,
              "k_density_grad's shared memory must fit beside the scatter");
// P10: the paper's p = 10 at compile time, with the x and y axes of the map, the flat
// top and the sums carried as packed float pairs (the same arithmetic, fewer issued
// instructions); otherwise one lane per value for any p.
template <bool P10>
__global__ void __launch_bounds__(DNT, 4)
k_density_grad(Model md, Bricks br, TrainWs ws, const float* __restrict__ xyz, float eps) {
  __shared__ TileMap tm;
  __shared__ float4 sx[DT][2];   // (x, x, y, y), (z, z, q, 0): the pairs the packed path multiplies by
  __shared__ float sg[kMaxGrids * 12];
  __shared__ double red[DNT];
  __shared__ int s_tile;
  const int tid = threadIdx.x, M = md.M;
  const int npg = DNT / M;             // point groups (M divides 256)
  const int gi = tid % M, pg = tid / M;
  if (tid == 0) build_tile_map(br, DT, tm);
  __syncthreads();
  const int total = tm.first[br.n];
  // the 13 sums: sum qE; sum qE e_d (d = x, y, z); sum qE e_d x_e (d major)
  float s0 = 0.f, s3 = 0.f, s10 = 0.f, s11 = 0.f, s12 = 0.f;
  f2_t s12p = 0ull, s47 = 0ull, s58 = 0ull, s69 = 0ull;   // (s1, s2), (s4, s7), (s5, s8), (s6, s9)

  auto flush = [&](int b) {
    const float v[13] = {s0, f2_lo(s12p), f2_hi(s12p), s3, f2_lo(s47), f2_lo(s58), f2_lo(s69),
                         f2_hi(s47), f2_hi(s58), f2_hi(s69), s10, s11, s12};
#pragma unroll
    for (int j = 0; j < 13; ++j) {
      red[tid] = (double)v[j];
      __syncthreads();
      if (pg == 0) {
        double s = 0.0;
        for (int q = 0; q < npg; ++q) s += red[q * M + gi];
        atomicAdd(ws.gsum + ((int64_t)b * M + gi) * 13 + j, s);
      }
      __syncthreads();
    }
    s0 = s3 = s10 = s11 = s12 = 0.f;
    s12p = s47 = s58 = s69 = 0ull;
  };

  int cur = -1;
  float invS = 0.f, hbar = 0.f, c = 0.f, n = 1.f;
  f2_t gax = 0ull, gay = 0ull, gaz = 0ull, gt = 0ull;   // rows 0 and 1 of the map, by column
  float g8 = 0.f, g9 = 0.f, g10 = 0.f, g11 = 0.f;       // row 2
  // tiles are taken from a counter (in increasing order per CTA), so CTAs that start
  // late -- beside or after the scatter -- share the remaining work
  for (;;) {
    if (tid == 0) s_tile = atomicAdd(ws.tile_ctr + 3, 1);
    __syncthreads();
    const int tile = s_tile;
    if (tile >= total) break;
    const int b = brick_of_tile(tm, br.n, tile, cur);
    if (b != cur) {
      if (cur >= 0) flush(cur);
      cur = b;
      for (int k = tid; k < M * 12; k += DNT) sg[k] = md.G[(int64_t)b * md.sG + k];
      const double nb = (double)(br.off[b + 1] - br.off[b]);
      n = (float)nb;
      invS = (float)(1.0 / ws.acc[b * kAccPerBrick + ACC_SUM_RHO]);
      hbar = (float)(ws.acc[b * kAccPerBrick + ACC_SUM_R2] / nb);
      c = (float)ws.acc[b * kAccPerBrick + ACC_C];
      __syncthreads();
      const float* g = sg + 12 * gi;
      gax = f2_pack(g[0], g[4]); gay = f2_pack(g[1], g[5]); gaz = f2_pack(g[2], g[6]); gt = f2_pack(g[3], g[7]);
      g8 = g[8]; g9 = g[9]; g10 = g[10]; g11 = g[11];
    }
    const int64_t p0 = br.off[b] + (int64_t)(tile - tm.first[b]) * DT;
    const int np = (ws.sched && !ws.sched[b].den_on) ? 0 : (int)min((int64_t)DT, br.off[b + 1] - p0);
    if (tid < DT) {
      float x = 0.f, y = 0.f, z = 0.f, q = 0.f;
      if (tid < np) {
        const int64_t gp = p0 + tid;
        x = xyz[3 * gp]; y = xyz[3 * gp + 1]; z = xyz[3 * gp + 2];
        const PointDensity d = point_density(ws.rho[gp], ws.herr[gp], invS, hbar, eps, n);
        q = (d.g - c) * invS;
      }
      sx[tid][0] = make_float4(x, x, y, y);
      sx[tid][1] = make_float4(z, z, q, 0.f);
    }
    __syncthreads();
    if constexpr (P10) {
#pragma unroll 4
      for (int p = pg; p < np; p += npg) {
        const float4 xa = sx[p][0], xb = sx[p][1];
        const f2_t xx = f2_pack(xa.x, xa.y), yy = f2_pack(xa.z, xa.w), zz = f2_pack(xb.x, xb.y);
        const float x = xa.x, y = xa.z, z = xb.x, q = xb.z;
        // Eq. 1 (rows 0 and 1 packed, row 2 alone) and exp(-sum_d u_d^20) with 20 u_d^19
        const f2_t uxy = f2_fma(gax, xx, f2_fma(gay, yy, f2_fma(gaz, zz, gt)));
        const float uz = fmaf(g8, x, fmaf(g9, y, fmaf(g10, z, g11)));
        const f2_t s2 = f2_mul(uxy, uxy);
        f2_t t = f2_mul(s2, s2);
        t = f2_mul(t, t);
        t = f2_mul(t, t);
        const f2_t p18 = f2_mul(t, s2);   // (u_x^18, u_y^18)
        const float z2 = uz * uz;
        float pz = z2 * z2;
        pz = pz * pz;
        pz = pz * pz;
        pz = pz * z2;
        const f2_t p20 = f2_mul(p18, s2);
        const float ssum = fmaf(pz, z2, f2_lo(p20) + f2_hi(p20));
        if (!(ssum <= 87.f)) continue;   // exp underflows in float32: no contribution
        const float w = q * __expf(-ssum);
        if (w == 0.f) continue;
        const float w20 = 20.f * w;
        const f2_t wxy = f2_mul(f2_pack(w20, w20), f2_mul(p18, uxy));   // (w e_x, w e_y)
        const float wz = w20 * pz * uz;
        s0 += w;
        s12p = f2_add(s12p, wxy);
        s3 += wz;
        s47 = f2_fma(wxy, xx, s47);
        s58 = f2_fma(wxy, yy, s58);
        s69 = f2_fma(wxy, zz, s69);
        s10 = fmaf(wz, x, s10); s11 = fmaf(wz, y, s11); s12 = fmaf(wz, z, s12);
      }
    } else {
      const float* gg = sg + 12 * gi;
#pragma unroll 4
      for (int p = pg; p < np; p += npg) {
        const float4 xa = sx[p][0], xb = sx[p][1];
        const float x = xa.x, y = xa.z, z = xb.x;
        float ux, uy, uz, ex, ey, ez;
        affine(gg, x, y, z, ux, uy, uz);
        const float E = flat_top(ux, uy, uz, md.p, &ex, &ey, &ez);
        const float w = xb.z * E;
        if (w == 0.f) continue;
        const float wx = w * ex, wy = w * ey, wz = w * ez;
        s0 += w;
        s12p = f2_pack(f2_lo(s12p) + wx, f2_hi(s12p) + wy);
        s3 += wz;
        s47 = f2_pack(fmaf(wx, x, f2_lo(s47)), fmaf(wy, x, f2_hi(s47)));
        s58 = f2_pack(fmaf(wx, y, f2_lo(s58)), fmaf(wy, y, f2_hi(s58)));
        s69 = f2_pack(fmaf(wx, z, f2_lo(s69)), fmaf(wy, z, f2_hi(s69)));
        s10 = fmaf(wz, x, s10); s11 = fmaf(wz, y, s11); s12 = fmaf(wz, z, s12);
      }
    }
    __syncthreads();
  }
  if (cur >= 0) flush(cur);
}

// ------------------------------------------------------------ finalisation
// One block per brick: losses and (with the density step) dG from the sums.
__global__ void k_finalize(Bricks br, Model md, TrainWs ws, int density, float* dG, int64_t sdG,
                           double* losses) {
  const int b = blockIdx.x, i = threadIdx.x;
  const double n = (double)(br.off[b + 1] - br.off[b]);
  const double* acc = ws.acc + b * kAccPerBrick;
  if (ws.sched) density = density && ws.sched[b].den_on;
  if (ws.rec_dg && !density && i < md.M) {   // G's gradient is the part through the features alone
    const double* r = ws.rsum + ((int64_t)b * md.M + i) * 12;
    float* d = dG + (int64_t)b * sdG + 12 * i;
    for (int j = 0; j < 12; ++j) d[j] = (float)r[j];
  }
  if (density && i < md.M) {
    const float* g = md.G + (int64_t)b * md.sG + 12 * i;
    const double a00 = g[0], a01 = g[1], a02 = g[2], a10 = g[4], a11 = g[5], a12 = g[6];
    const double a20 = g[8], a21 = g[9], a22 = g[10];
    // cofactors: det * A^{-T} is the cofactor matrix
    const double c00 = a11 * a22 - a12 * a21, c01 = a12 * a20 - a10 * a22, c02 = a10 * a21 - a11 * a20;
    const double c10 = a02 * a21 - a01 * a22, c11 = a00 * a22 - a02 * a20, c12 = a01 * a20 - a00 * a21;
    const double c20 = a01 * a12 - a02 * a11, c21 = a02 * a10 - a00 * a12, c22 = a00 * a11 - a01 * a10;
    const double det = a00 * c00 + a01 * c01 + a02 * c02;
    const double* s = ws.gsum + ((int64_t)b * md.M + i) * 13;
    float* d = dG + (int64_t)b * sdG + 12 * i;
    const double cof[3][3] = {{c00, c01, c02}, {c10, c11, c12}, {c20, c21, c22}};
    const double* rs = ws.rsum + ((int64_t)b * md.M + i) * 12;
    const double rw = ws.rec_dg ? 1.0 : 0.0;   // plus the part through the features (SRN_REC_DG)
    for (int r = 0; r < 3; ++r) {
      for (int e = 0; e < 3; ++e) d[4 * r + e] = (float)(cof[r][e] * s[0] - det * s[4 + 3 * r + e] + rw * rs[4 * r + e]);
      d[4 * r + 3] = (float)(-det * s[1 + r] + rw * rs[4 * r + 3]);
    }
  }
  if (i == 0) {
    const double lrec = acc[ACC_SUM_R2] / n;
    const double lden = density ? acc[ACC_LDEN] : 0.0;
    if (!isfinite(lrec) || !isfinite(lden)) atomicOr(ws.status, 1);
    if (losses) {
      losses[4 * b + 0] = lrec;
      losses[4 * b + 1] = lden;
      losses[4 * b + 2] = density ? acc[ACC_SUM_RHO] : 0.0;
      losses[4 * b + 3] = n;
    }
  }
}

// ------------------------------------------------------------ Adam
// Advances the step counters and computes Adam's bias corrections once (double).
// Advances the step counters and Adam's bias corrections (powers of beta kept as
// running double products; a count of 1 restarts them, the state starting zeroed).
__global__ void k_advance(StepState* st, int do_b, float b1, float b2) {
  st->step += 1;
  st->t_a += 1;
  st->p1a = st->t_a == 1 ? (double)b1 : st->p1a * (double)b1;
  st->p2a = st->t_a == 1 ? (double)b2 : st->p2a * (double)b2;
  if (do_b) {
    st->t_b += 1;
    st->p1b = st->t_b == 1 ? (double)b1 : st->p1b * (double)b1;
    st->p2b = st->t_b == 1 ? (double)b2 : st->p2b * (double)b2;
  }
  st->bc1a = (float)(1.0 - st->p1a);
  st->rbc2a = (float)(1.0 / (1.0 - st->p2a));
  st->bc1b = st->t_b > 0 ? (float)(1.0 - st->p1b) : 1.f;
  st->rbc2b = st->t_b > 0 ? (float)(1.0 / (1.0 - st->p2b)) : 1.f;
}

__device__ __forceinline__ float adam1(float& p, float g, float& m, float& v, float lr, float b1,
                                       float b2, float eps, float bc1, float rbc2) {
  m = fmaf(b1, m, (1.f - b1) * g);
  v = fmaf(b2, v, (1.f - b2) * g * g);
  const float mh = m / bc1;
  const float vh = v * rbc2;
  p -= lr * mh / (sqrtf(vh) + eps);
  return p;
}

__device__ __forceinline__ void adam4(float4& P, const float4 G, float4& Mm, float4& V, float lr, float b1, float b2,
                                      float eps, float bc1, float rbc2) {
  adam1(P.x, G.x, Mm.x, V.x, lr, b1, b2, eps, bc1, rbc2);
  adam1(P.y, G.y, Mm.y, V.y, lr, b1, b2, eps, bc1, rbc2);
  adam1(P.z, G.z, Mm.z, V.z, lr, b1, b2, eps, bc1, rbc2);
  adam1(P.w, G.w, Mm.w, V.w, lr, b1, b2, eps, bc1, rbc2);
}

// Adam over one brick's five segments (blockIdx.y = brick), two float4 groups per
// thread and iteration (independent loads in flight); F and the decoder (segments
// 0-3) also refresh their BF16 shadow.  With `sched`, the brick's plateau scale
// multiplies both learning rates, a finished brick is left alone, and G is updated
// when the brick's density decision says so, with its own bias corrections.
__global__ void k_adam(AdamLayout lay, float* __restrict__ p, float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, uint16_t* __restrict__ shadow, int do_b, float lr_a, float lr_b,
                       float b1, float b2, float eps, const StepState* st, const BrickSched* sched, float pfactor,
                       int seg0, int seg1) {
  const int b = blockIdx.y;
  float mult = 1.f, bc1b = st->bc1b, rbc2b = st->rbc2b;
  bool den = do_b != 0;
  if (sched) {
    const BrickSched& q = sched[b];
    if (q.finished) return;
    for (int k = 0; k < q.plateaus; ++k) mult *= pfactor;
    den = q.den_on != 0;
    bc1b = q.bc1b;
    rbc2b = q.rbc2b;
  }
  const float bc1a = st->bc1a, rbc2a = st->rbc2a;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int sgm = seg0; sgm < seg1; ++sgm) {
    const bool a = sgm < 4;
    if (!a && !den) break;
    const int64_t base = lay.off[sgm] + (int64_t)b * lay.size[sgm];   // a multiple of 64
    const int64_t n4 = lay.size[sgm] / 4;
    float4* P4 = reinterpret_cast<float4*>(p + base);
    const float4* G4 = reinterpret_cast<const float4*>(g + base);
    float4* M4 = reinterpret_cast<float4*>(m + base);
    float4* V4 = reinterpret_cast<float4*>(v + base);
    uint2* S2 = (shadow && a) ? reinterpret_cast<uint2*>(shadow + base) : nullptr;
    const float lr = (a ? lr_a : lr_b) * mult, bc1 = a ? bc1a : bc1b, rbc2 = a ? rbc2a : rbc2b;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += 2 * stride) {
      const int64_t q2 = q + stride;
      const bool two = q2 < n4;
      float4 P = P4[q], Mm = M4[q], V = V4[q];
      const float4 Gd = G4[q];
      float4 Pb = make_float4(0.f, 0.f, 0.f, 0.f), Mb = Pb, Vb = Pb, Gb = Pb;
      if (two) { Pb = P4[q2]; Mb = M4[q2]; Vb = V4[q2]; Gb = G4[q2]; }
      adam4(P, Gd, Mm, V, lr, b1, b2, eps, bc1, rbc2);
      P4[q] = P; M4[q] = Mm; V4[q] = V;
      if (S2) S2[q] = make_uint2(pack_bf16(P.x, P.y), pack_bf16(P.z, P.w));
      if (two) {
        adam4(Pb, Gb, Mb, Vb, lr, b1, b2, eps, bc1, rbc2);
        P4[q2] = Pb; M4[q2] = Mb; V4[q2] = Vb;
        if (S2) S2[q2] = make_uint2(pack_bf16(Pb.x, Pb.y), pack_bf16(Pb.z, Pb.w));
      }
    }
  }
}

// One thread per brick, after Adam: this iteration's losses update the plateau test
// (Sec. 5.2: L_rec not reduced by a relative `prel` for more than `pwin` iterations
// multiplies the learning rates by `pfactor`; the `pmax`-th time finishes the brick)
// and, if G was trained, the early-stop test (Sec. 4.3.2: the mean of L_den over the
// last `window` density iterations has not dropped by a relative `rel` below the mean
// of the window before); then the decisions for the next iteration are taken (G is
// trained after `delay` iterations, until early stop or `frac` of `total`).
__global__ void k_schedule(int B, BrickSched* __restrict__ s, double* __restrict__ ring,
                           const double* __restrict__ losses, SchedParams p, float b1, float b2) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  BrickSched q = s[b];
  if (!q.finished) {
    const double L = losses[4 * b + 0];
    if (q.it == 0 || L < q.best * (1.0 - (double)p.prel)) {
      q.best = L;
      q.bad = 0;
    } else {
      q.bad += 1;
    }
    if (q.bad > p.pwin) {
      q.plateaus += 1;
      q.bad = 0;
      if (q.plateaus >= p.pmax) q.finished = 1;
    }
    if (q.den_on) {
      const double x = losses[4 * b + 1];
      double* rg = ring + (int64_t)b * 2 * kMaxDensityWindow;
      const int W = p.window, i = q.den_n % (2 * W), j = (q.den_n + W) % (2 * W);
      const double old2 = q.den_n >= 2 * W ? rg[i] : 0.0;   // value of density iteration den_n - 2W
      const double old1 = q.den_n >= W ? rg[j] : 0.0;       // value of density iteration den_n - W
      q.s_cur += x - old1;
      q.s_prev += old1 - old2;
      rg[i] = x;
      q.den_n += 1;
      if (q.den_n >= 2 * W) {
        const double now = q.s_cur / W, before = q.s_prev / W;
        if (!(now < before - (double)p.rel * fabs(before))) q.den_stopped = 1;
      }
    }
  }
  q.it += 1;
  const long long next = q.it + 1;
  q.den_on = !q.finished && !q.den_stopped && next > p.delay && (double)next <= (double)p.frac * (double)p.total;
  if (q.den_on) {
    const int t = q.den_n + 1;
    q.bc1b = (float)(1.0 - pow((double)b1, t));
    q.rbc2b = (float)(1.0 / (1.0 - pow((double)b2, t)));
  }
  s[b] = q;
}

// BF16 shadow of the first n parameters (n a multiple of 4).
__global__ void k_shadow(const float* __restrict__ p, uint16_t* __restrict__ shadow, int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n / 4; q += (int64_t)gridDim.x * blockDim.x) {
    const float4 P = reinterpret_cast<const float4*>(p)[q];
    uint2 s;
    s.x = pack_bf16(P.x, P.y);
    s.y = pack_bf16(P.z, P.w);
    reinterpret_cast<uint2*>(shadow)[q] = s;
  }
}

// ------------------------------------------------------------ sampler
// Point n of brick b at sampler step s: one Philox4x32-10 block of counter (n, b, s, 0),
// its first three words as 24-bit uniforms in [-1, 1).
__device__ __forceinline__ float3 draw_point(uint32_t n, int b, unsigned long long s, uint2 key) {
  const uint4 r = philox(make_uint4(n, (uint32_t)b, (uint32_t)s, 0u), key);
  return make_float3(fmaf((float)(r.x >> 8), 0x1p-23f, -1.f), fmaf((float)(r.y >> 8), 0x1p-23f, -1.f),
                     fmaf((float)(r.z >> 8), 0x1p-23f, -1.f));
}

// Counting sort, pass 1: each point's rank within its brick's Morton bin.
__global__ void k_sample_gen(Bricks br, unsigned long long seed, unsigned long long step,
                             const unsigned long long* step_dev, uint32_t* rank, uint32_t* hist) {
  const int64_t total = br.off[br.n];
  const unsigned long long s = step_dev ? *step_dev : step;
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < total; gi += (int64_t)gridDim.x * blockDim.x) {
    const int b = brick_of_point(br, gi);
    const float3 p = draw_point((uint32_t)(gi - br.off[b]), b, s, key);
    rank[gi] = atomicAdd(hist + (int64_t)b * kSortBins + morton_bin(p.x, p.y, p.z), 1u);
  }
}

// Exclusive scan of one brick's kSortBins counters (one block of 1024 threads per brick):
// each thread scans 32 consecutive counters (vector loads), the warps scan their threads'
// totals with shuffles, and one warp scans the 32 warp totals.
__global__ void __launch_bounds__(1024) k_sample_scan(uint32_t* hist) {
  constexpr int per = kSortBins / 1024;
  static_assert(per % 4 == 0, "vector loads of the counters");
  __shared__ uint32_t wsum[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint4* h = reinterpret_cast<uint4*>(hist + (int64_t)blockIdx.x * kSortBins + threadIdx.x * per);
  uint4 v[per / 4];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < per / 4; ++k) {   // exclusive prefix within the thread
    v[k] = h[k];
    const uint32_t a = v[k].x, b = v[k].y, c = v[k].z, d = v[k].w;
    v[k] = make_uint4(s, s + a, s + a + b, s + a + b + c);
    s += a + b + c + d;
  }
  uint32_t incl = s;   // inclusive scan of the thread totals within the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = wsum[lane], wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    wsum[lane] = wi - w;   // exclusive
  }
  __syncthreads();
  const uint32_t base = wsum[warp] + incl - s;
#pragma unroll
  for (int k = 0; k < per / 4; ++k)
    h[k] = make_uint4(base + v[k].x, base + v[k].y, base + v[k].z, base + v[k].w);
}

// Pass 2 (after the scan): the point drawn again (cheaper than storing and re-reading
// it) and written at its bin's start plus its rank.
__global__ void k_sample_scatter(Bricks br, unsigned long long seed, unsigned long long step,
                                 const unsigned long long* step_dev, const uint32_t* __restrict__ rank,
                                 const uint32_t* __restrict__ hist, float* __restrict__ xyz) {
  const int64_t total = br.off[br.n];
  const unsigned long long s = step_dev ? *step_dev : step;
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < total; gi += (int64_t)gridDim.x * blockDim.x) {
    const int b = brick_of_point(br, gi);
    const float3 p = draw_point((uint32_t)(gi - br.off[b]), b, s, key);
    const int64_t dst = br.off[b] + hist[(int64_t)b * kSortBins + morton_bin(p.x, p.y, p.z)] + rank[gi];
    xyz[3 * dst] = p.x; xyz[3 * dst + 1] = p.y; xyz[3 * dst + 2] = p.z;
  }
}

// ------------------------------------------------------------ ground truth v(x)
// Element offset of voxel (x, y, z) in the tiled layout of a volume whose x and y extents
// span tx and ty tiles: tiles of kVolTile^3 voxels in x-fastest tile order, each tile's
// voxels x-fastest.  The eight corners of a trilinear lookup then lie in one 256-byte
// tile (and one DRAM page) unless the cell crosses a tile face.
__device__ __forceinline__ int64_t tiled_offset(int64_t x, int64_t y, int64_t z, int64_t tx, int64_t ty) {
  constexpr int S = kVolTile;
  const int64_t t = ((z / S) * ty + (y / S)) * tx + (x / S);
  return t * (S * S * S) + ((z % S) * S + (y % S)) * S + (x % S);
}

template <bool TILED>
__global__ void k_target(Bricks br, const float* __restrict__ vol, int64_t dx, int64_t dy, int64_t dz,
                         VolumeBoxes vb, const float* __restrict__ xyz, float* __restrict__ out) {
  const int64_t total = br.off[br.n];
  const int64_t tx = (dx + kVolTile - 1) / kVolTile, ty = (dy + kVolTile - 1) / kVolTile;
  for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < total; gi += (int64_t)gridDim.x * blockDim.x) {
    const int b = brick_of_point(br, gi);
    int c[3];
    float w[3];
    for (int d = 0; d < 3; ++d) {
      const float x = fminf(fmaxf(xyz[3 * gi + d], -1.f), 1.f);
      const int lo = vb.lo[b][d], hi = vb.hi[b][d];
      const float s = fmaf((x + 1.f) * 0.5f, (float)(hi - lo), (float)lo);
      const int ci = min(max((int)floorf(s), lo), hi - 1);
      c[d] = ci;
      w[d] = s - (float)ci;
    }
    float v[8];
    if constexpr (TILED) {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        v[k] = __ldg(vol + tiled_offset(c[0] + (k & 1), c[1] + ((k >> 1) & 1), c[2] + (k >> 2), tx, ty));
    } else {
      const int64_t base = ((int64_t)c[2] * dy + c[1]) * dx + c[0];
      const int64_t sy = dx, sz = dx * dy;
      v[0] = __ldg(vol + base); v[1] = __ldg(vol + base + 1);
      v[2] = __ldg(vol + base + sy); v[3] = __ldg(vol + base + sy + 1);
      v[4] = __ldg(vol + base + sz); v[5] = __ldg(vol + base + sz + 1);
      v[6] = __ldg(vol + base + sz + sy); v[7] = __ldg(vol + base + sz + sy + 1);
    }
    const float ax = 1.f - w[0], ay = 1.f - w[1], az = 1.f - w[2];
    out[gi] = az * (ay * (ax * v[0] + w[0] * v[1]) + w[1] * (ax * v[2] + w[0] * v[3])) +
              w[2] * (ay * (ax * v[4] + w[0] * v[5]) + w[1] * (ax * v[6] + w[0] * v[7]));
  }
  (void)dz;
}

// The tiled copy of an x-fastest volume (its padding, zeroed beforehand, stays zero).
__global__ void k_tile_volume(const float* __restrict__ vol, int64_t dx, int64_t dy, int64_t dz,
                              float* __restrict__ out) {
  const int64_t n = dx * dy * dz;
  const int64_t tx = (dx + kVolTile - 1) / kVolTile, ty = (dy + kVolTile - 1) / kVolTile;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = i % dx, y = (i / dx) % dy, z = i / (dx * dy);
    out[tiled_offset(x, y, z, tx, ty)] = vol[i];
  }
}

int blocks_for(int64_t n, int threads, int num_sms, int per_sm) {
  int64_t b = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms * per_sm;
  if (b > cap) b = cap;
  return b < 1 ? 1 : (int)b;
}

}  // namespace

cudaError_t launch_density_rho(const Launch& L, const Model& md, const Bricks& br, const TrainWs& ws,
                               const float* xyz) {
  if (br.off[br.n] == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(ws.tile_ctr + 4, 0, sizeof(int32_t), L.stream);
  if (e != cudaSuccess) return e;
  if (md.p == 10) k_density_rho<true><<<L.num_sms, RHT, 0, L.stream>>>(md, br, ws, xyz);
  else k_density_rho<false><<<L.num_sms, RHT, 0, L.stream>>>(md, br, ws, xyz);
  return cudaGetLastError();
}

cudaError_t launch_density(const Launch& L, const Model& md, const Bricks& br, const TrainWs& ws,
                           const float* xyz, float eps, int ctas_per_sm) {
  const int64_t total = br.off[br.n];
  if (total == 0) return cudaSuccess;
  int stiles = 0;
  for (int b = 0; b < br.n; ++b) stiles += (int)((br.off[b + 1] - br.off[b] + ST - 1) / ST);
  const int sgrid = stiles < 4 * L.num_sms ? stiles : 4 * L.num_sms;
  k_density_scalar<<<sgrid, ST, 0, L.stream>>>(br, ws, eps);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int tiles = 0;
  for (int b = 0; b < br.n; ++b) tiles += (int)((br.off[b + 1] - br.off[b] + DT - 1) / DT);
  const int grid = tiles < ctas_per_sm * L.num_sms ? tiles : ctas_per_sm * L.num_sms;   // 8 warps each
  if ((e = cudaMemsetAsync(ws.tile_ctr + 3, 0, sizeof(int32_t), L.stream)) != cudaSuccess) return e;
  if (md.p == 10) k_density_grad<true><<<grid, DNT, 0, L.stream>>>(md, br, ws, xyz, eps);
  else k_density_grad<false><<<grid, DNT, 0, L.stream>>>(md, br, ws, xyz, eps);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const Launch& L, const Bricks& br, const Model& md, const TrainWs& ws,
                            bool density, float* dG, int64_t sdG, double* losses) {
  k_finalize<<<br.n, kMaxGrids, 0, L.stream>>>(br, md, ws, density ? 1 : 0, dG, sdG, losses);
  return cudaGetLastError();
}

cudaError_t launch_adam(const Launch& L, const AdamLayout& lay, float* p, float* g, float* m, float* v,
                        uint16_t* shadow, bool do_b, float lr_a, float lr_b, float beta1, float beta2, float eps,
                        StepState* st, const BrickSched* sched, float pfactor, int seg0, int seg1, bool advance) {
  cudaError_t e;
  if (advance) {
    k_advance<<<1, 1, 0, L.stream>>>(st, do_b ? 1 : 0, beta1, beta2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  int64_t per_brick = 0;
  for (int k = seg0; k < seg1; ++k) per_brick += lay.size[k] / 4;
  if (per_brick == 0) return cudaSuccess;
  const int bx = (int)std::max<int64_t>(1, std::min<int64_t>((per_brick + 511) / 512,
                                                             (int64_t)8 * L.num_sms / lay.n_bricks + 1));
  k_adam<<<dim3(bx, lay.n_bricks), 256, 0, L.stream>>>(lay, p, g, m, v, shadow, do_b ? 1 : 0, lr_a, lr_b, beta1,
                                                       beta2, eps, st, sched, pfactor, seg0, seg1);
  return cudaGetLastError();
}

cudaError_t launch_schedule(const Launch& L, int n_bricks, BrickSched* s, double* ring, const double* losses,
                            const SchedParams& p, float beta1, float beta2) {
  k_schedule<<<1, 64, 0, L.stream>>>(n_bricks, s, ring, losses, p, beta1, beta2);
  return cudaGetLastError();
}

cudaError_t launch_shadow(const Launch& L, const float* p, uint16_t* shadow, int64_t n) {
  k_shadow<<<blocks_for(n / 4, 256, L.num_sms, 8), 256, 0, L.stream>>>(p, shadow, n);
  return cudaGetLastError();
}

cudaError_t launch_sample(const Launch& L, const Bricks& br, unsigned long long seed,
                          unsigned long long step, const unsigned long long* step_dev,
                          float* xyz, uint32_t* rank, uint32_t* hist) {
  const int64_t total = br.off[br.n];
  if (total == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * kSortBins * br.n, L.stream);
  if (e != cudaSuccess) return e;
  const int blocks = blocks_for(total, 256, L.num_sms, 8);
  k_sample_gen<<<blocks, 256, 0, L.stream>>>(br, seed, step, step_dev, rank, hist);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_sample_scan<<<br.n, 1024, 0, L.stream>>>(hist);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_sample_scatter<<<blocks, 256, 0, L.stream>>>(br, seed, step, step_dev, rank, hist, xyz);
  return cudaGetLastError();
}

cudaError_t launch_target(const Launch& L, const Bricks& br, const float* vol, int64_t dx,
                          int64_t dy, int64_t dz, const VolumeBoxes& vb, const float* xyz,
                          float* target, bool tiled) {
  const int64_t total = br.off[br.n];
  if (total == 0) return cudaSuccess;
  const int blocks = blocks_for(total, 256, L.num_sms, 8);
  if (tiled) k_target<true><<<blocks, 256, 0, L.stream>>>(br, vol, dx, dy, dz, vb, xyz, target);
  else k_target<false><<<blocks, 256, 0, L.stream>>>(br, vol, dx, dy, dz, vb, xyz, target);
  return cudaGetLastError();
}

int64_t tiled_volume_elems(int64_t dx, int64_t dy, int64_t dz) {
  const int64_t S = kVolTile;
  return ((dx + S - 1) / S) * ((dy + S - 1) / S) * ((dz + S - 1) / S) * S * S * S;
}

cudaError_t launch_tile_volume(const Launch& L, const float* vol, int64_t dx, int64_t dy, int64_t dz, float* out) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float) * tiled_volume_elems(dx, dy, dz), L.stream);
  if (e != cudaSuccess) return e;
  k_tile_volume<<<blocks_for(dx * dy * dz, 256, L.num_sms, 16), 256, 0, L.stream>>>(vol, dx, dy, dz, out);
  return cudaGetLastError();
}

}  // namespace srn
