// Headless neural volume renderer (Sec. 6) over a domain decomposition (Sec. 5.3).
//
// Per batch of rays: (1) every (ray, sample) computes its position, its brick
// through the spatial hash and its brick-local coordinate, and takes a rank in
// its brick's bucket; (2) bucket offsets; (3) samples are scattered into brick
// order; (4) the fused forward query runs over the buckets (device-side offsets);
// (5) each ray gathers its values back in sample order and composites front to
// back.  Sampling and opacity: midpoints t_j = t0 + (j + 1/2) dt of the ray's
// segment inside [-1,1]^3, alpha = 1 - exp(-a dt / (2/512)), the 256-entry RGBA
// transfer function read with linear interpolation.
#include "common.cuh"
#include "kernels.h"
#include "render.h"

namespace srn {
namespace {

struct Ray {
  float ox, oy, oz, dx, dy, dz, t0, dt;
  bool hit;
};

__device__ __forceinline__ Ray make_ray(const RenderParams& rp, int pix) {
  const int px = pix % rp.width, py = pix / rp.width;
  const float aspect = (float)rp.width / (float)rp.height;
  const float nx = (2.f * ((float)px + 0.5f) / (float)rp.width - 1.f) * rp.cam.scale * aspect;
  const float ny = (1.f - 2.f * ((float)py + 0.5f) / (float)rp.height) * rp.cam.scale;
  Ray r;
  const float* e = rp.cam.eye;
  const float* f = rp.cam.forward;
  const float* ri = rp.cam.right;
  const float* u = rp.cam.up;
  if (rp.cam.ortho) {
    r.ox = e[0] + nx * ri[0] + ny * u[0];
    r.oy = e[1] + nx * ri[1] + ny * u[1];
    r.oz = e[2] + nx * ri[2] + ny * u[2];
    r.dx = f[0]; r.dy = f[1]; r.dz = f[2];
  } else {
    r.ox = e[0]; r.oy = e[1]; r.oz = e[2];
    float dx = f[0] + nx * ri[0] + ny * u[0];
    float dy = f[1] + nx * ri[1] + ny * u[1];
    float dz = f[2] + nx * ri[2] + ny * u[2];
    const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
    r.dx = dx * inv; r.dy = dy * inv; r.dz = dz * inv;
  }
  // slab test against [-1, 1]^3
  float tmin = -INFINITY, tmax = INFINITY;
  const float o[3] = {r.ox, r.oy, r.oz}, d[3] = {r.dx, r.dy, r.dz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float inv = 1.f / d[a];
    const float ta = (-1.f - o[a]) * inv, tb = (1.f - o[a]) * inv;
    tmin = fmaxf(tmin, fminf(ta, tb));
    tmax = fminf(tmax, fmaxf(ta, tb));
  }
  tmin = fmaxf(tmin, 0.f);
  r.hit = tmax > tmin;
  r.t0 = tmin;
  r.dt = r.hit ? (tmax - tmin) / (float)rp.samples : 0.f;
  return r;
}

// Pixels of level l of the image hierarchy: its grid (a 2^l, b 2^l), ceil(W / 2^l) by
// ceil(H / 2^l).  Together, the levels coarser than l hold exactly level l+1's grid.
__device__ __forceinline__ int level_cols(const RenderParams& rp, int l) { return (rp.width + (1 << l) - 1) >> l; }
__device__ __forceinline__ int level_pixels(const RenderParams& rp, int l) {
  return level_cols(rp, l) * ((rp.height + (1 << l) - 1) >> l);
}

// Flat pixel of the k-th pixel of the render order.  Progressive order (Sec. 6): the
// coarsest level's pixel (0, 0), then each finer level l's pixels not on level l+1's
// grid, row by row: an even row b of the level has its odd columns, an odd row all.
__device__ __forceinline__ int pixel_of(const RenderParams& rp, int k) {
  if (!rp.order || k == 0) return k;
  int l = rp.levels - 1;
  while (level_pixels(rp, l) <= k) --l;   // level_pixels(0) = W H > k
  const int q = k - level_pixels(rp, l + 1);
  const int wa = level_cols(rp, l), half = wa >> 1, pair = q / (half + wa), r = q - pair * (half + wa);
  const int a = r < half ? 2 * r + 1 : r - half, b = r < half ? 2 * pair : 2 * pair + 1;
  return (b << l) * rp.width + (a << l);
}

// Position of pixel (x, y) in the progressive order (the inverse of pixel_of).
__device__ __forceinline__ int order_of(const RenderParams& rp, int x, int y) {
  if ((x | y) == 0) return 0;
  const int l = __ffs(x | y) - 1;   // the finest level holding the pixel; < L since x, y < 2^L
  const int a = x >> l, b = y >> l, wa = level_cols(rp, l), half = wa >> 1;
  return level_pixels(rp, l + 1) + (b >> 1) * (half + wa) + ((b & 1) ? half + a : a >> 1);
}

// Samples of a block take their rank in their brick's bucket in three levels: lanes of
// a warp with the same brick (match), one shared-memory count per warp group, one global
// reservation per brick per block.  A block's samples stay together in each bucket.
__global__ void __launch_bounds__(256) k_render_gen(RenderParams rp, int pix0, int npix, float* __restrict__ loc,
                                                    uint32_t* __restrict__ rank, uint32_t* __restrict__ bid,
                                                    uint32_t* __restrict__ cnt) {
  __shared__ uint32_t s_cnt[SRN_MAX_BRICKS], s_base[SRN_MAX_BRICKS];
  const int nb = rp.grid[0] * rp.grid[1] * rp.grid[2];
  const int64_t total = render_slots(rp.rg, rp.jb, rp.samples, npix);
  const int nsb = (rp.samples + rp.jb - 1) / rp.jb;
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < total; base += (int64_t)gridDim.x * blockDim.x) {
    for (int k = threadIdx.x; k < nb; k += blockDim.x) s_cnt[k] = 0;
    __syncthreads();
    const int64_t idx = base + threadIdx.x;
    uint32_t b = 0xffffffffu;
    // the slot's ray and sample (the inverse of render_slot)
    const int js = (int)(idx % rp.jb);
    const int64_t q1 = idx / rp.jb;
    const int rl = (int)(q1 % rp.rg);
    const int64_t q2 = q1 / rp.rg;
    const int ray = (int)(q2 / nsb) * rp.rg + rl, j = (int)(q2 % nsb) * rp.jb + js;
    if (idx < total && ray < npix && j < rp.samples) {
      const Ray r = make_ray(rp, pixel_of(rp, pix0 + ray));
      if (r.hit) {
        const float t = r.t0 + ((float)j + 0.5f) * r.dt;
        const float p[3] = {r.ox + t * r.dx, r.oy + t * r.dy, r.oz + t * r.dz};
        int cell[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {   // Sec. 5.3 hash, clamped to the brick grid
          const int n = rp.grid[a];
          cell[a] = min(max((int)floorf((float)n * (p[a] + 1.f) * 0.5f), 0), n - 1);
        }
        b = (uint32_t)(cell[0] + rp.grid[0] * (cell[1] + rp.grid[1] * cell[2]));
        const float half = 0.5f * (float)(rp.vox - 1);
#pragma unroll
        for (int a = 0; a < 3; ++a) {   // global -> brick-local [-1, 1]
          const float sc = (p[a] + 1.f) * half;
          const float lo = (float)rp.lo[b][a], hi = (float)rp.hi[b][a];
          loc[3 * idx + a] = (sc - lo) / (hi - lo) * 2.f - 1.f;
        }
      }
    }
    const unsigned grp = __match_any_sync(0xffffffffu, b);
    const int leader = __ffs(grp) - 1;
    const uint32_t before = __popc(grp & ((1u << lane) - 1u));
    uint32_t wbase = 0;
    if (b != 0xffffffffu && lane == leader) wbase = atomicAdd(s_cnt + b, (uint32_t)__popc(grp));
    wbase = __shfl_sync(0xffffffffu, wbase, leader);
    __syncthreads();
    for (int k = threadIdx.x; k < nb; k += blockDim.x) s_base[k] = s_cnt[k] ? atomicAdd(cnt + k, s_cnt[k]) : 0u;
    __syncthreads();
    if (idx < total) {
      bid[idx] = b;
      if (b != 0xffffffffu) rank[idx] = s_base[b] + wbase + before;
    }
    __syncthreads();
  }
}

__global__ void k_render_offsets(int nb, const uint32_t* __restrict__ cnt, int64_t* __restrict__ off) {
  if (threadIdx.x == 0) {
    int64_t a = 0;
    for (int b = 0; b < nb; ++b) { off[b] = a; a += cnt[b]; }
    off[nb] = a;
  }
}

__global__ void k_render_scatter(int64_t total, const float* __restrict__ loc, const uint32_t* __restrict__ rank,
                                 const uint32_t* __restrict__ bid, const int64_t* __restrict__ off,
                                 float* __restrict__ xyz, uint32_t* __restrict__ pos) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t b = bid[idx];
    if (b == 0xffffffffu) continue;
    const int64_t dst = off[b] + rank[idx];
    xyz[3 * dst] = loc[3 * idx];
    xyz[3 * dst + 1] = loc[3 * idx + 1];
    xyz[3 * dst + 2] = loc[3 * idx + 2];
    pos[idx] = (uint32_t)dst;
  }
}

// Decode: brick-local coordinates of a voxel block in scanline order.
__global__ void k_decode_gen(DecodeChunk c, float* __restrict__ xyz) {
  const int64_t n = (int64_t)c.nx * c.ny * c.nz;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(idx % c.nx);
    const int64_t r = idx / c.nx;
    const int y = (int)(r % c.ny), z = (int)(r / c.ny);
    const int v[3] = {c.x0 + x, c.y0 + y, c.z0 + z};
#pragma unroll
    for (int a = 0; a < 3; ++a)   // voxel index = (p + 1)/2 (vox - 1): global -> brick-local [-1, 1]
      xyz[3 * idx + a] = ((float)v[a] - (float)c.lo[a]) / (float)(c.hi[a] - c.lo[a]) * 2.f - 1.f;
  }
}

// Decode: the block's values (scanline order) into the volume [vox][vox][vox].
__global__ void k_decode_store(DecodeChunk c, const float* __restrict__ val, float* __restrict__ out) {
  const int64_t n = (int64_t)c.nx * c.ny * c.nz;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(idx % c.nx);
    const int64_t r = idx / c.nx;
    const int y = (int)(r % c.ny), z = (int)(r / c.ny);
    out[((int64_t)(c.z0 + z) * c.vox + (c.y0 + y)) * c.vox + c.x0 + x] = val[idx];
  }
}

// One thread per ray: gather the ray's values in sample order and composite.
__global__ void k_render_composite(RenderParams rp, int pix0, int npix, const uint32_t* __restrict__ pos,
                                   const float* __restrict__ val, const float* __restrict__ lut,
                                   float* __restrict__ rgba) {
  const int ray = blockIdx.x * blockDim.x + threadIdx.x;
  if (ray >= npix) return;
  const int pix = pixel_of(rp, pix0 + ray);
  const Ray r = make_ray(rp, pix);
  float cr = 0.f, cg = 0.f, cb = 0.f, T = 1.f;
  if (r.hit) {
    const float k = r.dt / (2.f / 512.f);
    const float inv_span = 1.f / (rp.vmax - rp.vmin);
    for (int j = 0; j < rp.samples; ++j) {
      const float f = val[pos[render_slot(rp.rg, rp.jb, rp.samples, ray, j)]];
      const float s = fminf(fmaxf((f - rp.vmin) * inv_span, 0.f), 1.f) * 255.f;
      const int i0 = min((int)s, 254);
      const float fr = s - (float)i0;
      const float4 a = reinterpret_cast<const float4*>(lut)[i0];
      const float4 c = reinterpret_cast<const float4*>(lut)[i0 + 1];
      const float red = a.x + (c.x - a.x) * fr, grn = a.y + (c.y - a.y) * fr, blu = a.z + (c.z - a.z) * fr;
      const float op = a.w + (c.w - a.w) * fr;
      const float alpha = 1.f - expf(-op * k);
      const float w = T * alpha;
      cr = fmaf(w, red, cr); cg = fmaf(w, grn, cg); cb = fmaf(w, blu, cb);
      T *= 1.f - alpha;
    }
  }
  reinterpret_cast<float4*>(rgba)[pix] = make_float4(cr, cg, cb, 1.f - T);
}

// In-progress image of progressive rendering: evaluated pixels as they are, the others
// bilinear between the four samples of the finest complete level around (x, y) / 2^l.
__global__ void k_render_preview(RenderParams rp, int done, int level, const float4* __restrict__ rgba,
                                 float4* __restrict__ out) {
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= rp.width * rp.height) return;
  const int x = pix % rp.width, y = pix / rp.width;
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (order_of(rp, x, y) < done) {
    v = rgba[pix];
  } else if (done > 0) {
    const int nx = level_cols(rp, level), ny = (rp.height + (1 << level) - 1) >> level;
    const float s = 1.f / (float)(1 << level);
    const float fx = (float)x * s, fy = (float)y * s;   // exact: a power-of-two scale
    const int a0 = min(x >> level, nx - 1), b0 = min(y >> level, ny - 1);
    const int a1 = min(a0 + 1, nx - 1), b1 = min(b0 + 1, ny - 1);
    const float tx = a1 == a0 ? 0.f : fx - (float)a0, ty = b1 == b0 ? 0.f : fy - (float)b0;
    const float4 p00 = rgba[(b0 << level) * rp.width + (a0 << level)];
    const float4 p10 = rgba[(b0 << level) * rp.width + (a1 << level)];
    const float4 p01 = rgba[(b1 << level) * rp.width + (a0 << level)];
    const float4 p11 = rgba[(b1 << level) * rp.width + (a1 << level)];
    const float ux = 1.f - tx, uy = 1.f - ty;
    v.x = uy * (ux * p00.x + tx * p10.x) + ty * (ux * p01.x + tx * p11.x);
    v.y = uy * (ux * p00.y + tx * p10.y) + ty * (ux * p01.y + tx * p11.y);
    v.z = uy * (ux * p00.z + tx * p10.z) + ty * (ux * p01.z + tx * p11.z);
    v.w = uy * (ux * p00.w + tx * p10.w) + ty * (ux * p01.w + tx * p11.w);
  }
  out[pix] = v;
}

int blocks_for(int64_t n, int threads, int num_sms) {
  int64_t b = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms * 8;
  if (b > cap) b = cap;
  return b < 1 ? 1 : (int)b;
}

}  // namespace

cudaError_t launch_render_batch(const Launch& L, const RenderParams& rp, const RenderWs& w, int pix0,
                                int npix, const Model& md, const float* lut, float* rgba) {
  const int64_t total = render_slots(rp.rg, rp.jb, rp.samples, npix);
  const int nb = rp.grid[0] * rp.grid[1] * rp.grid[2];
  cudaError_t e = cudaMemsetAsync(w.cnt, 0, sizeof(uint32_t) * nb, L.stream);
  if (e != cudaSuccess) return e;
  k_render_gen<<<blocks_for(total, 256, L.num_sms), 256, 0, L.stream>>>(rp, pix0, npix, w.loc, w.rank, w.bid, w.cnt);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_render_offsets<<<1, 32, 0, L.stream>>>(nb, w.cnt, w.off);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_render_scatter<<<blocks_for(total, 256, L.num_sms), 256, 0, L.stream>>>(total, w.loc, w.rank, w.bid, w.off, w.xyz, w.pos);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  Bricks br{};
  br.n = nb;
  br.dev = w.off;
  Grads gr{};
  TrainWs tw{};
  e = md.F16 ? launch_forward_bf16(L, md, br, w.xyz, w.val)
             : launch_query_fp32(L, kForward, md, gr, br, tw, w.xyz, nullptr, w.val);
  if (e != cudaSuccess) return e;
  k_render_composite<<<(npix + 127) / 128, 128, 0, L.stream>>>(rp, pix0, npix, w.pos, w.val, lut, rgba);
  return cudaGetLastError();
}

cudaError_t launch_render_preview(const Launch& L, const RenderParams& rp, int done, int level,
                                  const float* rgba, float* preview) {
  const int n = rp.width * rp.height;
  k_render_preview<<<(n + 255) / 256, 256, 0, L.stream>>>(rp, done, level, reinterpret_cast<const float4*>(rgba),
                                                         reinterpret_cast<float4*>(preview));
  return cudaGetLastError();
}

cudaError_t launch_decode_chunk(const Launch& L, const DecodeChunk& c, const RenderWs& w, const Model& md,
                                float* out) {
  const int64_t n = (int64_t)c.nx * c.ny * c.nz;
  if (n == 0) return cudaSuccess;
  k_decode_gen<<<blocks_for(n, 256, L.num_sms), 256, 0, L.stream>>>(c, w.xyz);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  Bricks br{};
  br.n = c.n_bricks;
  br.dev = nullptr;
  for (int b = 0; b <= c.n_bricks; ++b) br.off[b] = b <= c.brick ? 0 : n;
  Grads gr{};
  TrainWs tw{};
  e = md.F16 ? launch_forward_bf16(L, md, br, w.xyz, w.val)
             : launch_query_fp32(L, kForward, md, gr, br, tw, w.xyz, nullptr, w.val);
  if (e != cudaSuccess) return e;
  k_decode_store<<<blocks_for(n, 256, L.num_sms), 256, 0, L.stream>>>(c, w.val, out);
  return cudaGetLastError();
}

}  // namespace srn
