// The per-(point, grid) step of Eq. 1-2 of the BF16 training pass's encoder (k_enc): a
// grid's node box over a tile of points is staged in shared memory as the float32
// values of its BF16 nodes (C per entry: one 8-byte f32x2 pair for C = 2), node by node
// with one column per lane, so the eight corner reads of a warp (32 lanes = 32 grids,
// one point) fall in distinct banks, and each corner arrives as a ready f32x2 operand.
// A point whose cell is not inside its grid's box takes the corners from global memory.
#pragma once
#include <type_traits>

#include "bf16_ops.cuh"

namespace srn {

constexpr float kMagic = 12582912.f;        // 1.5 * 2^23: for |x| < 2^22, x + kMagic holds round(x)
constexpr int32_t kMagicBits = 0x4B400000;  // in its low bits, offset by these bits of kMagic

// Eq. 2's cell and weight along one axis of a grid with R even, without a float-to-int
// conversion: the addend ct = (R-1)/2 - 1/2 + kMagic is then an integer, so one FMA
// gives t = kMagic + round(s - 1/2) for the exact s = (u+1)(R-1)/2: the cell floor(s)
// off the nodes, and on a node either neighbouring cell (weight 1 or 0 there, the same
// value; on the upper face R-2, the even neighbour).  The cell comes back as its
// float's bits (cell + kMagicBits); the weight is s - cell with s rounded as make_cell
// rounds it, which lies in [cell, cell + 1], so the weight is exact and in [0, 1].
__device__ __forceinline__ int32_t axis_cell(float u, float hs, float ct, float& w) {
  const float t = fmaf(u, hs, ct);
  w = fmaf(u, hs, hs) - (t - kMagic);
  return __float_as_int(t);
}

template <int C>
using EncNode = std::conditional_t<C == 2, uint32_t, uint16_t>;   // one node in global memory: C bf16 values
template <int C>
using EncSNode = std::conditional_t<C == 2, unsigned long long, float>;   // one staged node: C float32

// Packed float pairs (two channels at once).
__device__ __forceinline__ unsigned long long f2_bits(float lo, float hi) {
  return (unsigned long long)__float_as_uint(lo) | ((unsigned long long)__float_as_uint(hi) << 32);
}
__device__ __forceinline__ unsigned long long bf2_bits(uint32_t v) {   // bf16x2 -> f32x2
  return f2_bits(__uint_as_float(v << 16), __uint_as_float(v & 0xffff0000u));
}
// a + w (b - a) on both halves
__device__ __forceinline__ unsigned long long lerp2(unsigned long long a, unsigned long long b,
                                                    unsigned long long w) {
  unsigned long long d, r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(b), "l"(a));
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(w), "l"(d), "l"(a));
  return r;
}

__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// axis_cell for two axes at once, u = (ua, ub) as a packed pair, hs2 = (hs, hs),
// ct2 = (ct, ct), m2 = (kMagic, kMagic): the same roundings as two axis_cell calls.
__device__ __forceinline__ void axis_cell2(unsigned long long u, unsigned long long hs2, unsigned long long ct2,
                                           unsigned long long m2, int32_t& ta, int32_t& tb, float& wa, float& wb) {
  const unsigned long long t = fma2(u, hs2, ct2), s = fma2(u, hs2, hs2);
  unsigned long long tm, w;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(tm) : "l"(t), "l"(m2));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(w) : "l"(s), "l"(tm));
  ta = (int32_t)(uint32_t)t;
  tb = (int32_t)(uint32_t)(t >> 32);
  wa = __uint_as_float((uint32_t)w);
  wb = __uint_as_float((uint32_t)(w >> 32));
}

// One staged node (C float32 values) at shared address a + OFF.
template <int C, int OFF>
__device__ __forceinline__ EncSNode<C> enc_node(uint32_t a) {
  EncSNode<C> v;
  if constexpr (C == 2) asm volatile("ld.shared.b64 %0, [%1+%2];" : "=l"(v) : "r"(a), "n"(OFF));
  else asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(a), "n"(OFF));
  return v;
}
// Eq. 2 from the grid in global memory (a point outside its tile's box), packed as Y.
template <int C>
__device__ __noinline__ uint32_t enc_global(const __nv_bfloat16* Fi, Cell c, int R) {
  float f0 = 0.f, f1 = 0.f;
  trilinear_bf16_any(Fi, c, R, C, f0, f1);
  return C == 2 ? pack_bf16(f0, f1) : (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(f0));
}

// One grid's staged node box as a lane sees it: lo / nodes per axis (bytes of a box
// word pair: lo[3] | n[3]), the byte address of this lane's column, and the node
// strides of y and z in bytes.
struct EncBox {
  int lox, loy, loz, nxb, nyb, nzb;
  bool boxed;                  // the box is staged (non-empty, and fits)
  uint32_t col_s, oy, oz;
  int32_t mlox, mloy, mloz;    // kMagicBits + lo (cells of axis_cell relative to the box)
};
template <int C>
__device__ __forceinline__ EncBox enc_box(uint2 bx, int capn, uint32_t col_s) {
  constexpr uint32_t kRow = 32 * sizeof(EncSNode<C>);   // bytes of one node row
  EncBox e;
  e.nxb = (int)(bx.y & 0xffu); e.nyb = (int)((bx.y >> 8) & 0xffu); e.nzb = (int)((bx.y >> 16) & 0xffu);
  e.lox = (int)(bx.x & 0xffu); e.loy = (int)((bx.x >> 8) & 0xffu); e.loz = (int)((bx.x >> 16) & 0xffu);
  const int nodes = e.nxb * e.nyb * e.nzb;
  e.boxed = nodes > 0 && nodes <= capn;
  e.col_s = col_s;
  e.oy = (uint32_t)e.nxb * kRow;
  e.oz = (uint32_t)(e.nxb * e.nyb) * kRow;
  e.mlox = kMagicBits + e.lox; e.mloy = kMagicBits + e.loy; e.mloz = kMagicBits + e.loz;
  return e;
}

// Stages one grid's node box (nodes of the box in x-fastest order) into this lane's
// column as float32: the threads of a grid group take nodes n0, n0 + nstep, ..., four
// loads in flight.  Fg is the grid's BF16 nodes [R][R][R] (C per node).
template <int C>
__device__ __forceinline__ void enc_stage(const EncBox& e, const EncNode<C>* __restrict__ Fg, int R,
                                          EncSNode<C>* col, int n0, int nstep) {
  using E = EncNode<C>;
  const int nodes = e.nxb * e.nyb * e.nzb;
  int qz = n0 / (e.nxb * e.nyb), qr = n0 - qz * e.nxb * e.nyb;
  int qy = qr / e.nxb, qx = qr - qy * e.nxb;
  for (int n = n0; n < nodes; n += 4 * nstep) {
    E v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      v[u] = 0;
      if (n + u * nstep < nodes) v[u] = __ldg(Fg + ((e.loz + qz) * R + (e.loy + qy)) * R + e.lox + qx);   // < R^3
      qx += nstep;
      while (qx >= e.nxb) {
        qx -= e.nxb;
        if (++qy == e.nyb) { qy = 0; ++qz; }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (n + u * nstep < nodes) {
        if constexpr (C == 2) col[(n + u * nstep) * 32] = bf2_bits(v[u]);
        else col[(n + u * nstep) * 32] = __uint_as_float((uint32_t)v[u] << 16);
      }
    }
  }
}

// Eq. 1-2 for one (point, grid): the C features of the grid at point (x, y, z), packed as
// C bf16 (0 outside the grid: Eq. 2's inclusive mask), from the staged box when the
// point's cell lies in it, else from global memory.  gi is the grid's transform, hs =
// (R-1)/2, ct = hs - 1/2 + kMagic (used when R is even), Fi the grid's BF16 nodes.
template <int C, bool EVEN_R>
__device__ __forceinline__ uint32_t encode_point(const float (&gi)[12], float x, float y, float z, const EncBox& e,
                                                 float hs, float ct, int R, const __nv_bfloat16* Fi) {
  constexpr uint32_t kRow = 32 * sizeof(EncSNode<C>);
  float ux, uy, uz;
  affine(gi, x, y, z, ux, uy, uz);
  uint32_t yv = 0u;
  // Eq. 2's mask.  With R even a cell in the box already means the point is inside the
  // grid (the box's cells lie in [0, R-2], and beyond a face axis_cell gives -1 or R-1
  // on that axis), so the mask is tested only for the points that miss the box.
  const bool inside_now = EVEN_R || ((fabsf(ux) <= 1.f) & (fabsf(uy) <= 1.f) & (fabsf(uz) <= 1.f));
  if (inside_now) {
    // Eq. 2's set-up: inside the grid s lies in [0, R-1] (the rounding of fmaf is
    // monotone).  R even: axis_cell.  R odd: the cell floor(s), which differs from
    // min(floor(s), R-2) only at s = R-1, whose cell R-1 is never in a box and takes
    // the exact path below
    float wx, wy, wz;
    unsigned lx, ly, lz;   // cell relative to the box
    if constexpr (EVEN_R) {
      int32_t tx, ty;   // x and y as one packed pair
      axis_cell2(f2_bits(ux, uy), f2_bits(hs, hs), f2_bits(ct, ct), f2_bits(kMagic, kMagic), tx, ty, wx, wy);
      lx = (unsigned)(tx - e.mlox);
      ly = (unsigned)(ty - e.mloy);
      lz = (unsigned)(axis_cell(uz, hs, ct, wz) - e.mloz);
    } else {
      const float sx = fmaf(ux, hs, hs), sy = fmaf(uy, hs, hs), sz = fmaf(uz, hs, hs);
      const int cx = (int)sx, cy = (int)sy, cz = (int)sz;
      wx = sx - (float)cx; wy = sy - (float)cy; wz = sz - (float)cz;
      lx = (unsigned)(cx - e.lox); ly = (unsigned)(cy - e.loy); lz = (unsigned)(cz - e.loz);
    }
    if (e.boxed && lx < (unsigned)(e.nxb - 1) && ly < (unsigned)(e.nyb - 1) && lz < (unsigned)(e.nzb - 1)) {
      const uint32_t a0 = e.col_s + ((lz * (unsigned)e.nyb + ly) * (unsigned)e.nxb + lx) * kRow;
      const uint32_t a1 = a0 + e.oy, a2 = a0 + e.oz, a3 = a2 + e.oy;
      if constexpr (C == 2) {
        const unsigned long long px = f2_bits(wx, wx), py = f2_bits(wy, wy), pz = f2_bits(wz, wz);
        const unsigned long long e0 = lerp2(enc_node<C, 0>(a0), enc_node<C, kRow>(a0), px);
        const unsigned long long e1 = lerp2(enc_node<C, 0>(a1), enc_node<C, kRow>(a1), px);
        const unsigned long long e2 = lerp2(enc_node<C, 0>(a2), enc_node<C, kRow>(a2), px);
        const unsigned long long e3 = lerp2(enc_node<C, 0>(a3), enc_node<C, kRow>(a3), px);
        const unsigned long long f = lerp2(lerp2(e0, e1, py), lerp2(e2, e3, py), pz);
        yv = pack_bf16(__uint_as_float((uint32_t)f), __uint_as_float((uint32_t)(f >> 32)));
      } else {
        const float v0 = enc_node<C, 0>(a0), v1 = enc_node<C, kRow>(a0);
        const float v2 = enc_node<C, 0>(a1), v3 = enc_node<C, kRow>(a1);
        const float v4 = enc_node<C, 0>(a2), v5 = enc_node<C, kRow>(a2);
        const float v6 = enc_node<C, 0>(a3), v7 = enc_node<C, kRow>(a3);
        const float e0 = fmaf(wx, v1 - v0, v0), e1 = fmaf(wx, v3 - v2, v2);
        const float e2 = fmaf(wx, v5 - v4, v4), e3 = fmaf(wx, v7 - v6, v6);
        const float f01 = fmaf(wy, e1 - e0, e0), f23 = fmaf(wy, e3 - e2, e2);
        yv = __bfloat16_as_ushort(__float2bfloat16_rn(fmaf(wz, f23 - f01, f01)));
      }
    } else if (!EVEN_R || ((fabsf(ux) <= 1.f) & (fabsf(uy) <= 1.f) & (fabsf(uz) <= 1.f))) {
      yv = enc_global<C>(Fi, make_cell(ux, uy, uz, R), R);   // outside the box: corners from global memory
    }
  }
  return yv;
}

// Node box (lo | nodes per axis, as bytes) of grid g over the axis-aligned block
// [lo, hi] of brick-local space: the block's image under Eq. 1, padded by 1e-3 in s
// against the rounding of the per-point map, clipped to the grid.  n = 0 (no nodes):
// no point of the block is inside the grid.
__device__ __forceinline__ uint2 block_box(const float (&lo)[3], const float (&hi)[3], const float* __restrict__ g,
                                           int R) {
  const float h = 0.5f * (float)(R - 1);
  uint32_t blo = 0, bn = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float umin = g[4 * d + 3], umax = umin;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float a = g[4 * d + k];
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

}  // namespace srn
