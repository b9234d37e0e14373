// Building blocks of the BF16 kernels: swizzled shared-memory matrices, ldmatrix /
// mma.sync (m16n8k16, bf16 in, f32 accumulate) wrappers, and the BF16 grid reads and
// float32 gradient writes of Eq. 2 and its adjoint.
#pragma once
#include "common.cuh"

namespace srn {

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

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* g, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(g), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }

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

// Eq. 2 for grids of RC nodes per axis known at compile time: one 32-bit node index and
// eight reads at constant offsets from it.  Same arithmetic as trilinear_bf16.
template <int RC>
__device__ __forceinline__ void trilinear_bf16_r(const __nv_bfloat16* Fi, const Cell& c, int C, float& o0,
                                                 float& o1) {
  const uint32_t b = ((uint32_t)c.cz * RC + (uint32_t)c.cy) * RC + (uint32_t)c.cx;
  const float ax = 1.f - c.wx, ay = 1.f - c.wy, az = 1.f - c.wz;
  if (C == 2) {
    const unsigned int* p = reinterpret_cast<const unsigned int*>(Fi) + b;
    const float2 v0 = unpack_bf16(__ldg(p)), v1 = unpack_bf16(__ldg(p + 1));
    const float2 v2 = unpack_bf16(__ldg(p + RC)), v3 = unpack_bf16(__ldg(p + RC + 1));
    const float2 v4 = unpack_bf16(__ldg(p + RC * RC)), v5 = unpack_bf16(__ldg(p + RC * RC + 1));
    const float2 v6 = unpack_bf16(__ldg(p + RC * RC + RC)), v7 = unpack_bf16(__ldg(p + RC * RC + RC + 1));
    o0 = az * (ay * (ax * v0.x + c.wx * v1.x) + c.wy * (ax * v2.x + c.wx * v3.x)) +
         c.wz * (ay * (ax * v4.x + c.wx * v5.x) + c.wy * (ax * v6.x + c.wx * v7.x));
    o1 = az * (ay * (ax * v0.y + c.wx * v1.y) + c.wy * (ax * v2.y + c.wx * v3.y)) +
         c.wz * (ay * (ax * v4.y + c.wx * v5.y) + c.wy * (ax * v6.y + c.wx * v7.y));
  } else {
    const unsigned short* p = reinterpret_cast<const unsigned short*>(Fi) + b;
    auto ld = [&](uint32_t o) { return __uint_as_float(static_cast<uint32_t>(__ldg(p + o)) << 16); };
    const float v0 = ld(0), v1 = ld(1), v2 = ld(RC), v3 = ld(RC + 1);
    const float v4 = ld(RC * RC), v5 = ld(RC * RC + 1), v6 = ld(RC * RC + RC), v7 = ld(RC * RC + RC + 1);
    o0 = az * (ay * (ax * v0 + c.wx * v1) + c.wy * (ax * v2 + c.wx * v3)) +
         c.wz * (ay * (ax * v4 + c.wx * v5) + c.wy * (ax * v6 + c.wx * v7));
    o1 = 0.f;
  }
}

// Eq. 2, with the common resolution R = 32 on the constant-offset path.
__device__ __forceinline__ void trilinear_bf16_any(const __nv_bfloat16* Fi, const Cell& c, int R, int C, float& o0,
                                                   float& o1) {
  if (R == 32) trilinear_bf16_r<32>(Fi, c, C, o0, o1);
  else trilinear_bf16(Fi, c, R, C, o0, o1);
}

// Adjoint of Eq. 2 for one point: add g * weight into each corner of cell c of the
// float32 gradient grid (8 float2 / float atomics).
__device__ __forceinline__ void scatter_point(float* dFi, const Cell& c, int R, int C, float g0, float g1) {
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

}  // namespace srn
