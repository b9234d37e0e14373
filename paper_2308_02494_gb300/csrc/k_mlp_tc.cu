// Decoder forward and backward of the BF16 training pass for K = M*C = 128 features on
// the fifth-generation tensor cores (Sec. 4.1.2's MLP 128 -> 64 -> 64 -> 1 without
// biases, L_rec of Sec. 4.3.1, and its gradient):
//
//   Z1 = Y W1^T      H1 = ReLU(Z1)      Z2 = H1 W2^T      H2 = ReLU(Z2)
//   f  = (H2 . w3)(max - min) + min     dm = dL/df (max - min)
//   dZ2 = dm w3 [Z2 > 0]   dH1 = dZ2 W2   dZ1 = dH1 [H1 > 0]   dY = dZ1 W1
//   dW1 += dZ1^T Y   dW2 += dZ2^T H1   dw3 += dm^T H2
//
// A CTA of 128 threads takes 128-point tiles.  One thread issues tcgen05.mma with
// BF16 operands in 128-byte-swizzled shared memory and FP32 accumulators in tensor
// memory (256 columns per CTA: Z1 / dH1 / dY in columns 0..127, Z2 in 64..127, and
// the brick's dW1^T and dW2^T accumulated across tiles in 128..255); thread r of the
// CTA owns tile row r in every epilogue (tcgen05.ld of its tensor-memory lane),
// applies ReLU / the loss / the masks and writes the next operand back to shared
// memory as BF16.  Y tiles arrive by TMA tensor loads counted on an mbarrier (the
// tensor map's 128-byte swizzle is the operand layout), and dL/dy leaves by TMA tensor
// stores from a swizzled stage, which is also read for the largest |dL/dy| of every
// grid over the tile (the scatter's fixed-point scales).  The accumulated weight
// gradients go to global memory with one atomic per entry when the CTA moves to
// another brick or finishes.  Every wait on the tensor cores and on the tensor loads is
// bounded; on giving up the CTA sets bit 1 of the status word, stops, and frees its
// tensor memory.
#include <climits>
#include <cuda.h>
#include <cudaTypedefs.h>

#include "bf16_ops.cuh"
#include "kernels.h"
#include "tc_ops.cuh"

namespace srn {
namespace {

constexpr int TT = 128;    // points per tile (the MMA's M)
constexpr int TK = 128;    // features (K = M*C)
constexpr int TNT = 128;   // threads
constexpr uint32_t kPolls = 1u << 22;

// Shared memory (offsets from a 1024-byte aligned base; operand blocks 1024-aligned).
struct TcLay {
  static constexpr uint32_t Y = 0;           // [128 pts][128 feats] bf16
  static constexpr uint32_t W1 = 32768;      // [64][128]
  static constexpr uint32_t W2 = 49152;      // [64][64]
  static constexpr uint32_t H1 = 57344;      // [128][64] ReLU(Z1)
  static constexpr uint32_t DZ2 = 73728;     // [128][64] dL/dZ2
  static constexpr uint32_t DZ1 = 90112;     // [128][64] dL/dZ1
  static constexpr uint32_t W3 = 106496;     // [64] f32
  static constexpr uint32_t DW3 = W3 + 256;  // [64] f32 reduction scratch
  static constexpr uint32_t BYTES = DW3 + 256;
};
// Staging of dL/dy for the tensor store: the tile [128][128] bf16 in the operand layout
// (two 1024-aligned blocks of 64 columns, the tensor map's 128-byte swizzle), over H1
// and DZ2, both free by then.  Row-wise writes and chunk-wise reads are conflict-free.
constexpr uint32_t kDyStage = TcLay::H1;
static_assert(kDyStage % 1024 == 0 && TcLay::DZ2 == kDyStage + 16384, "dL/dy staging must be H1 then DZ2");
// Tensor-memory columns.
constexpr uint32_t kColZ1 = 0, kColZ2 = 64, kColDY = 0, kColDW1 = 128, kColDW2 = 192, kCols = 256;

constexpr uint32_t kIdZ = tc::idesc_bf16(128, 64, false, false);    // Z1, Z2
constexpr uint32_t kIdDH = tc::idesc_bf16(128, 64, false, true);    // dH1 (W2 read transposed)
constexpr uint32_t kIdDY = tc::idesc_bf16(128, 128, false, true);   // dY (W1 read transposed)
constexpr uint32_t kIdW = tc::idesc_bf16(128, 64, true, true);      // dW1^T, dW2^T

__device__ __forceinline__ float bits(uint32_t u) { return __uint_as_float(u); }
// bf16 pair {ReLU(lo), ReLU(hi)} (round to nearest even), one instruction.
__device__ __forceinline__ uint32_t relu_pack(uint32_t lo, uint32_t hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(bits(hi)), "f"(bits(lo)));
  return d;
}
// For a pair of non-negative bf16 values (ReLU outputs), 0xffff in each half that is
// nonzero: adding 0x7fff to a half sets its bit 15 exactly when the half is nonzero
// (never carrying into the other half), and the permute replicates bits 15 and 31
// over their halves.
__device__ __forceinline__ uint32_t nonzero_halves(uint32_t h) {
  uint32_t m;
  asm("prmt.b32 %0, %1, 0, 0xBB99;" : "=r"(m) : "r"(h + 0x7fff7fffu));
  return m;
}

// At most 200 registers: two CTAs (2 x 128 x 200) and one CTA of the density pass
// beside them (256 x 56) fill the register file exactly.
// tmY / tmDY: ws.Y and ws.dY as [points][128] bf16 tensors, boxes of 64 x 128 with the
// 128-byte swizzle.
__global__ void __maxnreg__(200)
k_mlp_tc(Model md, Grads gr, Bricks brp, TrainWs ws, const float* __restrict__ target,
         const __grid_constant__ CUtensorMap tmY, const __grid_constant__ CUtensorMap tmDY) {
  extern __shared__ unsigned char raw[];
  __shared__ TileMap tm;
  __shared__ Bricks br;
  __shared__ uint32_t tslot;
  __shared__ uint32_t s_gmax[TK];   // largest |dL/dy| bits per grid of the tile being written
  __shared__ __align__(8) unsigned long long mbar_s, mbar_y_s;
  load_bricks(brp, br);
  const uint32_t base0 = su32(raw), base = (base0 + 1023u) & ~1023u;
  unsigned char* sm = raw + (base - base0);
  const uint32_t sY = base + TcLay::Y, sW1 = base + TcLay::W1, sW2 = base + TcLay::W2;
  const uint32_t sH1 = base + TcLay::H1, sDZ2 = base + TcLay::DZ2, sDZ1 = base + TcLay::DZ1;
  float* w3s = reinterpret_cast<float*>(sm + TcLay::W3);
  float* dw3s = reinterpret_cast<float*>(sm + TcLay::DW3);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t mbar = su32(&mbar_s), mbar_y = su32(&mbar_y_s);
  if (tid == 0) {
    build_tile_map(br, TT, tm);
    tc::mbar_init(mbar, 1);
    tc::mbar_init(mbar_y, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc::tmem_alloc(su32(&tslot), kCols);
  if (tid < TK) s_gmax[tid] = 0u;
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);   // this warp's 32 lanes
  const int total = tm.first[br.n];
  const int per = (total + gridDim.x - 1) / gridDim.x;
  const int tb = blockIdx.x * per, te = min(total, tb + per);
  const int r = tid;   // the tile row this thread owns in the epilogues

  uint32_t phase = 0, phase_y = 0;
  bool gave_up = false, y_pending = false;
  auto wait_mma = [&]() {
    if (tc::mbar_wait(mbar, phase, kPolls)) phase ^= 1u;
    else gave_up = true;   // the phase stays: the final wait below retries it
    tc::fence_after_sync();
  };

  f2_t dw3p[32];   // dw3 partial sums of this thread's rows, as float pairs
#pragma unroll
  for (int j = 0; j < 32; ++j) dw3p[j] = 0ull;
  double sum_r2 = 0.0;

  // Weight gradients of brick b: tensor memory (dW1^T, dW2^T) and registers (dw3) to
  // global memory.  Every MMA of the brick has completed (each tile waits for its last).
  auto flush = [&](int b) {
    tc::fence_after_sync();
    float* gW1 = gr.dW1 + (int64_t)b * gr.sW1;   // [64][128]
    float* gW2 = gr.dW2 + (int64_t)b * gr.sW2;   // [64][64]
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 16) {
      uint32_t d[16];
      tc::ld16(trow + kColDW1 + c0, d);
      tc::ld_wait();
#pragma unroll
      for (int j = 0; j < 16; ++j) atomicAdd(gW1 + (c0 + j) * TK + r, bits(d[j]));
    }
    if (warp < 2) {   // dW2^T lives in lanes 0..63
#pragma unroll
      for (int c0 = 0; c0 < 64; c0 += 16) {
        uint32_t d[16];
        tc::ld16(trow + kColDW2 + c0, d);
        tc::ld_wait();
#pragma unroll
        for (int j = 0; j < 16; ++j) atomicAdd(gW2 + (c0 + j) * 64 + r, bits(d[j]));
      }
    }
    if (tid < 64) dw3s[tid] = 0.f;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 64; ++j) {
      float v = (j & 1) ? f2_hi(dw3p[j >> 1]) : f2_lo(dw3p[j >> 1]);
      v += __shfl_xor_sync(0xffffffffu, v, 16);
      v += __shfl_xor_sync(0xffffffffu, v, 8);
      v += __shfl_xor_sync(0xffffffffu, v, 4);
      v += __shfl_xor_sync(0xffffffffu, v, 2);
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      if (lane == 0) atomicAdd(dw3s + j, v);
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) dw3p[j] = 0ull;
    __syncthreads();
    if (tid < 64) atomicAdd(gr.dw3 + (int64_t)b * gr.sw3 + tid, dw3s[tid]);
    double s = sum_r2;
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) atomicAdd(ws.acc + b * kAccPerBrick + ACC_SUM_R2, s);
    sum_r2 = 0.0;
    tc::fence_before_sync();
    __syncthreads();
  };

  // The features of tile t+1 are requested (two tensor loads, 32 KB counted on mbar_y)
  // as soon as the last MMA of tile t has read Y, so the copy overlaps tile t's dL/dy
  // epilogue; its targets likewise.  Rows past the batch read as zero; rows past a
  // brick's last point hold the next brick's features, which add nothing (their dL/dm
  // is zero).
  int hint = -1;
  int64_t nxt_p0 = 0;
  int nxt_np = 0, nxt_b = 0;
  float nxt_v = 0.f;
  auto prefetch = [&](int tile) {
    nxt_b = brick_of_tile(tm, br.n, tile, hint);
    hint = nxt_b;
    nxt_p0 = br.off[nxt_b] + (int64_t)(tile - tm.first[nxt_b]) * TT;
    nxt_np = (int)min((int64_t)TT, br.off[nxt_b + 1] - nxt_p0);
    if (tid == 0) {
      tc::mbar_expect_tx(mbar_y, TT * TK * 2);
      tc::tma_load_2d(sY, &tmY, mbar_y, 0, (int)nxt_p0);
      tc::tma_load_2d(sY + TT * 128, &tmY, mbar_y, 64, (int)nxt_p0);
    }
    y_pending = true;
    nxt_v = r < nxt_np ? target[nxt_p0 + r] : 0.f;
  };
  if (tb < te) prefetch(tb);

  int cur = -1;
  bool fresh = true;   // first tile of a brick: the dW accumulators start over
  float span = 0.f, vmin = 0.f, inv_n = 0.f;
  for (int tile = tb; tile < te; ++tile) {
    const int b = nxt_b;
    const int64_t p0 = nxt_p0;
    const int np = nxt_np;
    const float vr = nxt_v;
    if (b != cur) {
      if (cur >= 0) flush(cur);
      cur = b;
      const uint4* w1 = reinterpret_cast<const uint4*>(md.W1h + (int64_t)b * md.sW1);
      for (int q = tid; q < 64 * TK / 8; q += TNT)
        *reinterpret_cast<uint4*>(sm + TcLay::W1 + tc::sw128_off(q >> 4, (q & 15) * 8, 64)) = w1[q];
      const uint4* w2 = reinterpret_cast<const uint4*>(md.W2h + (int64_t)b * md.sW2);
      for (int q = tid; q < 64 * 64 / 8; q += TNT)
        *reinterpret_cast<uint4*>(sm + TcLay::W2 + tc::sw128_off(q >> 3, (q & 7) * 8, 64)) = w2[q];
      if (tid < 64) w3s[tid] = md.w3[(int64_t)b * md.sw3 + tid];
      vmin = md.range[2 * b];
      span = md.range[2 * b + 1] - vmin;
      inv_n = 1.f / (float)(br.off[b + 1] - br.off[b]);
      fresh = true;
    }
    // ---- the tile's features (requested one tile ahead); the previous tile's dL/dy
    //      store has read its staging (H1 and DZ2, rewritten below)
    const bool rv = r < np;
    if (tc::mbar_wait(mbar_y, phase_y, kPolls)) {
      phase_y ^= 1u;
      y_pending = false;
    } else {
      gave_up = true;
    }
    if (tid == 0) tc::bulk_wait_read();
    tc::fence_async_smem();   // a brick's weights, written above, are read by the MMAs
    tc::fence_before_sync();
    __syncthreads();

    // ---- Z1 = Y W1^T
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < TK / 16; ++kk)
        tc::mma(tmem + kColZ1, tc::desc_kmajor(sY, kk, TT), tc::desc_kmajor(sW1, kk, 64), kIdZ, kk > 0);
      tc::commit(mbar);
    }
    wait_mma();
    // ---- H1 = ReLU(Z1) -> shared memory
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 32) {   // two tensor-memory loads per wait
      uint32_t z[32], h[16];
      tc::ld16(trow + kColZ1 + c0, *reinterpret_cast<uint32_t(*)[16]>(z));
      tc::ld16(trow + kColZ1 + c0 + 16, *reinterpret_cast<uint32_t(*)[16]>(z + 16));
      tc::ld_wait();
#pragma unroll
      for (int j = 0; j < 16; ++j) h[j] = relu_pack(z[2 * j], z[2 * j + 1]);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4*>(sm + TcLay::H1 + tc::sw128_off(r, c0 + 8 * q, TT)) =
            make_uint4(h[4 * q], h[4 * q + 1], h[4 * q + 2], h[4 * q + 3]);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();

    // ---- Z2 = H1 W2^T
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        tc::mma(tmem + kColZ2, tc::desc_kmajor(sH1, kk, TT), tc::desc_kmajor(sW2, kk, 64), kIdZ, kk > 0);
      tc::commit(mbar);
    }
    wait_mma();
    // ---- f, the loss, dm; dZ2 -> shared memory; dw3.  Z2 is read from tensor memory
    //      once; the dot with w3, dw3 and dm w3 run on packed float pairs.
    f2_t h2[32];
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 32) {   // two tensor-memory loads per wait
      uint32_t z[32];
      tc::ld16(trow + kColZ2 + c0, *reinterpret_cast<uint32_t(*)[16]>(z));
      tc::ld16(trow + kColZ2 + c0 + 16, *reinterpret_cast<uint32_t(*)[16]>(z + 16));
      tc::ld_wait();
#pragma unroll
      for (int j = 0; j < 16; ++j) h2[c0 / 2 + j] = f2_pack(fmaxf(bits(z[2 * j]), 0.f), fmaxf(bits(z[2 * j + 1]), 0.f));
    }
    const f2_t* w3p = reinterpret_cast<const f2_t*>(w3s);
    f2_t macc = 0ull;
#pragma unroll
    for (int j = 0; j < 32; ++j) macc = f2_fma(h2[j], w3p[j], macc);
    const float m = f2_lo(macc) + f2_hi(macc);
    float dm;
    if (ws.upstream) {   // caller-supplied dL/df: dL/dm = dL/df (max - min)
      dm = rv ? vr * span : 0.f;
    } else {             // L_rec: dL/dm = 2 (f - v) (max - min) / N
      const float e = rv ? fmaf(m, span, vmin) - vr : 0.f;
      if (rv) ws.herr[p0 + r] = e * e;
      sum_r2 += (double)e * e;
      dm = 2.f * e * span * inv_n;
    }
    const f2_t dm2 = f2_pack(dm, dm);
#pragma unroll
    for (int j = 0; j < 32; ++j) dw3p[j] = f2_fma(dm2, h2[j], dw3p[j]);
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 16) {
      uint32_t d[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {   // ReLU outputs are never negative: > 0 iff nonzero
        const f2_t q = f2_mul(dm2, w3p[c0 / 2 + j]);
        const f2_t hh = h2[c0 / 2 + j];
        d[j] = pack_bf16(f2_lo(hh) != 0.f ? f2_lo(q) : 0.f, f2_hi(hh) != 0.f ? f2_hi(q) : 0.f);
      }
      *reinterpret_cast<uint4*>(sm + TcLay::DZ2 + tc::sw128_off(r, c0, TT)) = make_uint4(d[0], d[1], d[2], d[3]);
      *reinterpret_cast<uint4*>(sm + TcLay::DZ2 + tc::sw128_off(r, c0 + 8, TT)) = make_uint4(d[4], d[5], d[6], d[7]);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();

    // ---- dH1 = dZ2 W2 and dW2^T += H1^T dZ2 (rows 64..127 of that MMA read the dZ2
    //      block as a second A atom and are discarded)
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        tc::mma(tmem + kColZ1, tc::desc_kmajor(sDZ2, kk, TT), tc::desc_mnmajor(sW2, kk, 64), kIdDH, kk > 0);
#pragma unroll
      for (int kk = 0; kk < TT / 16; ++kk)
        tc::mma(tmem + kColDW2, tc::sdesc(sH1 + (uint32_t)kk * 2048u, TcLay::DZ2 - TcLay::H1, 1024u),
                tc::desc_mnmajor(sDZ2, kk, TT), kIdW, !(fresh && kk == 0));
      tc::commit(mbar);
    }
    wait_mma();
    // ---- dZ1 = dH1 [H1 > 0] -> shared memory
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 16) {
      uint32_t z[16], d[8];
      tc::ld16(trow + kColZ1 + c0, z);
      tc::ld_wait();
      const uint4 ha = *reinterpret_cast<const uint4*>(sm + TcLay::H1 + tc::sw128_off(r, c0, TT));
      const uint4 hb = *reinterpret_cast<const uint4*>(sm + TcLay::H1 + tc::sw128_off(r, c0 + 8, TT));
      const uint32_t hw[8] = {ha.x, ha.y, ha.z, ha.w, hb.x, hb.y, hb.z, hb.w};
#pragma unroll
      for (int j = 0; j < 8; ++j)   // ReLU outputs are never negative: > 0 iff nonzero
        d[j] = pack_bf16(bits(z[2 * j]), bits(z[2 * j + 1])) & nonzero_halves(hw[j]);
      *reinterpret_cast<uint4*>(sm + TcLay::DZ1 + tc::sw128_off(r, c0, TT)) = make_uint4(d[0], d[1], d[2], d[3]);
      *reinterpret_cast<uint4*>(sm + TcLay::DZ1 + tc::sw128_off(r, c0 + 8, TT)) = make_uint4(d[4], d[5], d[6], d[7]);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();

    // ---- dY = dZ1 W1 and dW1^T += Y^T dZ1
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        tc::mma(tmem + kColDY, tc::desc_kmajor(sDZ1, kk, TT), tc::desc_mnmajor(sW1, kk, 64), kIdDY, kk > 0);
#pragma unroll
      for (int kk = 0; kk < TT / 16; ++kk)
        tc::mma(tmem + kColDW1, tc::desc_mnmajor(sY, kk, TT), tc::desc_mnmajor(sDZ1, kk, TT), kIdW,
                !(fresh && kk == 0));
      tc::commit(mbar);
    }
    wait_mma();
    if (tile + 1 < te && !gave_up) prefetch(tile + 1);   // Y has been read by every MMA of this tile
    // ---- dL/dy to global memory, point-major bf16: row p0 + r holds the K features'
    //      gradients in feature order (grid-major, channel-minor, as Y).  Staged in the
    //      (now free) H1 / DZ2 buffers in the tensor map's swizzled layout, then written
    //      by two tensor stores (thread 0) when the tile is full; a brick's last, partial
    //      tile is copied out row by row, so that nothing lands on the next brick's rows.
#pragma unroll 1
    for (int c0 = 0; c0 < TK; c0 += 32) {
      uint32_t za[16], zb[16], d[16];
      tc::ld16(trow + kColDY + c0, za);
      tc::ld16(trow + kColDY + c0 + 16, zb);
      tc::ld_wait();
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        d[i] = pack_bf16(bits(za[2 * i]), bits(za[2 * i + 1]));
        d[8 + i] = pack_bf16(bits(zb[2 * i]), bits(zb[2 * i + 1]));
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4*>(sm + kDyStage + tc::sw128_off(r, c0 + 8 * q, TT)) =
            make_uint4(d[4 * q], d[4 * q + 1], d[4 * q + 2], d[4 * q + 3]);
    }
    tc::fence_async_smem();
    __syncthreads();
    const bool full = np == TT;
    auto store_tile = [&]() {   // the full tile's two tensor stores, after the reads below
      if (full && tid == 0) {
        tc::tma_store_2d(&tmDY, base + kDyStage, 0, (int)p0);
        tc::tma_store_2d(&tmDY, base + kDyStage + TT * 128, 64, (int)p0);
        tc::bulk_commit();
      }
    };
    if (!full || ws.gmax_blk) {
      // thread t always reads chunk t mod 16, so it also takes the largest |dL/dy| of
      // that chunk's features over the tile (for the scatter's fixed-point scales),
      // reduced over the threads of the same chunk
      uint32_t mx[4] = {0u, 0u, 0u, 0u};
      auto take = [&](const uint4& v) {
        mx[0] = __vmaxu2(mx[0], v.x & 0x7fff7fffu);
        mx[1] = __vmaxu2(mx[1], v.y & 0x7fff7fffu);
        mx[2] = __vmaxu2(mx[2], v.z & 0x7fff7fffu);
        mx[3] = __vmaxu2(mx[3], v.w & 0x7fff7fffu);
      };
      if (full) {   // all 16 reads in flight at once (the tensor cores share these banks)
        uint4 v[TT * TK / 8 / TNT];
#pragma unroll
        for (int i = 0; i < TT * TK / 8 / TNT; ++i) {
          const int q = tid + i * TNT;
          v[i] = *reinterpret_cast<const uint4*>(sm + kDyStage + tc::sw128_off(q >> 4, 8 * (q & 15), TT));
        }
#pragma unroll
        for (int i = 0; i < TT * TK / 8 / TNT; ++i) take(v[i]);
      } else {
        for (int q = tid; q < np * (TK / 8); q += TNT) {
          const int row = q >> 4, k = q & 15;
          const uint4 v = *reinterpret_cast<const uint4*>(sm + kDyStage + tc::sw128_off(row, 8 * k, TT));
          *reinterpret_cast<uint4*>(ws.dY + (p0 + row) * TK + 8 * k) = v;
          take(v);
        }
      }
      store_tile();
      if (ws.gmax_blk) {
#pragma unroll
        for (int j = 0; j < 4; ++j) mx[j] = __vmaxu2(mx[j], __shfl_xor_sync(0xffffffffu, mx[j], 16));
        if (lane < 16) {
          const int k = tid & 15;   // features 8k .. 8k + 7
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (md.C == 2) {
              atomicMax(s_gmax + 4 * k + j, max(mx[j] & 0xffffu, mx[j] >> 16));
            } else {
              atomicMax(s_gmax + 8 * k + 2 * j, mx[j] & 0xffffu);
              atomicMax(s_gmax + 8 * k + 2 * j + 1, mx[j] >> 16);
            }
          }
        }
        __syncthreads();
        if (tid < md.M) {
          ws.gmax_blk[(int64_t)tile * md.M + tid] = (uint16_t)s_gmax[tid];
          s_gmax[tid] = 0u;
        }
      }
    } else {
      store_tile();
    }
    fresh = false;
    tc::fence_before_sync();
    if (__syncthreads_or(gave_up)) {
      gave_up = true;
      break;
    }
  }
  if (gave_up) {   // let MMAs still in flight finish (bounded) before freeing tensor memory
    tc::mbar_wait(mbar, phase, kPolls);
    if (tid == 0) atomicOr(ws.status, 2);
  } else if (cur >= 0) {
    flush(cur);
  }
  if (y_pending) tc::mbar_wait(mbar_y, phase_y, kPolls);   // a feature copy requested ahead (bounded)
  if (tid == 0) tc::bulk_wait();                            // the last dL/dy stores are written
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kCols);
}

}  // namespace

namespace {
// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda).
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}
// [rows][128] bf16 at base (rows 256 bytes apart) as a tensor of boxes 64 x 128 with the
// 128-byte swizzle of the operand layout; reads outside the rows return zeros.
cudaError_t feature_map(CUtensorMap* m, const void* base, int64_t rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_tiled();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {(cuuint64_t)TK, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)TK * 2};
  const cuuint32_t box[2] = {64, (cuuint32_t)TT};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}
}  // namespace

// The decoder pass of the BF16 training step when K = 128 (2 CTAs per SM).
cudaError_t launch_mlp_tc(const Launch& L, const Model& md, const Grads& gr, const Bricks& br, const TrainWs& ws,
                          const float* target) {
  if (md.K != TK) return cudaErrorInvalidValue;
  int tiles = 0;
  for (int b = 0; b < br.n; ++b) tiles += (int)((br.off[b + 1] - br.off[b] + TT - 1) / TT);
  if (tiles == 0) return cudaSuccess;
  const int64_t rows = br.off[br.n];
  if (rows > INT32_MAX) return cudaErrorInvalidValue;   // tensor coordinates are 32-bit
  CUtensorMap tmY, tmDY;
  cudaError_t e;
  if ((e = feature_map(&tmY, ws.Y, rows)) != cudaSuccess) return e;
  if ((e = feature_map(&tmDY, ws.dY, rows)) != cudaSuccess) return e;
  const int smem = (int)TcLay::BYTES + 1024;
  if ((e = cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
  const int grid = std::min(tiles, 2 * L.num_sms);
  k_mlp_tc<<<grid, TNT, smem, L.stream>>>(md, gr, br, ws, target, tmY, tmDY);
  return cudaGetLastError();
}

}  // namespace srn
