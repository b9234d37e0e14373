// Renderer launch parameters and workspace (internal to libsrn).
#pragma once
#include "common.cuh"
#include "kernels.h"

namespace srn {

struct RenderParams {
  srn_camera cam;
  int32_t width, height, samples;
  int32_t order;    // 0: raster order; 1: the progressive (image-hierarchy) order
  int32_t levels;   // L: the coarsest hierarchy level, 2^L >= max(width, height)
  // Sample slots of a batch: groups of rg consecutive rays x blocks of jb consecutive
  // samples (render_slot), so that 128 consecutive slots (rg = 8, jb = 16) are a compact
  // bundle of ray segments: the forward query's tiles then read few cache lines per grid.
  int32_t rg, jb;
  int32_t grid[3];
  int64_t vox;
  float vmin, vmax;
  int32_t lo[SRN_MAX_BRICKS][3];
  int32_t hi[SRN_MAX_BRICKS][3];
};

// Slot of sample j of ray `ray` in a batch, and the number of slots of npix rays (padded
// to whole ray groups and sample blocks; padding slots hold no sample).
__host__ __device__ inline int64_t render_slot(int rg, int jb, int samples, int ray, int j) {
  const int nsb = (samples + jb - 1) / jb;
  return (((int64_t)(ray / rg) * nsb + j / jb) * rg + ray % rg) * jb + j % jb;
}
__host__ __device__ inline int64_t render_slots(int rg, int jb, int samples, int npix) {
  return (int64_t)((npix + rg - 1) / rg) * rg * ((samples + jb - 1) / jb) * jb;
}

struct RenderWs {
  float* loc;       // [max_points][3] brick-local sample coordinates, ray order
  uint32_t* rank;   // [max_points] rank inside the brick bucket
  uint32_t* bid;    // [max_points] brick of the sample (all ones: ray missed)
  uint32_t* pos;    // [max_points] bucketed position of each sample
  float* xyz;       // [max_points][3] bucketed coordinates
  float* val;       // [max_points] queried values, bucketed order
  uint32_t* cnt;    // [B] bucket sizes
  int64_t* off;     // [B + 1] bucket offsets
};

cudaError_t launch_render_batch(const Launch& L, const RenderParams& rp, const RenderWs& w, int pix0,
                                int npix, const Model& md, const float* lut, float* rgba);
// In-progress image after `done` pixels of the progressive order; `level` is the finest
// complete hierarchy level (ignored when done = 0).
cudaError_t launch_render_preview(const Launch& L, const RenderParams& rp, int done, int level,
                                  const float* rgba, float* preview);

// One batch of the full-volume decode: the voxels [x0, x0+nx) x [y0, y0+ny) x [z0, z0+nz)
// (all in brick `brick`, x fastest) queried in that brick's local coordinates.
struct DecodeChunk {
  int64_t vox;
  int32_t brick, n_bricks;
  int32_t x0, nx, y0, ny, z0, nz;
  int32_t lo[3], hi[3];   // the brick's voxel box (its local [-1, 1] corners)
};
cudaError_t launch_decode_chunk(const Launch& L, const DecodeChunk& c, const RenderWs& w, const Model& md,
                                float* out);

}  // namespace srn
