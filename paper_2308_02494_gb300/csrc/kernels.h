// Host-side launch wrappers of the libsrn kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace srn {

enum QueryMode { kForward = 0, kTrain = 1, kTrainDensity = 2 };

struct Launch {
  cudaStream_t stream;
  int num_sms;
};

// BF16 path: fused forward query, and the three-kernel training pass (encoder,
// decoder forward/backward, scatter), batched over bricks.
cudaError_t launch_forward_bf16(const Launch& L, const Model& md, const Bricks& br, const float* xyz,
                                float* out);
// Optional pair of CUDA events recorded around one kernel of the BF16 training pass
// (which: 0 encoder, 1 decoder, 2 scatter); the measurement hook passes it.
struct KernelMark {
  int which;
  cudaEvent_t start, stop;
};
// A second stream for the density loss beside the main chain: with `dens` its first
// pass (rho, which needs only the points and the transforms) is forked after the encoder
// and runs beside the decoder; the other two (which need the decoder's h) wait for the
// decoder and run beside the scatter; the pass joins before it returns.
struct SideStream {
  cudaStream_t stream;
  cudaEvent_t fork, join, enc_done;
  bool defer_join;   // the caller waits for `join` itself (later work can run beside the tail)
};
// Launch shape of the BF16 training pass, set per handle (srn_set_tuning, srn_autotune).
// A tile is a run of Morton-consecutive points of one brick inside one aligned Morton
// block of at most 2^tile_level units, holding at most tile_points points; the block's
// node box in every grid is what the encoder stages and the scatter accumulates.
constexpr int kMinTilePoints = 128;
constexpr int kMaxTilePoints = 1024;   // the encoder's and the scatter's point staging
constexpr int kMaxTileLevel = 9;
constexpr int kMaxDensityCtas = 4;     // eight warps of 64 registers each fill an SM at 4
struct Tuning {
  int tile_points;    // kMinTilePoints .. kMaxTilePoints, a multiple of 32
  int tile_level;     // 0 .. kMaxTileLevel (each brick further capped by its node boxes)
  int density_ctas;   // CTAs per SM of the density-gradient pass beside the scatter
};
constexpr Tuning kDefaultTuning{kMaxTilePoints, kMaxTileLevel, 2};
cudaError_t launch_train_bf16(const Launch& L, bool dens, const Model& md, const Grads& gr, const Bricks& br,
                              const TrainWs& ws, const float* xyz, const float* target, const Tuning& tn,
                              const KernelMark* mark = nullptr, const SideStream* side = nullptr);
// The decoder kernel of the BF16 training pass on the tcgen05 tensor cores (K = 128).
cudaError_t launch_mlp_tc(const Launch& L, const Model& md, const Grads& gr, const Bricks& br, const TrainWs& ws,
                          const float* target);
// FP32 path: one fused kernel per mode (encoder + SIMT decoder + per-corner scatter).
cudaError_t launch_query_fp32(const Launch& L, QueryMode mode, const Model& md, const Grads& gr,
                              const Bricks& br, const TrainWs& ws, const float* xyz,
                              const float* target, float* out);

// Density loss (Eq. 7-9) second and third passes, and the per-brick finalisation.
cudaError_t launch_density(const Launch& L, const Model& md, const Bricks& br, const TrainWs& ws,
                           const float* xyz, float eps, int ctas_per_sm = 4);
// The first pass alone (rho per point and its sum per brick), one CTA per SM.
cudaError_t launch_density_rho(const Launch& L, const Model& md, const Bricks& br, const TrainWs& ws,
                               const float* xyz);
// Shared memory a CTA of the third density pass needs on its SM (static + reserved).
constexpr int kDensityCtaSmem = 16 * 1024;
cudaError_t launch_finalize(const Launch& L, const Bricks& br, const Model& md, const TrainWs& ws,
                            bool density, float* dG, int64_t sdG, double* losses);

// Adam over the flat parameter buffer; the step state lives in device memory.
struct StepState {
  unsigned long long step;   // sampler step (advanced once per srn_step)
  int t_a, t_b;              // Adam step counts of group A (F, decoder) and B (G)
  float bc1a, rbc2a;         // 1 - beta1^t_a and 1 / (1 - beta2^t_a)
  float bc1b, rbc2b;         // the same for t_b
  double p1a, p2a, p1b, p2b; // beta1^t_a, beta2^t_a, beta1^t_b, beta2^t_b (running products)
};
// The training routine of Sec. 4.3.2 (delayed start and early stop of the transform
// updates) and the plateau scheduler of Sec. 5.2, kept per brick on the device.
constexpr int kMaxDensityWindow = 4096;
struct BrickSched {
  long long it;               // iterations this brick has trained
  int plateaus, bad;          // plateau reductions so far; iterations without improvement
  int finished;               // no further updates (the last plateau fired)
  int den_on;                 // G is updated at the next iteration
  int den_stopped;            // early stop (or the iteration cutoff) has fired
  int den_n;                  // density iterations so far
  double best;                // lowest L_rec of the plateau test
  double s_cur, s_prev;       // sums of L_den over the last and the previous window
  float bc1b, rbc2b;          // Adam bias corrections of G for the next density iteration
};
struct SchedParams {
  int delay, window;
  float rel, frac;
  long long total;
  int pwin;
  float prel, pfactor;
  int pmax;
};
cudaError_t launch_schedule(const Launch& L, int n_bricks, BrickSched* s, double* ring, const double* losses,
                            const SchedParams& p, float beta1, float beta2);

// Adam, one grid row of CTAs per brick over the brick's five parameter segments
// (F, W1, W2, w3, G).  With `sched`, a brick's learning rates take its plateau scale,
// a finished brick is skipped, and G follows the brick's density decision.
struct AdamLayout {
  int64_t off[5], size[5];    // segment offsets and per-brick strides (floats)
  int n_bricks;
};
// Segments [seg0, seg1) of (F, W1, W2, w3, G); `advance` first advances the step state
// (once per step, before the first segments).
cudaError_t launch_adam(const Launch& L, const AdamLayout& lay, float* p, float* g, float* m, float* v,
                        uint16_t* shadow, bool do_b, float lr_a, float lr_b, float beta1, float beta2, float eps,
                        StepState* st, const BrickSched* sched, float pfactor, int seg0 = 0, int seg1 = 5,
                        bool advance = true);
cudaError_t launch_shadow(const Launch& L, const float* p, uint16_t* shadow, int64_t n);

// Sampler (Philox + Morton counting sort) and ground-truth lookup.  The scanned
// histogram the sampler leaves in `hist` holds each brick's bin starts.
cudaError_t launch_sample(const Launch& L, const Bricks& br, unsigned long long seed,
                          unsigned long long step, const unsigned long long* step_dev,
                          float* xyz, uint32_t* rank, uint32_t* hist);
struct VolumeBoxes {
  int32_t lo[SRN_MAX_BRICKS][3];
  int32_t hi[SRN_MAX_BRICKS][3];
};
// v(x) by trilinear lookup; `tiled`: vol is in the layout launch_tile_volume writes.
cudaError_t launch_target(const Launch& L, const Bricks& br, const float* vol, int64_t dx,
                          int64_t dy, int64_t dz, const VolumeBoxes& vb, const float* xyz,
                          float* target, bool tiled);
// The tiled layout of a dx x dy x dz volume: tiles of kVolTile^3 voxels (x-fastest tile
// order, x-fastest inside a tile), each extent padded to whole tiles.
constexpr int kVolTile = 4;
int64_t tiled_volume_elems(int64_t dx, int64_t dy, int64_t dz);
cudaError_t launch_tile_volume(const Launch& L, const float* vol, int64_t dx, int64_t dy, int64_t dz, float* out);

// Sets the calling thread's srn_last_error() message and returns s.
srn_status report(srn_status s, const char* message);

}  // namespace srn
