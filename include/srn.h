/*
 * srn.h -- C ABI of libsrn, the GB300 (sm_103a) implementation of the APMGSRN
 * point query (Wurster et al., "Adaptively Placed Multi-Grid Scene Representation
 * Networks for Large-Scale Data Visualization"), its training step and its renderer.
 *
 * Conventions shared by every entry point
 *   - All pointers named *_dev point to device memory; all others to host memory.
 *   - The caller owns every buffer (parameters, gradients, Adam moments, BF16
 *     shadow, workspace, inputs, outputs).  The handle keeps non-owning pointers.
 *   - Calls taking a `stream` (a cudaStream_t passed as void*) are asynchronous on
 *     that stream; NULL means the legacy default stream.  They return SRN_OK once
 *     the work is enqueued.  Arguments are validated before anything is launched;
 *     a bad argument returns SRN_ERR_INVALID_ARG (or SRN_ERR_UNSUPPORTED for a
 *     legal but unimplemented shape) with nothing enqueued.  A launch failure
 *     returns SRN_ERR_CUDA.  srn_last_error() gives a message for the calling thread.
 *   - Nothing throws across the ABI.  No entry point allocates device memory.
 *   - Layouts (all row-major, C order):
 *       points   xyz[N][3] float32, points of brick b contiguous in
 *                [offsets[b], offsets[b+1]); coordinates in the brick's local
 *                domain [-1, 1]^3 (Sec. 4.1: a model maps [-1,1]^3 to a scalar).
 *       features F[B][M][R][R][R][C]: grid i, node (z, y, x), channel c; the
 *                local coordinate u_x runs along the fastest node axis.
 *       transforms G[B][M][3][4]: first three rows of the 4x4 matrix of Eq. 1.
 *       decoder  W1[B][H][K], W2[B][H][H], w3[B][H] (K = M*C, H = 64), no biases.
 */
#ifndef SRN_H
#define SRN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SRN_MAX_BRICKS 64

typedef struct srn_handle srn_handle;

typedef enum {
  SRN_OK = 0,
  SRN_ERR_INVALID_ARG = 1,     /* null pointer, bad size, inconsistent offsets */
  SRN_ERR_UNSUPPORTED = 2,     /* legal shape this build does not implement */
  SRN_ERR_CUDA = 3,            /* a CUDA call or launch failed */
  SRN_ERR_DEVICE_TIMEOUT = 4,  /* a bounded device-side wait gave up (reported by srn_get_status) */
  SRN_ERR_NONFINITE = 5,       /* a loss came out NaN/Inf (reported by srn_get_status) */
  SRN_ERR_STATE = 6            /* call out of order (e.g. step before any backward) */
} srn_status;

typedef enum { SRN_FP32 = 0, SRN_BF16 = 1 } srn_precision;

/* Flags of srn_backward / srn_step / srn_train_step. */
#define SRN_DENSITY 1u   /* step (2) of Sec. 4.3.2: L_den (Eq. 9) and its gradient into G */
#define SRN_UPSTREAM 2u  /* srn_backward only: target_dev holds dL/df per point (any upstream
                            loss) instead of v(x); no L_rec is formed; excludes SRN_DENSITY */
#define SRN_SCHEDULE 4u  /* srn_train_step only: the training routine set by srn_set_schedule
                            decides, per brick on the device, whether G is trained and the
                            learning-rate scale; SRN_DENSITY is then ignored */
#define SRN_VOLUME_TILED 16u /* srn_train_step only: volume_dev is the tiled copy written by
                                srn_tile_volume (same dims), read by the ground-truth lookup */
#define SRN_REC_DG 8u    /* srn_backward only: also the gradient of L_rec (or, with SRN_UPSTREAM,
                            of the upstream loss) with respect to G through Eq. 1-2, added into
                            G's gradient.  Sec. 4.3.2 trains G with L_den alone, so training
                            never sets it: it is the rest of the full gradient of f, for
                            diagnostics and for autograd through the transforms */

/* Model and optimiser configuration (Sec. 4.1, 4.2, 6).  Supported in this build:
 * hidden = 64; channels in {1, 2}; K = n_grids*channels in {16, 32, 64, 128};
 * 2 <= res <= 64; 1 <= flat_top_p <= 16; 1 <= n_bricks <= SRN_MAX_BRICKS. */
typedef struct {
  int32_t n_bricks;      /* B: independent models trained and queried together (Sec. 5) */
  int32_t n_grids;       /* M feature grids per model (Sec. 4.1.1) */
  int32_t channels;      /* C features per grid node */
  int32_t res;           /* R: every grid is R x R x R nodes */
  int32_t hidden;        /* H neurons in each of the two hidden layers (Sec. 4.1.2) */
  int32_t precision;     /* srn_precision: FP32 everywhere, or BF16 grids/decoder */
  int32_t flat_top_p;    /* p of Eq. 7; the exponent is 2p (the paper uses p = 10) */
  float density_eps;     /* epsilon of Eq. 8 (also used inside Eq. 9's log) */
  float lr_feat;         /* Adam learning rate of F and the decoder (0.01, Sec. 6) */
  float lr_xform;        /* Adam learning rate of G (0.001, Sec. 6) */
  float beta1, beta2;    /* Adam betas (0.9, 0.99, Sec. 6) */
  float adam_eps;        /* Adam epsilon (not given in the paper; 1e-8 by default) */
} srn_config;

/* Element offsets into the flat float32 parameter buffer.  The gradient and the two
 * Adam moment buffers use the same layout.  [0, n_group_a) holds every F and
 * decoder tensor (learning rate lr_feat; the BF16 shadow mirrors this range);
 * [n_group_a, n_params) holds every G (learning rate lr_xform).  Brick b's copy of
 * tensor X starts at off_X + b * size_X.  Every offset is a multiple of 64. */
typedef struct {
  int64_t n_params, n_group_a;
  int64_t off_F, off_W1, off_W2, off_w3, off_G;
  int64_t size_F, size_W1, size_W2, size_w3, size_G;
} srn_layout;

/* Caller-owned device tensors (see srn_layout). */
typedef struct {
  float* params_dev;       /* [n_params] float32 master weights */
  float* grads_dev;        /* [n_params] written by srn_backward */
  float* adam_m_dev;       /* [n_params] first moments, zero-initialised by the caller */
  float* adam_v_dev;       /* [n_params] second moments, zero-initialised by the caller */
  uint16_t* shadow_dev;    /* [n_group_a] bfloat16 copy read by the BF16 kernels; NULL for FP32 */
  const float* range_dev;  /* [B][2] saved (min, max) of each brick's data (Sec. 4.1.2 "Scaling") */
} srn_tensors;

/* Pinhole or orthographic camera (Sec. 6): eye position and an orthonormal basis.
 * scale = tan(fov/2) (perspective) or half the view height (orthographic). */
typedef struct {
  float eye[3], forward[3], right[3], up[3];
  float scale;
  int32_t ortho;
} srn_camera;

/* Fill *out with the parameter layout of cfg.  Host only. */
srn_status srn_param_layout(const srn_config* cfg, srn_layout* out);

/* Bytes of device workspace srn_create needs for batches of up to max_points
 * points (all bricks together) and renders of up to max_points samples per pass. */
srn_status srn_workspace_size(const srn_config* cfg, int64_t max_points, size_t* bytes);

/* Create a handle over caller-owned tensors and a workspace of at least
 * srn_workspace_size(cfg, max_points) bytes (256-byte aligned).  Zeroes the device
 * step counters in the workspace with a synchronous memset. */
srn_status srn_create(const srn_config* cfg, const srn_tensors* tensors, void* workspace_dev,
                      size_t workspace_bytes, int64_t max_points, srn_handle** out);

/* Destroy a handle (frees its host state and cached CUDA graphs; no device buffer). */
srn_status srn_destroy(srn_handle* h);

/* Message of the last error on the calling thread ("" if none). */
const char* srn_last_error(void);

/* Re-derive the BF16 shadow of [0, n_group_a) from the float32 master (call after
 * writing parameters by hand).  A no-op for FP32 handles. */
srn_status srn_sync_shadow(srn_handle* h, void* stream);

/* Batch sampling (Sec. 6 "Training": points uniform in [-1,1]^3 each iteration).
 * Point n of brick b at this step comes from Philox4x32-10 with counter
 * (n, b, step, 0) and key (seed, seed >> 32); coordinate d = 2 (r_d >> 8) 2^-24 - 1.
 * Within each brick the points are then reordered by the Morton code of their
 * 32^3 bin, which does not change the batch as a set.  offsets[B+1] (host):
 * brick b gets offsets[b+1] - offsets[b] points, offsets[B] <= max_points.
 * If step_dev is non-NULL the step is read from device memory (graph replays). */
srn_status srn_sample_points(srn_handle* h, void* stream, uint64_t seed, uint64_t step,
                             const uint64_t* step_dev, const int64_t* offsets, float* xyz_dev);

/* Allocation-free variant of srn_sample_points (the paper has no counterpart; this is
 * an interface convenience).  Some callers cannot allocate device memory at all -- a
 * plug-in running inside a host application that owns the GPU memory budget, or a
 * real-time loop whose allocator must not be entered -- so they cannot create a handle
 * with its workspace.  This entry point needs neither: its scratch (each point's rank
 * in its bin and the bin histograms) is a file-scope __device__ array of 1.5 MiB that
 * every GPU which loads the library holds until the process exits.  It calls no
 * allocation routine of any kind.
 *   - At most SRN_STATIC_SAMPLER_MAX_POINTS points over at most
 *     SRN_STATIC_SAMPLER_MAX_BRICKS bricks; larger requests return SRN_ERR_INVALID_ARG.
 *   - Same draws and same per-brick Morton ordering as srn_sample_points with
 *     step_dev = NULL (order inside a bin may differ between runs).
 *   - The first call on a device looks up that device's copy of the array (with the
 *     device current); make that first call before any stream capture.  The address
 *     is kept per device index for the rest of the process: it belongs to the CUDA
 *     runtime's primary context of that device, so calls must run with that context
 *     current (a caller's own driver-API context on the same device is not
 *     supported), and after cudaDeviceReset the kept address is stale -- do not call
 *     this entry point again in that process.
 *   - All calls share the one array: calls that overlap on the GPU (two streams, or two
 *     host threads) race on it and must be serialised by the caller.  The histograms
 *     are cleared on the stream at the start of every call. */
#define SRN_STATIC_SAMPLER_MAX_POINTS 131072
#define SRN_STATIC_SAMPLER_MAX_BRICKS 8
srn_status srn_sample_points_static(void* stream, uint64_t seed, uint64_t step, int32_t n_bricks,
                                    const int64_t* offsets, float* xyz_dev);

/* Ground truth v(x) of Sec. 4.3.1: trilinear interpolation of a float32 volume
 * [dims[2]][dims[1]][dims[0]] (x fastest).  Brick b's local [-1,1]^3 spans the
 * inclusive voxel box boxes[b] = (lo_x, lo_y, lo_z, hi_x, hi_y, hi_z) (host
 * [B][6]; hi > lo per axis), corner-aligned (Sec. 5.1: ghost cells included). */
srn_status srn_sample_target(srn_handle* h, void* stream, const float* volume_dev,
                             const int64_t dims[3], const int64_t* boxes,
                             const float* xyz_dev, const int64_t* offsets, float* target_dev);

/* A tiled copy of a float32 volume for the ground-truth lookup v(x) of Sec. 4.3.1, which
 * reads eight corners per point: the copy holds tiles of 4 x 4 x 4 voxels (tile
 * (i, j, k) at tile index (k * ceil(dims[1]/4) + j) * ceil(dims[0]/4) + i, 64 floats per
 * tile; inside a tile voxel (x, y, z) mod 4 at ((z * 4) + y) * 4 + x), each extent
 * padded to whole tiles with zeros, so that a point's corners usually share one
 * 256-byte tile instead of four rows far apart.  It is an input layout, not a cache:
 * the copy reflects volume_dev when srn_tile_volume ran.
 * srn_tiled_volume_bytes: the size of the copy for dims (each >= 2).
 * srn_tile_volume: writes it (device memory, 16-byte aligned, of that size) on `stream`
 * from the x-fastest volume_dev; does not need a handle.
 * srn_sample_target_tiled: srn_sample_target reading such a copy (dims of the volume
 * it came from); the results are identical. */
srn_status srn_tiled_volume_bytes(const int64_t dims[3], size_t* bytes);
srn_status srn_tile_volume(void* stream, const float* volume_dev, const int64_t dims[3], float* tiled_dev);
srn_status srn_sample_target_tiled(srn_handle* h, void* stream, const float* tiled_dev,
                                   const int64_t dims[3], const int64_t* boxes,
                                   const float* xyz_dev, const int64_t* offsets, float* target_dev);

/* Forward query f(x) = d(e(x)) (Eq. 1-3 and Sec. 4.1.2) of every brick's points:
 * out_dev[n] for xyz_dev[n].  offsets as in srn_sample_points. */
srn_status srn_forward(srn_handle* h, void* stream, const float* xyz_dev,
                       const int64_t* offsets, float* out_dev);

/* BF16 handles run the density passes of srn_backward / srn_train_step on a second
 * stream of their own, created by srn_create: it is forked from and joined back into
 * the caller's stream within the call, so work that the caller orders after the call
 * on `stream` sees every result.
 *
 * Forward, L_rec (Sec. 4.3.1) and its gradient into F and the decoder (step (1) of
 * Sec. 4.3.2), written (not accumulated) into the gradient buffer.  With
 * SRN_UPSTREAM the gradient is instead that of any loss whose dL/df is given.  With
 * SRN_DENSITY it also evaluates L_den (Eq. 7-9, with h(x) = (f(x) - v(x))^2 and the
 * target rho* held constant) and writes its gradient into G (step (2)).  With
 * SRN_REC_DG the gradient of L_rec (or of the upstream loss) through the features
 * is added into G's gradient; with neither flag G's gradient is zero.  losses_dev (device [B][4] float64, may be NULL) receives
 * per brick (L_rec, L_den, sum of rho over the batch, point count). */
srn_status srn_backward(srn_handle* h, void* stream, const float* xyz_dev,
                        const float* target_dev, const int64_t* offsets, uint32_t flags,
                        double* losses_dev);

/* One Adam step (Sec. 6: beta = (0.9, 0.99), lr 0.01 for F and the decoder) on
 * [0, n_group_a); with SRN_DENSITY also on G (lr 0.001), whose bias correction
 * counts only the steps that updated it.  Refreshes the BF16 shadow. */
srn_status srn_step(srn_handle* h, void* stream, uint32_t flags);

/* One whole training iteration: sample -> target -> backward -> Adam, with the
 * sampler step read from the device counter that srn_step advances.  On a
 * non-default stream the sequence is captured once per (flags, offsets, volume)
 * into a CUDA graph and replayed.  losses_dev as in srn_backward.  On the BF16 path
 * with the density loss the Adam step of F and the decoder runs while the gradient
 * of L_den into G is still being formed (G's Adam step follows it); the results are
 * those of the sequence above. */
srn_status srn_train_step(srn_handle* h, void* stream, uint64_t seed, const float* volume_dev,
                          const int64_t dims[3], const int64_t* boxes, const int64_t* offsets,
                          uint32_t flags, float* xyz_dev, float* target_dev, double* losses_dev);

/* The training routine of Sec. 4.3.2 and the plateau scheduler of Sec. 5.2, applied
 * per brick on the device by srn_train_step with SRN_SCHEDULE (no host round trip):
 *   - G (the transforms) is trained from iteration delay_iters + 1 (500 in the paper) ...
 *   - ... until the mean of L_den over the last density_window density iterations
 *     (1000) has not dropped by a relative density_rel (1e-4) below the mean of the
 *     window before, or past density_frac (0.8) of total_iters: then G stays fixed;
 *   - when L_rec has not dropped by a relative plateau_rel (1e-4) below its best for
 *     more than plateau_window (500) iterations, the brick's learning rates are
 *     multiplied by plateau_factor (0.1); at the plateau_max-th (3rd) time the brick
 *     has finished and its parameters are no longer updated.
 * srn_set_schedule stores the routine and restarts every brick's state (iteration 0);
 * density_window <= 4096, all counts positive, 0 < rel, 0 < frac <= 1,
 * 0 < plateau_factor <= 1.  srn_read_schedule copies the per-brick state to host
 * memory (synchronising `stream`). */
typedef struct {
  int32_t delay_iters;
  int32_t density_window;
  float density_rel;
  float density_frac;
  int64_t total_iters;
  int32_t plateau_window;
  float plateau_rel;
  float plateau_factor;
  int32_t plateau_max;
} srn_schedule;
typedef struct {
  int64_t iteration;        /* iterations trained */
  float lr_scale;           /* plateau_factor ^ plateaus */
  int32_t plateaus;         /* plateau reductions so far */
  int32_t finished;         /* 1: the brick is no longer updated */
  int32_t density_on;       /* 1: G is trained at the next iteration */
  int32_t density_stopped;  /* 1: early stop or the iteration cutoff has fired */
  int32_t density_iters;    /* iterations that trained G */
  double best_rec;          /* lowest L_rec of the plateau test */
} srn_brick_schedule;
srn_status srn_set_schedule(srn_handle* h, const srn_schedule* sched);
srn_status srn_read_schedule(srn_handle* h, void* stream, srn_brick_schedule* out_host);

/* Batch shares after bricks finish (Sec. 5.2: a finished model frees its GPU for the next
 * one; here the bricks share one GPU, and a finished brick frees its share of each
 * batch for the bricks still training).  Host only; no handle, no GPU.
 * base_counts[n_bricks] (each >= 1) are the points per brick while all train; state is
 * srn_read_schedule's output (only `finished` is read).  out_offsets[n_bricks + 1]
 * receives batch offsets with the same total: a finished brick keeps
 * min(min_points, base) points (min_points >= 1, so its L_rec stays defined), and the
 * points the finished bricks give up, P, go to the unfinished bricks in proportion to
 * their base counts: brick a gets floor(P base_a / W) more (W = the unfinished bricks'
 * base total), and the points that flooring leaves go one each to the unfinished bricks
 * with the largest remainders (P base_a mod W), ties to the lower index.  With no
 * brick finished, or every brick finished, the offsets are those of the base counts.
 * Passing the new offsets to srn_train_step captures a new CUDA graph for them. */
srn_status srn_rebalance(int32_t n_bricks, const int64_t* base_counts, const srn_brick_schedule* state,
                         int64_t min_points, int64_t* out_offsets);

/* Headless volume render (Sec. 6) of the domain decomposition (Sec. 5.3) into
 * rgba_dev [height][width][4].  Each ray is clipped to [-1,1]^3 and sampled at
 * `samples` midpoints; every sample is hashed to its brick (grid[3] = I, J, K,
 * B = I J K) and mapped into that brick's local domain using boxes[B][6] inside a
 * volume of `vox` voxels per axis; the value is mapped through the 256 x RGBA
 * lut_dev between vmin and vmax and composited front to back with
 * alpha = 1 - exp(-a dt / (2/512)).  Batches of at most max_points samples. */
srn_status srn_render(srn_handle* h, void* stream, const srn_camera* cam, const float* lut_dev,
                      float vmin, float vmax, int32_t width, int32_t height, int32_t samples,
                      const int32_t grid[3], const int64_t* boxes, int64_t vox, float* rgba_dev);

/* Progressive rendering (Sec. 6): the same pixels as srn_render, evaluated in the
 * order of an image hierarchy.  Level l holds the pixels (a 2^l, b 2^l); the coarsest
 * level L (the first with 2^L >= max(width, height)) is pixel (0, 0), and each finer
 * level adds, row by row and left to right, the pixels no coarser level holds (three
 * of every 2 x 2 block: a checkerboard).  This call renders the pixels first ..
 * first + count - 1 of that order into rgba_dev ([height][width][4]; other pixels
 * untouched; count is the pass's batch size: small passes answer sooner, large ones
 * finish the frame sooner).  If preview_dev ([height][width][4], not rgba_dev) is not
 * NULL it receives the in-progress image after first + count pixels: evaluated pixels
 * as they are, the others the bilinear upscale of the finest complete level (sample
 * index clamped to the level's grid; 0 when nothing is evaluated).  rgba_dev must hold
 * the pixels of the earlier passes.  Other arguments as srn_render;
 * width * height < 2^31, 0 <= first, 0 <= count, first + count <= width * height. */
srn_status srn_render_progressive(srn_handle* h, void* stream, const srn_camera* cam, const float* lut_dev,
                                  float vmin, float vmax, int32_t width, int32_t height, int32_t samples,
                                  const int32_t grid[3], const int64_t* boxes, int64_t vox, int64_t first,
                                  int64_t count, float* rgba_dev, float* preview_dev);

/* Checkpointing (no counterpart in the paper beyond saving trained models, Sec. 5.2).
 * The caller owns and saves the parameters, Adam moments and data ranges; these calls
 * move the rest of the training state (sampler step, Adam step counts and bias
 * corrections, and the per-brick training-routine state with its parameters) as an
 * opaque blob of srn_state_bytes() bytes, tagged with the brick and grid counts.  Both synchronise `stream`.  Loading a blob of another build or
 * shape is SRN_ERR_INVALID_ARG. */
srn_status srn_state_bytes(srn_handle* h, size_t* bytes);
srn_status srn_save_state(srn_handle* h, void* stream, void* dst, size_t bytes);
srn_status srn_load_state(srn_handle* h, void* stream, const void* src, size_t bytes);

/* Full-volume decode (the decompression of Sec. 7): f at every voxel of a volume of
 * `vox` voxels per axis modelled by the domain decomposition of Sec. 5.  Voxel (i, j, k)
 * sits at the global position -1 + 2 (i, j, k) / (vox - 1); along each axis it belongs
 * to brick min(floor(n i / (vox - 1)), n - 1) of the grid[3] = (I, J, K) bricks (the
 * Sec. 5.3 hash at that position), and is queried in that brick's local [-1, 1]^3
 * given by boxes[B][6] (lo xyz, hi xyz voxels, as in srn_render).  out_dev receives
 * [vox][vox][vox] float32, z slowest.  Batches of at most max_points voxels; FP32 or
 * BF16 as the handle. */
srn_status srn_decode(srn_handle* h, void* stream, const int32_t grid[3], const int64_t* boxes, int64_t vox,
                      float* out_dev);

/* Measurement hook (no counterpart in the paper).  `target` picks what is timed:
 * SRN_TIME_OFF nothing; SRN_TIME_QUERY every launch of the query pass (srn_forward,
 * srn_backward, and srn_train_step when it runs eagerly: the fused kernel, or the
 * three kernels of the BF16 training pass together); SRN_TIME_ENCODER,
 * SRN_TIME_DECODER or SRN_TIME_SCATTER one kernel of the BF16 training pass
 * (srn_backward of a BF16 handle; other calls are not timed).  Launches made outside
 * stream capture are bracketed by CUDA events on their stream.  srn_read_timing
 * synchronises on the recorded events and returns the summed kernel time in
 * milliseconds and the number of timed launches since the last read (then resets
 * both).  Changing the target clears the counters.  Any other target is
 * SRN_ERR_INVALID_ARG. */
#define SRN_TIME_OFF 0
#define SRN_TIME_QUERY 1
#define SRN_TIME_ENCODER 2
#define SRN_TIME_DECODER 3
#define SRN_TIME_SCATTER 4
srn_status srn_set_timing(srn_handle* h, int32_t target);
srn_status srn_read_timing(srn_handle* h, double* total_ms, int64_t* launches);

/* Launch shape of the BF16 training pass (no counterpart in the paper; the paper's
 * encoder and scatter are library kernels).  The pass cuts each brick's Morton-sorted
 * points into tiles: runs of consecutive points inside one aligned Morton block of at
 * most 2^tile_level units (a unit is 1/16 of the domain per axis), holding at most
 * tile_points points, and within that block's node box in every grid (a brick's level is
 * further capped so that its boxes fit the kernels' shared memory).  density_ctas is the
 * CTAs per SM of the density-gradient pass that runs beside the scatter.  Every tuning
 * gives the same results up to the rounding of the fixed-point gradient sums (their
 * quantum is set per tile and grid).  The default, set by srn_create, is
 * {1024, 9, 2}.
 *   srn_get_tuning  copies the handle's tuning to *out.
 *   srn_set_tuning  installs *t: 128 <= tile_points <= 1024 and a multiple of 32,
 *                   0 <= tile_level <= 9, 1 <= density_ctas <= 4, else
 *                   SRN_ERR_INVALID_ARG.  Training steps captured in CUDA graphs by
 *                   srn_train_step are re-captured.  FP32 handles store it unused.
 *   srn_autotune    picks the tile shape (tile_points, tile_level) of a BF16 handle by
 *                   timing srn_backward(stream, xyz_dev, target_dev, offsets, flags) for
 *                   each candidate of a fixed set ({256, 512, 768, 1024} points x
 *                   levels {2, 3, 4, 6, 9}), the handle's current tuning first: each
 *                   candidate runs once untimed, then `reps` (1..100) times bracketed by
 *                   CUDA events on `stream`; its score is the median, and a candidate
 *                   replaces the best so far only when at least 1% faster.  It installs
 *                   the winner as srn_set_tuning does, writes it to *out (may be NULL),
 *                   then runs srn_backward once more with it, so that the gradient buffer
 *                   holds that pass's gradient.  Parameters, Adam moments and step
 *                   counters are not touched.  Synchronises `stream`; not allowed while
 *                   `stream` is being captured (SRN_ERR_STATE) or on FP32 handles
 *                   (SRN_ERR_UNSUPPORTED).  Arguments otherwise as srn_backward. */
typedef struct {
  int32_t tile_points;
  int32_t tile_level;
  int32_t density_ctas;
} srn_tuning;
srn_status srn_get_tuning(srn_handle* h, srn_tuning* out);
srn_status srn_set_tuning(srn_handle* h, const srn_tuning* t);
srn_status srn_autotune(srn_handle* h, void* stream, const float* xyz_dev, const float* target_dev,
                        const int64_t* offsets, uint32_t flags, int32_t reps, srn_tuning* out);

/* Synchronise `stream` and report device-side status since the last call (then clear
 * it): SRN_ERR_DEVICE_TIMEOUT if a kernel gave up a bounded wait on the tensor cores
 * (its outputs are then invalid), else SRN_ERR_NONFINITE if a loss was NaN/Inf, else
 * SRN_OK. */
srn_status srn_get_status(srn_handle* h, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SRN_H */
