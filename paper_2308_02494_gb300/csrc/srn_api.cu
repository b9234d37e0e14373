// C ABI of libsrn (declared in include/srn.h): argument validation, workspace
// carving, kernel dispatch and the CUDA-graph cache of srn_train_step.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "render.h"

namespace {

thread_local std::string g_err;

srn_status fail(srn_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

srn_status cuda_fail(cudaError_t e, const char* where) {
  return fail(SRN_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

}  // namespace

// Entry points defined in other translation units report through this.
srn_status srn::report(srn_status s, const char* message) { return fail(s, "%s", message); }

namespace {

int64_t round64(int64_t n) { return (n + 63) / 64 * 64; }
size_t align256(size_t n) { return (n + 255) / 256 * 256; }

srn_status check_config(const srn_config* c) {
  if (!c) return fail(SRN_ERR_INVALID_ARG, "config is NULL");
  if (c->n_bricks < 1 || c->n_bricks > SRN_MAX_BRICKS)
    return fail(SRN_ERR_INVALID_ARG, "n_bricks %d outside [1, %d]", c->n_bricks, SRN_MAX_BRICKS);
  if (c->n_grids < 1 || c->channels < 1 || c->res < 2 || c->hidden < 1)
    return fail(SRN_ERR_INVALID_ARG, "non-positive model size");
  if (c->hidden != srn::kHidden) return fail(SRN_ERR_UNSUPPORTED, "hidden must be 64");
  if (c->channels > 2) return fail(SRN_ERR_UNSUPPORTED, "channels must be 1 or 2");
  const int K = c->n_grids * c->channels;
  if (K != 16 && K != 32 && K != 64 && K != 128)
    return fail(SRN_ERR_UNSUPPORTED, "n_grids*channels = %d not in {16, 32, 64, 128}", K);
  if (c->res > 64) return fail(SRN_ERR_UNSUPPORTED, "res %d > 64", c->res);
  if (c->flat_top_p < 1 || c->flat_top_p > 16)
    return fail(SRN_ERR_UNSUPPORTED, "flat_top_p %d outside [1, 16]", c->flat_top_p);
  if (c->precision != SRN_FP32 && c->precision != SRN_BF16)
    return fail(SRN_ERR_INVALID_ARG, "unknown precision %d", c->precision);
  if (!(c->density_eps > 0.f) || !(c->lr_feat >= 0.f) || !(c->lr_xform >= 0.f) ||
      !(c->beta1 >= 0.f && c->beta1 < 1.f) || !(c->beta2 >= 0.f && c->beta2 < 1.f) ||
      !(c->adam_eps > 0.f))
    return fail(SRN_ERR_INVALID_ARG, "bad optimiser or epsilon setting");
  return SRN_OK;
}

void make_layout(const srn_config* c, srn_layout* L) {
  const int64_t B = c->n_bricks, M = c->n_grids, R = c->res, C = c->channels;
  const int64_t K = M * C;
  L->size_F = round64(M * R * R * R * C);
  L->size_W1 = round64(64 * K);
  L->size_W2 = round64(64 * 64);
  L->size_w3 = round64(64);
  L->size_G = round64(M * 12);
  L->off_F = 0;
  L->off_W1 = L->off_F + B * L->size_F;
  L->off_W2 = L->off_W1 + B * L->size_W1;
  L->off_w3 = L->off_W2 + B * L->size_W2;
  L->n_group_a = L->off_w3 + B * L->size_w3;
  L->off_G = L->n_group_a;
  L->n_params = L->off_G + B * L->size_G;
}

// Workspace carving (every piece 256-byte aligned).
struct WsLayout {
  size_t state, acc, gsum, rsum, rho, herr, sort_rank, sort_hist, feat, dfeat, gmax, ustart, tiles, tile_ctr;
  size_t sched, sring;
  size_t r_loc, r_rank, r_bid, r_pos, r_xyz, r_val, r_cnt, r_off, total;
};

WsLayout ws_layout(const srn_config* c, int64_t maxp) {
  WsLayout w{};
  size_t o = 0;
  w.state = o; o += align256(sizeof(srn::StepState) + 64);
  w.acc = o; o += align256(sizeof(double) * srn::kAccPerBrick * c->n_bricks);
  w.gsum = o; o += align256(sizeof(double) * 13 * c->n_grids * c->n_bricks);
  w.rsum = o; o += align256(sizeof(double) * 12 * c->n_grids * c->n_bricks);
  w.rho = o; o += align256(sizeof(float) * maxp);
  w.herr = o; o += align256(sizeof(float) * maxp);
  w.sort_rank = o; o += align256(sizeof(uint32_t) * maxp);
  w.sort_hist = o; o += align256(sizeof(uint32_t) * srn::kSortBins * c->n_bricks);
  // BF16 training pass: features Y [N][K] and dL/dy [M][N][C], both bfloat16
  const size_t kbytes = c->precision == SRN_BF16 ? sizeof(uint16_t) * c->n_grids * c->channels : 0;
  w.feat = o; o += align256(kbytes * maxp);
  w.dfeat = o; o += align256(kbytes * maxp);
  // largest |dL/dy| per grid and 128-point decoder tile (tcgen05 decoder, K = 128)
  const int64_t dec_tiles = maxp / 128 + c->n_bricks + 1;
  w.gmax = o; o += c->precision == SRN_BF16 ? align256(sizeof(uint16_t) * srn::kMaxGrids * dec_tiles) : 0;
  // BF16 tiles: unit starts, and at most one tile per unit plus one per kMinTilePoints
  // points (the smallest tile any tuning allows)
  const bool bf16 = c->precision == SRN_BF16;
  const int64_t max_tiles = (int64_t)c->n_bricks * (srn::kUnits + 1) + maxp / srn::kMinTilePoints + 1;
  w.ustart = o; o += bf16 ? align256(sizeof(int32_t) * (srn::kUnits + 1) * c->n_bricks) : 0;
  w.tiles = o; o += bf16 ? align256(sizeof(srn::ScatTile) * max_tiles) : 0;
  w.tile_ctr = o; o += align256(sizeof(int32_t) * 4);
  w.sched = o; o += align256(sizeof(srn::BrickSched) * c->n_bricks);
  w.sring = o; o += align256(sizeof(double) * 2 * srn::kMaxDensityWindow * c->n_bricks);
  w.r_loc = o; o += align256(sizeof(float) * 3 * maxp);
  w.r_rank = o; o += align256(sizeof(uint32_t) * maxp);
  w.r_bid = o; o += align256(sizeof(uint32_t) * maxp);
  w.r_pos = o; o += align256(sizeof(uint32_t) * maxp);
  w.r_xyz = o; o += align256(sizeof(float) * 3 * maxp);
  w.r_val = o; o += align256(sizeof(float) * maxp);
  w.r_cnt = o; o += align256(sizeof(uint32_t) * c->n_bricks);
  w.r_off = o; o += align256(sizeof(int64_t) * (c->n_bricks + 1));
  w.total = o;
  return w;
}

struct GraphKey {
  uint32_t flags;
  uint64_t seed;
  const void* vol;
  int64_t dims[3];
  std::vector<int64_t> boxes, offsets;
  const void *xyz, *target, *losses;
  cudaStream_t stream;
  bool operator==(const GraphKey& o) const {
    return flags == o.flags && seed == o.seed && vol == o.vol && dims[0] == o.dims[0] &&
           dims[1] == o.dims[1] && dims[2] == o.dims[2] && boxes == o.boxes &&
           offsets == o.offsets && xyz == o.xyz && target == o.target && losses == o.losses &&
           stream == o.stream;
  }
};

struct GraphEntry {
  GraphKey key;
  int eager_runs;
  cudaGraphExec_t exec;
};

}  // namespace

struct srn_handle {
  srn_config cfg;
  srn_layout lay;
  srn_tensors t;
  unsigned char* ws;
  size_t ws_bytes;
  int64_t max_points;
  WsLayout wl;
  int num_sms;
  std::vector<GraphEntry> graphs;
  // training routine (srn_set_schedule)
  bool has_sched = false;
  srn_schedule sched_cfg{};
  // measurement hook: a ring of event pairs around the query pass or one of its kernels
  int32_t timing = SRN_TIME_OFF;
  std::vector<cudaEvent_t> ev_start, ev_stop;
  std::vector<char> ev_used;
  size_t ev_next = 0;
  double timed_ms = 0.0;
  int64_t timed_launches = 0;
  // BF16 training: a second stream for the density passes beside the scatter
  srn::SideStream side{nullptr, nullptr, nullptr, nullptr, false};
  // set by the training step around its backward pass: the batch is the sampler's, whose
  // histogram holds the bin starts the BF16 tile list needs
  const uint32_t* batch_bins = nullptr;
  // launch shape of the BF16 training pass (srn_set_tuning / srn_autotune)
  srn::Tuning tune = srn::kDefaultTuning;

  srn::StepState* state() const { return reinterpret_cast<srn::StepState*>(ws + wl.state); }
  srn::BrickSched* sched() const { return reinterpret_cast<srn::BrickSched*>(ws + wl.sched); }
  double* sring() const { return reinterpret_cast<double*>(ws + wl.sring); }
  srn::SchedParams sched_params() const {
    const srn_schedule& c = sched_cfg;
    return srn::SchedParams{c.delay_iters, c.density_window, c.density_rel, c.density_frac, c.total_iters,
                            c.plateau_window, c.plateau_rel, c.plateau_factor, c.plateau_max};
  }
  int32_t* status() const { return reinterpret_cast<int32_t*>(ws + wl.state + sizeof(srn::StepState)); }
  srn::TrainWs train_ws() const {
    srn::TrainWs w;
    w.rho = reinterpret_cast<float*>(ws + wl.rho);
    w.herr = reinterpret_cast<float*>(ws + wl.herr);
    w.acc = reinterpret_cast<double*>(ws + wl.acc);
    w.gsum = reinterpret_cast<double*>(ws + wl.gsum);
    w.rsum = reinterpret_cast<double*>(ws + wl.rsum);
    w.rec_dg = 0;
    w.status = status();
    w.upstream = 0;
    w.Y = reinterpret_cast<__nv_bfloat16*>(ws + wl.feat);
    w.dY = reinterpret_cast<__nv_bfloat16*>(ws + wl.dfeat);
    w.gmax_blk = cfg.precision == SRN_BF16 && cfg.n_grids * cfg.channels == 128
                     ? reinterpret_cast<uint16_t*>(ws + wl.gmax) : nullptr;
    w.ustart = reinterpret_cast<int32_t*>(ws + wl.ustart);
    w.tiles = reinterpret_cast<srn::ScatTile*>(ws + wl.tiles);
    w.tile_ctr = reinterpret_cast<int32_t*>(ws + wl.tile_ctr);
    w.sched = nullptr;
    w.eps = cfg.density_eps;
    w.bin_start = batch_bins;
    return w;
  }
  srn::Model model() const {
    srn::Model m{};
    const float* p = t.params_dev;
    const __nv_bfloat16* s = reinterpret_cast<const __nv_bfloat16*>(t.shadow_dev);
    m.G = p + lay.off_G;
    m.range = t.range_dev;
    m.F32 = p + lay.off_F;
    m.W1f = p + lay.off_W1;
    m.W2f = p + lay.off_W2;
    m.w3 = p + lay.off_w3;
    m.F16 = s ? s + lay.off_F : nullptr;
    m.W1h = s ? s + lay.off_W1 : nullptr;
    m.W2h = s ? s + lay.off_W2 : nullptr;
    m.sF = lay.size_F; m.sW1 = lay.size_W1; m.sW2 = lay.size_W2; m.sw3 = lay.size_w3; m.sG = lay.size_G;
    m.M = cfg.n_grids; m.C = cfg.channels; m.R = cfg.res; m.K = cfg.n_grids * cfg.channels;
    m.p = cfg.flat_top_p;
    return m;
  }
  srn::Grads grads() const {
    srn::Grads g{};
    float* d = t.grads_dev;
    g.dF = d + lay.off_F; g.dW1 = d + lay.off_W1; g.dW2 = d + lay.off_W2; g.dw3 = d + lay.off_w3;
    g.sF = lay.size_F; g.sW1 = lay.size_W1; g.sW2 = lay.size_W2; g.sw3 = lay.size_w3;
    return g;
  }
  srn::Launch launch(void* stream) const { return srn::Launch{static_cast<cudaStream_t>(stream), num_sms}; }
};

namespace {

srn_status check_handle(const srn_handle* h) {
  if (!h) return fail(SRN_ERR_INVALID_ARG, "handle is NULL");
  return SRN_OK;
}

srn_status make_bricks(const srn_handle* h, const int64_t* offsets, srn::Bricks* br) {
  if (!offsets) return fail(SRN_ERR_INVALID_ARG, "offsets is NULL");
  const int B = h->cfg.n_bricks;
  if (offsets[0] != 0) return fail(SRN_ERR_INVALID_ARG, "offsets[0] must be 0");
  for (int b = 0; b < B; ++b)
    if (offsets[b + 1] < offsets[b]) return fail(SRN_ERR_INVALID_ARG, "offsets decrease at brick %d", b);
  if (offsets[B] > h->max_points)
    return fail(SRN_ERR_INVALID_ARG, "%lld points exceed max_points %lld", (long long)offsets[B],
                (long long)h->max_points);
  br->n = B;
  br->dev = nullptr;
  for (int b = 0; b <= B; ++b) br->off[b] = offsets[b];
  return SRN_OK;
}

srn_status check_training_counts(const srn::Bricks& br) {
  for (int b = 0; b < br.n; ++b)
    if (br.off[b + 1] == br.off[b])
      return fail(SRN_ERR_INVALID_ARG, "brick %d has no points (its losses are means over the batch)", b);
  return SRN_OK;
}

srn_status run_query(srn_handle* h, void* stream, srn::QueryMode mode, const srn::Bricks& br,
                     const float* xyz, const float* target, float* out, int upstream = 0,
                     const srn::BrickSched* sched = nullptr, int rec_dg = 0) {
  const srn::Launch L = h->launch(stream);
  const srn::Model md = h->model();
  const srn::Grads gr = h->grads();
  srn::TrainWs ws = h->train_ws();
  ws.upstream = upstream;
  ws.sched = sched;
  ws.rec_dg = rec_dg;
  size_t slot = 0;
  bool timed = false;
  const bool bf16_train = h->cfg.precision == SRN_BF16 && mode != srn::kForward;
  const bool time_pass = h->timing == SRN_TIME_QUERY;
  const bool time_kernel = h->timing >= SRN_TIME_ENCODER && bf16_train;
  srn::KernelMark mark{};
  if ((time_pass || time_kernel) && !h->ev_start.empty()) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(L.stream, &cap);
    if (cap == cudaStreamCaptureStatusNone) {
      slot = h->ev_next++ % h->ev_start.size();
      if (h->ev_used[slot]) {  // retire the oldest pair before reusing it
        float ms = 0.f;
        cudaEventSynchronize(h->ev_stop[slot]);
        cudaEventElapsedTime(&ms, h->ev_start[slot], h->ev_stop[slot]);
        h->timed_ms += ms;
        h->timed_launches += 1;
        h->ev_used[slot] = 0;
      }
      if (time_pass) cudaEventRecord(h->ev_start[slot], L.stream);
      mark = srn::KernelMark{h->timing - SRN_TIME_ENCODER, h->ev_start[slot], h->ev_stop[slot]};
      timed = true;
    }
  }
  cudaError_t e;
  if (h->cfg.precision != SRN_BF16)
    e = srn::launch_query_fp32(L, mode, md, gr, br, ws, xyz, target, out);
  else if (mode == srn::kForward)
    e = srn::launch_forward_bf16(L, md, br, xyz, out);
  else
    e = srn::launch_train_bf16(L, mode == srn::kTrainDensity, md, gr, br, ws, xyz, target, h->tune,
                               timed && time_kernel ? &mark : nullptr, h->side.stream ? &h->side : nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "query kernel");
  if (timed) {
    if (time_pass) cudaEventRecord(h->ev_stop[slot], L.stream);
    h->ev_used[slot] = 1;
  }
  return SRN_OK;
}

srn_status do_finalize(srn_handle* h, void* stream, const srn::Bricks& br, uint32_t flags, double* losses) {
  const srn::BrickSched* sched = (flags & SRN_SCHEDULE) ? h->sched() : nullptr;
  const bool dens = (flags & SRN_DENSITY) != 0 || sched;
  srn::TrainWs tws = h->train_ws();
  tws.sched = sched;
  tws.rec_dg = (flags & SRN_REC_DG) ? 1 : 0;
  cudaError_t e = srn::launch_finalize(h->launch(stream), br, h->model(), tws, dens, h->t.grads_dev + h->lay.off_G,
                                       h->lay.size_G, losses);
  if (e != cudaSuccess) return cuda_fail(e, "finalize kernel");
  return SRN_OK;
}

// With `split` (the BF16 pass with its density passes on the second stream) the pass
// returns before the finalisation and without waiting for the second stream: the caller
// waits for h->side.join and calls do_finalize.
srn_status do_backward(srn_handle* h, void* stream, const float* xyz, const float* target,
                       const srn::Bricks& br, uint32_t flags, double* losses, bool split = false) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // with the training routine, the density passes always run and each brick follows
  // its device-side decision
  const srn::BrickSched* sched = (flags & SRN_SCHEDULE) ? h->sched() : nullptr;
  const bool dens = (flags & SRN_DENSITY) != 0 || sched;
  cudaError_t e = cudaMemsetAsync(h->t.grads_dev, 0, sizeof(float) * h->lay.n_params, s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(h->ws + h->wl.acc, 0, h->wl.rsum - h->wl.acc + sizeof(double) * 12 * h->cfg.n_grids * h->cfg.n_bricks, s);
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  const int rec_dg = (flags & SRN_REC_DG) ? 1 : 0;
  h->side.defer_join = split;
  srn_status st = run_query(h, stream, dens ? srn::kTrainDensity : srn::kTrain, br, xyz, target,
                            nullptr, (flags & SRN_UPSTREAM) ? 1 : 0, sched, rec_dg);
  h->side.defer_join = false;
  if (st != SRN_OK || split) return st;
  const srn::Launch L = h->launch(stream);
  const srn::Model md = h->model();
  srn::TrainWs tws = h->train_ws();
  tws.sched = sched;
  tws.rec_dg = rec_dg;
  if (dens && !(h->cfg.precision == SRN_BF16 && h->side.stream)) {   // else run beside the BF16 scatter
    e = srn::launch_density(L, md, br, tws, xyz, h->cfg.density_eps);
    if (e != cudaSuccess) return cuda_fail(e, "density kernels");
  }
  return do_finalize(h, stream, br, flags, losses);
}

srn_status do_step(srn_handle* h, void* stream, uint32_t flags, int seg0 = 0, int seg1 = 5, bool advance = true) {
  const srn_config& c = h->cfg;
  const srn_layout& ly = h->lay;
  srn::AdamLayout al{};
  const int64_t off[5] = {ly.off_F, ly.off_W1, ly.off_W2, ly.off_w3, ly.off_G};
  const int64_t size[5] = {ly.size_F, ly.size_W1, ly.size_W2, ly.size_w3, ly.size_G};
  for (int k = 0; k < 5; ++k) { al.off[k] = off[k]; al.size[k] = size[k]; }
  al.n_bricks = c.n_bricks;
  const bool sch = (flags & SRN_SCHEDULE) != 0;
  cudaError_t e = srn::launch_adam(h->launch(stream), al, h->t.params_dev, h->t.grads_dev, h->t.adam_m_dev,
                                   h->t.adam_v_dev, c.precision == SRN_BF16 ? h->t.shadow_dev : nullptr,
                                   (flags & SRN_DENSITY) != 0, c.lr_feat, c.lr_xform, c.beta1, c.beta2,
                                   c.adam_eps, h->state(), sch ? h->sched() : nullptr,
                                   sch ? h->sched_cfg.plateau_factor : 1.f, seg0, seg1, advance);
  if (e != cudaSuccess) return cuda_fail(e, "adam kernel");
  return SRN_OK;
}

srn_status make_boxes(const srn_handle* h, const int64_t dims[3], const int64_t* boxes,
                      srn::VolumeBoxes* vb) {
  if (!dims || !boxes) return fail(SRN_ERR_INVALID_ARG, "dims or boxes is NULL");
  for (int d = 0; d < 3; ++d)
    if (dims[d] < 2) return fail(SRN_ERR_INVALID_ARG, "volume dimension %d < 2", d);
  for (int b = 0; b < h->cfg.n_bricks; ++b) {
    for (int d = 0; d < 3; ++d) {
      const int64_t lo = boxes[6 * b + d], hi = boxes[6 * b + 3 + d];
      if (lo < 0 || hi >= dims[d] || hi <= lo)
        return fail(SRN_ERR_INVALID_ARG, "box of brick %d invalid on axis %d", b, d);
      vb->lo[b][d] = (int32_t)lo;
      vb->hi[b][d] = (int32_t)hi;
    }
  }
  return SRN_OK;
}

srn_status enqueue_train_step(srn_handle* h, void* stream, uint64_t seed, const float* vol,
                              const int64_t dims[3], const srn::VolumeBoxes& vb, const srn::Bricks& br,
                              uint32_t flags, float* xyz, float* target, double* losses) {
  const srn::Launch L = h->launch(stream);
  unsigned char* ws = h->ws;
  uint32_t* hist = reinterpret_cast<uint32_t*>(ws + h->wl.sort_hist);
  cudaError_t e = srn::launch_sample(L, br, seed, 0, &h->state()->step, xyz,
                                     reinterpret_cast<uint32_t*>(ws + h->wl.sort_rank), hist);
  if (e != cudaSuccess) return cuda_fail(e, "sampler");
  // v(x) on the sorted batch (the volume reads of neighbouring points then share lines)
  e = srn::launch_target(L, br, vol, dims[0], dims[1], dims[2], vb, xyz, target, (flags & SRN_VOLUME_TILED) != 0);
  if (e != cudaSuccess) return cuda_fail(e, "target lookup");
  // BF16 with the density loss: Adam of F and the decoder runs while the density
  // gradient (second stream) finishes; the transforms' Adam after the finalisation
  const bool split = h->cfg.precision == SRN_BF16 && h->side.stream && (flags & (SRN_DENSITY | SRN_SCHEDULE));
  h->batch_bins = hist;
  srn_status st = do_backward(h, stream, xyz, target, br, flags, losses, split);
  h->batch_bins = nullptr;
  if (st != SRN_OK) return st;
  if (split) {
    if ((st = do_step(h, stream, flags, 0, 4, true)) != SRN_OK) return st;
    e = cudaStreamWaitEvent(L.stream, h->side.join, 0);
    if (e != cudaSuccess) return cuda_fail(e, "join");
    if ((st = do_finalize(h, stream, br, flags, losses)) != SRN_OK) return st;
    if ((st = do_step(h, stream, flags, 4, 5, false)) != SRN_OK) return st;
  } else if ((st = do_step(h, stream, flags)) != SRN_OK) {
    return st;
  }
  if (flags & SRN_SCHEDULE) {
    e = srn::launch_schedule(L, h->cfg.n_bricks, h->sched(), h->sring(), losses, h->sched_params(), h->cfg.beta1,
                             h->cfg.beta2);
    if (e != cudaSuccess) return cuda_fail(e, "schedule kernel");
  }
  return SRN_OK;
}

}  // namespace

extern "C" {

const char* srn_last_error(void) { return g_err.c_str(); }

srn_status srn_param_layout(const srn_config* cfg, srn_layout* out) {
  srn_status s = check_config(cfg);
  if (s != SRN_OK) return s;
  if (!out) return fail(SRN_ERR_INVALID_ARG, "out is NULL");
  make_layout(cfg, out);
  return SRN_OK;
}

srn_status srn_workspace_size(const srn_config* cfg, int64_t max_points, size_t* bytes) {
  srn_status s = check_config(cfg);
  if (s != SRN_OK) return s;
  if (!bytes || max_points < 1) return fail(SRN_ERR_INVALID_ARG, "bytes is NULL or max_points < 1");
  *bytes = ws_layout(cfg, max_points).total;
  return SRN_OK;
}

srn_status srn_create(const srn_config* cfg, const srn_tensors* t, void* workspace, size_t ws_bytes,
                      int64_t max_points, srn_handle** out) {
  srn_status s = check_config(cfg);
  if (s != SRN_OK) return s;
  if (!t || !out || !workspace) return fail(SRN_ERR_INVALID_ARG, "tensors, workspace or out is NULL");
  if (!t->params_dev || !t->grads_dev || !t->adam_m_dev || !t->adam_v_dev || !t->range_dev)
    return fail(SRN_ERR_INVALID_ARG, "a required device tensor is NULL");
  if (cfg->precision == SRN_BF16 && !t->shadow_dev)
    return fail(SRN_ERR_INVALID_ARG, "BF16 precision needs the shadow buffer");
  if (max_points < 1) return fail(SRN_ERR_INVALID_ARG, "max_points < 1");
  const WsLayout wl = ws_layout(cfg, max_points);
  if (ws_bytes < wl.total)
    return fail(SRN_ERR_INVALID_ARG, "workspace of %zu bytes < %zu needed", ws_bytes, wl.total);
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0)
    return fail(SRN_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  for (const void* p : {(const void*)t->params_dev, (const void*)t->grads_dev, (const void*)t->adam_m_dev,
                        (const void*)t->adam_v_dev, (const void*)t->shadow_dev})
    if (reinterpret_cast<uintptr_t>(p) % 16 != 0)
      return fail(SRN_ERR_INVALID_ARG, "tensor pointers must be 16-byte aligned");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "device query");
  e = cudaMemset(static_cast<unsigned char*>(workspace) + wl.state, 0, wl.acc - wl.state);
  if (e != cudaSuccess) return cuda_fail(e, "workspace init");
  srn_handle* h = new srn_handle();
  h->cfg = *cfg;
  make_layout(cfg, &h->lay);
  h->t = *t;
  h->ws = static_cast<unsigned char*>(workspace);
  h->ws_bytes = ws_bytes;
  h->max_points = max_points;
  h->wl = wl;
  h->num_sms = sms;
  if (cfg->precision == SRN_BF16) {
    e = cudaStreamCreateWithFlags(&h->side.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->side.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->side.join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->side.enc_done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      srn_destroy(h);
      return cuda_fail(e, "side stream");
    }
  }
  *out = h;
  return SRN_OK;
}

srn_status srn_destroy(srn_handle* h) {
  if (!h) return fail(SRN_ERR_INVALID_ARG, "handle is NULL");
  for (auto& g : h->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (size_t i = 0; i < h->ev_start.size(); ++i) {
    cudaEventDestroy(h->ev_start[i]);
    cudaEventDestroy(h->ev_stop[i]);
  }
  if (h->side.fork) cudaEventDestroy(h->side.fork);
  if (h->side.join) cudaEventDestroy(h->side.join);
  if (h->side.enc_done) cudaEventDestroy(h->side.enc_done);
  if (h->side.stream) cudaStreamDestroy(h->side.stream);
  delete h;
  return SRN_OK;
}

srn_status srn_set_timing(srn_handle* h, int32_t target) {
  srn_status s = check_handle(h);
  if (s != SRN_OK) return s;
  if (target < SRN_TIME_OFF || target > SRN_TIME_SCATTER)
    return fail(SRN_ERR_INVALID_ARG, "srn_set_timing: unknown target %d", (int)target);
  if (target != SRN_TIME_OFF && h->ev_start.empty()) {
    const int n = 256;
    h->ev_start.resize(n);
    h->ev_stop.resize(n);
    h->ev_used.assign(n, 0);
    for (int i = 0; i < n; ++i) {
      cudaError_t e = cudaEventCreate(&h->ev_start[i]);
      if (e == cudaSuccess) e = cudaEventCreate(&h->ev_stop[i]);
      if (e != cudaSuccess) return cuda_fail(e, "event create");
    }
  }
  std::fill(h->ev_used.begin(), h->ev_used.end(), 0);
  h->ev_next = 0;
  h->timed_ms = 0.0;
  h->timed_launches = 0;
  h->timing = target;
  return SRN_OK;
}

srn_status srn_read_timing(srn_handle* h, double* total_ms, int64_t* launches) {
  srn_status s = check_handle(h);
  if (s != SRN_OK) return s;
  if (!total_ms || !launches) return fail(SRN_ERR_INVALID_ARG, "NULL output");
  for (size_t i = 0; i < h->ev_used.size(); ++i) {
    if (!h->ev_used[i]) continue;
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(h->ev_stop[i]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, h->ev_start[i], h->ev_stop[i]);
    if (e != cudaSuccess) return cuda_fail(e, "event read");
    h->timed_ms += ms;
    h->timed_launches += 1;
    h->ev_used[i] = 0;
  }
  *total_ms = h->timed_ms;
  *launches = h->timed_launches;
  h->timed_ms = 0.0;
  h->timed_launches = 0;
  return SRN_OK;
}

srn_status srn_sync_shadow(srn_handle* h, void* stream) {
  srn_status s = check_handle(h);
  if (s != SRN_OK) return s;
  if (h->cfg.precision != SRN_BF16) return SRN_OK;
  cudaError_t e = srn::launch_shadow(h->launch(stream), h->t.params_dev, h->t.shadow_dev, h->lay.n_group_a);
  return e == cudaSuccess ? SRN_OK : cuda_fail(e, "shadow kernel");
}

srn_status srn_sample_points(srn_handle* h, void* stream, uint64_t seed, uint64_t step,
                             const uint64_t* step_dev, const int64_t* offsets, float* xyz) {
  srn_status s = check_handle(h);
  if (s != SRN_OK) return s;
  srn::Bricks br;
  if ((s = make_bricks(h, offsets, &br)) != SRN_OK) return s;
  if (br.off[br.n] == 0) return SRN_OK;
  if (!xyz) return fail(SRN_ERR_INVALID_ARG, "xyz is NULL");
  cudaError_t e = srn::launch_sample(h->launch(stream), br, seed, step,
                                     reinterpret_cast<const unsigned long long*>(step_dev), xyz,
                                     reinterpret_cast<uint32_t*>(h->ws + h->wl.sort_rank),
                                     reinterpret_cast<uint32_t*>(h->ws + h->wl.sort_hist));
  return e == cudaSuccess ? SRN_OK : cuda_fail(e, "sampler");
}

srn_status srn_sample_target(srn_handle* h, void* stream, const float* vol, const int64_t dims[3],
                             const int64_t* boxes, const float* xyz, const int64_t* offsets,
                             float* target) {
  srn_status s = check_handle(h);
  if (s != SRN_OK) return s;
  srn::Bricks br;
  srn::VolumeBoxes vb;
  if ((s = make_bricks(h, offsets, &br)) != SRN_OK) return s;
  if ((s = make_boxes(h, dims, boxes, &vb)) != SRN_OK) return s;
  if (br.off[br.n] == 0) return SRN_OK;
  if (!vol || !xyz || !target) return fail(SRN_ERR_INVALID_ARG, "volume, xyz or target is NULL");
  cudaError_t e = srn::launch_target(h->launch(stream), br, vol, dims[0], dims[1], dims[2], vb, xyz, target, false);
  return e == cudaSuccess ? SRN_OK : cuda_fail(e, "target lookup");
}

srn_status srn_sample_target_tiled(srn_handle* h, void* stream, const float* tiled, const int64_t dims[3],
                                   const int64_t* boxes, const float* xyz, const int64_t* offsets, float* target) {
  srn_status s = check_handle(h);
  if (s != SRN_OK) return s;
  srn::Bricks br;
  srn::VolumeBoxes vb;
  if ((s = make_bricks(h, offsets, &br)) != SRN_OK) return s;
  if ((s = make_boxes(h, dims, boxes, &vb)) != SRN_OK) return s;
  if (br.off[br.n] == 0) return SRN_OK;
  if (!tiled || !xyz || !target) return fail(SRN_ERR_INVALID_ARG, "volume, xyz or target is NULL");
  cudaError_t e = srn::launch_target(h->launch(stream), br, tiled, dims[0], dims[1], dims[2], vb, xyz, target, true);
  return e == cudaSuccess ? SRN_OK : cuda_fail(e, "target lookup");
}

srn_status srn_tiled_volume_bytes(const int64_t dims[3], size_t* bytes) {
  if (!dims || !bytes) return fail(SRN_ERR_INVALID_ARG, "dims or bytes is NULL");
  for (int d = 0; d < 3; ++d)
    if (dims[d] < 2) return fail(SRN_ERR_INVALID_ARG, "volume dimension %d < 2", d);
  *bytes = sizeof(float) * (size_t)srn::tiled_volume_elems(dims[0], dims[1], dims[2]);
  return SRN_OK;
}

srn_status srn_tile_volume(void* stream, const float* vol, const int64_t dims[3], float* tiled) {
  size_t bytes = 0;
  srn_status s = srn_tiled_volume_bytes(dims, &bytes);
  if (s != SRN_OK) return s;
  if (!vol || !tiled) return fail(SRN_ERR_INVALID_ARG, "volume or tiled is NULL");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = srn::launch_tile_volume(srn::Launch{static_cast<cudaStream_t>(stream), sms}, vol, dims[0], dims[1], dims[2],
                                tiled);
  return e == cudaSuccess ? SRN_OK : cuda_fail(e, "volume tiling");
}

srn_status srn_forward(srn_handle* h, void* stream, const float* xyz, const int64_t* offsets, float* out) {
  srn_status s = check_handle(h);
  if (s != SRN_OK) return s;
  srn::Bricks br;
  if ((s = make_bricks(h, offsets, &br)) != SRN_OK) return s;
  if (br.off[br.n] == 0) return SRN_OK;  // nothing to query (empty tensors may have NULL data)
  if (!xyz || !out) return fail(SRN_ERR_INVALID_ARG, "xyz or out is NULL");
  return run_query(h, stream, srn::kForward, br, xyz, nullptr, out);
}

srn_status srn_backward(srn_handle* h, void* stream, const float* xyz, const float* target,
                        const int64_t* offsets, uint32_t flags, double* losses) {
  srn_status s = check_handle(h);
  if (s != SRN_OK) return s;
  srn::Bricks br;
  if ((s = make_bricks(h, offsets, &br)) != SRN_OK) return s;
  if ((s = check_training_counts(br)) != SRN_OK) return s;
  if (!xyz || !target) return fail(SRN_ERR_INVALID_ARG, "xyz or target is NULL");
  if (flags & ~(SRN_DENSITY | SRN_UPSTREAM | SRN_REC_DG)) return fail(SRN_ERR_INVALID_ARG, "unknown flags 0x%x", flags);
  if ((flags & SRN_DENSITY) && (flags & SRN_UPSTREAM))
    return fail(SRN_ERR_INVALID_ARG, "SRN_DENSITY needs the per-point error, which SRN_UPSTREAM lacks");
  return do_backward(h, stream, xyz, target, br, flags, losses);
}

srn_status srn_step(srn_handle* h, void* stream, uint32_t flags) {
  srn_status s = check_handle(h);
  if (s != SRN_OK) return s;
  if (flags & ~SRN_DENSITY) return fail(SRN_ERR_INVALID_ARG, "unknown flags 0x%x", flags);
  return do_step(h, stream, flags);
}

srn_status srn_train_step(srn_handle* h, void* stream, uint64_t seed, const float* vol,
                          const int64_t dims[3], const int64_t* boxes, const int64_t* offsets,
                          uint32_t flags, float* xyz, float* target, double* losses) {
  srn_status s = check_handle(h);
  if (s != SRN_OK) return s;
  srn::Bricks br;
  srn::VolumeBoxes vb;
  if ((s = make_bricks(h, offsets, &br)) != SRN_OK) return s;
  if ((s = check_training_counts(br)) != SRN_OK) return s;
  if ((s = make_boxes(h, dims, boxes, &vb)) != SRN_OK) return s;
  if (!vol || !xyz || !target) return fail(SRN_ERR_INVALID_ARG, "volume, xyz or target is NULL");
  if (flags & ~(SRN_DENSITY | SRN_SCHEDULE | SRN_VOLUME_TILED))
    return fail(SRN_ERR_INVALID_ARG, "unknown flags 0x%x", flags);
  if (flags & SRN_SCHEDULE) {
    if (!h->has_sched) return fail(SRN_ERR_STATE, "SRN_SCHEDULE before srn_set_schedule");
    if (!losses) return fail(SRN_ERR_INVALID_ARG, "SRN_SCHEDULE needs losses_dev");
  }
  if (stream == nullptr)
    return enqueue_train_step(h, stream, seed, vol, dims, vb, br, flags, xyz, target, losses);

  GraphKey key;
  key.flags = flags; key.seed = seed; key.vol = vol;
  for (int d = 0; d < 3; ++d) key.dims[d] = dims[d];
  key.boxes.assign(boxes, boxes + 6 * h->cfg.n_bricks);
  key.offsets.assign(offsets, offsets + h->cfg.n_bricks + 1);
  key.xyz = xyz; key.target = target; key.losses = losses;
  key.stream = static_cast<cudaStream_t>(stream);
  GraphEntry* ge = nullptr;
  for (auto& g : h->graphs)
    if (g.key == key) ge = &g;
  if (!ge) {
    h->graphs.push_back(GraphEntry{key, 0, nullptr});
    ge = &h->graphs.back();
  }
  if (!ge->exec) {
    if (ge->eager_runs == 0) {  // first call: run eagerly (sets kernel attributes outside capture)
      ge->eager_runs = 1;
      return enqueue_train_step(h, stream, seed, vol, dims, vb, br, flags, xyz, target, losses);
    }
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "begin capture");
    s = enqueue_train_step(h, stream, seed, vol, dims, vb, br, flags, xyz, target, losses);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cs, &graph);
    if (s != SRN_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&ge->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      ge->exec = nullptr;
      return cuda_fail(e, "graph instantiate");
    }
  }
  cudaError_t e = cudaGraphLaunch(ge->exec, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SRN_OK : cuda_fail(e, "graph launch");
}

namespace {
// Training state as srn_save_state writes it: this header, then the per-brick
// routine state [B] and the L_den history [B][2 kMaxDensityWindow].
struct StateBlob {
  uint32_t magic;      // 'SRNS'
  uint32_t version;
  int32_t n_bricks, n_grids;
  int32_t has_sched, pad;
  srn_schedule sched_cfg;
  srn::StepState st;
};
constexpr uint32_t kStateMagic = 0x534e5253u, kStateVersion = 2;
size_t sched_bytes(const srn_handle* h) { return sizeof(srn::BrickSched) * h->cfg.n_bricks; }
size_t ring_bytes(const srn_handle* h) { return sizeof(double) * 2 * srn::kMaxDensityWindow * h->cfg.n_bricks; }
}  // namespace

srn_status srn_state_bytes(srn_handle* h, size_t* bytes) {
  srn_status s = check_handle(h);
  if (s != SRN_OK) return s;
  if (!bytes) return fail(SRN_ERR_INVALID_ARG, "NULL argument");
  *bytes = sizeof(StateBlob) + sched_bytes(h) + ring_bytes(h);
  return SRN_OK;
}

srn_status srn_set_schedule(srn_handle* h, const srn_schedule* c) {
  srn_status s = check_handle(h);
  if (s != SRN_OK) return s;
  if (!c) return fail(SRN_ERR_INVALID_ARG, "NULL schedule");
  if (c->delay_iters < 0 || c->density_window < 1 || c->density_window > srn::kMaxDensityWindow ||
      c->total_iters < 1 || c->plateau_window < 1 || c->plateau_max < 1 || !(c->density_rel > 0.f) ||
      !(c->density_frac > 0.f && c->density_frac <= 1.f) || !(c->plateau_rel > 0.f) ||
      !(c->plateau_factor > 0.f && c->plateau_factor <= 1.f))
    return fail(SRN_ERR_INVALID_ARG, "bad training-routine setting");
  // every brick at iteration 0; the decision for iteration 1 as k_schedule would take it
  std::vector<srn::BrickSched> init(h->cfg.n_bricks);
  for (auto& q : init) {
    q = srn::BrickSched{};
    q.den_on = 1 > c->delay_iters && 1.0 <= (double)c->density_frac * (double)c->total_iters;
    q.bc1b = (float)(1.0 - h->cfg.beta1);
    q.rbc2b = (float)(1.0 / (1.0 - h->cfg.beta2));
  }
  cudaError_t e = cudaMemcpy(h->sched(), init.data(), sched_bytes(h), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(h->sring(), 0, ring_bytes(h));
  if (e != cudaSuccess) return cuda_fail(e, "schedule init");
  h->sched_cfg = *c;
  h->has_sched = true;
  return SRN_OK;
}

srn_status srn_read_schedule(srn_handle* h, void* stream, srn_brick_schedule* out) {
  srn_status s = check_handle(h);
  if (s != SRN_OK) return s;
  if (!out) return fail(SRN_ERR_INVALID_ARG, "NULL output");
  if (!h->has_sched) return fail(SRN_ERR_STATE, "no training routine set");
  std::vector<srn::BrickSched> q(h->cfg.n_bricks);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(q.data(), h->sched(), sched_bytes(h), cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) return cuda_fail(e, "schedule read");
  for (int b = 0; b < h->cfg.n_bricks; ++b) {
    srn_brick_schedule& o = out[b];
    o.iteration = q[b].it;
    o.plateaus = q[b].plateaus;
    float sc = 1.f;
    for (int k = 0; k < q[b].plateaus; ++k) sc *= h->sched_cfg.plateau_factor;
    o.lr_scale = sc;
    o.finished = q[b].finished;
    o.density_on = q[b].den_on;
    o.density_stopped = q[b].den_stopped;
    o.density_iters = q[b].den_n;
    o.best_rec = q[b].best;
  }
  return SRN_OK;
}

srn_status srn_rebalance(int32_t n_bricks, const int64_t* base, const srn_brick_schedule* state,
                         int64_t min_points, int64_t* out) {
  if (n_bricks < 1 || n_bricks > SRN_MAX_BRICKS)
    return fail(SRN_ERR_INVALID_ARG, "n_bricks %d outside [1, %d]", (int)n_bricks, SRN_MAX_BRICKS);
  if (!base || !state || !out) return fail(SRN_ERR_INVALID_ARG, "NULL argument");
  if (min_points < 1) return fail(SRN_ERR_INVALID_ARG, "min_points must be >= 1");
  const int64_t kCap = (int64_t)1 << 56;   // keeps every sum and product below 2^120
  int64_t total = 0, freed = 0, w = 0;
  int n_done = 0;
  for (int b = 0; b < n_bricks; ++b) {
    if (base[b] < 1 || base[b] > kCap) return fail(SRN_ERR_INVALID_ARG, "base count of brick %d out of range", b);
    total += base[b];
    if (total > kCap) return fail(SRN_ERR_INVALID_ARG, "base counts sum beyond 2^56");
    if (state[b].finished) {
      freed += base[b] - std::min(min_points, base[b]);
      ++n_done;
    } else {
      w += base[b];
    }
  }
  std::vector<int64_t> cnt(base, base + n_bricks);
  if (n_done > 0 && n_done < n_bricks) {
    std::vector<std::pair<int64_t, int>> rem;   // (remainder, brick) of the unfinished bricks
    int64_t given = 0;
    for (int b = 0; b < n_bricks; ++b) {
      if (state[b].finished) {
        cnt[b] = std::min(min_points, base[b]);
        continue;
      }
      const unsigned __int128 q = (unsigned __int128)freed * (unsigned __int128)base[b];
      const int64_t more = (int64_t)(q / (unsigned __int128)w);
      cnt[b] += more;
      given += more;
      rem.emplace_back((int64_t)(q % (unsigned __int128)w), b);
    }
    std::stable_sort(rem.begin(), rem.end(), [](const std::pair<int64_t, int>& x, const std::pair<int64_t, int>& y) {
      return x.first > y.first;
    });
    for (int64_t k = 0; k < freed - given; ++k) cnt[rem[(size_t)k].second] += 1;
  }
  out[0] = 0;
  for (int b = 0; b < n_bricks; ++b) out[b + 1] = out[b] + cnt[b];
  return SRN_OK;
}

srn_status srn_save_state(srn_handle* h, void* stream, void* dst, size_t bytes) {
  srn_status s = check_handle(h);
  if (s != SRN_OK) return s;
  if (!dst) return fail(SRN_ERR_INVALID_ARG, "NULL destination");
  if (bytes < sizeof(StateBlob)) return fail(SRN_ERR_INVALID_ARG, "state buffer of %zu bytes < %zu", bytes, sizeof(StateBlob));
  size_t need = 0;
  srn_state_bytes(h, &need);
  if (bytes < need) return fail(SRN_ERR_INVALID_ARG, "state buffer of %zu bytes < %zu", bytes, need);
  StateBlob b{};
  b.magic = kStateMagic;
  b.version = kStateVersion;
  b.n_bricks = h->cfg.n_bricks;
  b.n_grids = h->cfg.n_grids;
  b.has_sched = h->has_sched ? 1 : 0;
  b.sched_cfg = h->sched_cfg;
  unsigned char* out = static_cast<unsigned char*>(dst);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(&b.st, h->state(), sizeof(srn::StepState), cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out + sizeof b, h->sched(), sched_bytes(h), cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out + sizeof b + sched_bytes(h), h->sring(), ring_bytes(h), cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) return cuda_fail(e, "state read");
  std::memcpy(out, &b, sizeof b);
  return SRN_OK;
}

srn_status srn_load_state(srn_handle* h, void* stream, const void* src, size_t bytes) {
  srn_status s = check_handle(h);
  if (s != SRN_OK) return s;
  if (!src) return fail(SRN_ERR_INVALID_ARG, "NULL source");
  size_t need = 0;
  srn_state_bytes(h, &need);
  if (bytes < sizeof(StateBlob)) return fail(SRN_ERR_INVALID_ARG, "state buffer of %zu bytes < %zu", bytes, need);
  StateBlob b;
  std::memcpy(&b, src, sizeof b);
  if (b.magic != kStateMagic || b.version != kStateVersion) return fail(SRN_ERR_INVALID_ARG, "not a training state of this build");
  if (bytes < need) return fail(SRN_ERR_INVALID_ARG, "state buffer of %zu bytes < %zu", bytes, need);
  if (b.n_bricks != h->cfg.n_bricks || b.n_grids != h->cfg.n_grids)
    return fail(SRN_ERR_INVALID_ARG, "training state of %d bricks x %d grids, handle has %d x %d", b.n_bricks,
                b.n_grids, h->cfg.n_bricks, h->cfg.n_grids);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  const unsigned char* in = static_cast<const unsigned char*>(src);
  cudaError_t e = cudaMemcpyAsync(h->state(), &b.st, sizeof(srn::StepState), cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->sched(), in + sizeof b, sched_bytes(h), cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->sring(), in + sizeof b + sched_bytes(h), ring_bytes(h), cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) return cuda_fail(e, "state write");
  h->has_sched = b.has_sched != 0;
  h->sched_cfg = b.sched_cfg;
  return SRN_OK;
}

srn_status srn_decode(srn_handle* h, void* stream, const int32_t grid[3], const int64_t* boxes, int64_t vox,
                      float* out) {
  srn_status s = check_handle(h);
  if (s != SRN_OK) return s;
  if (!grid || !boxes || !out) return fail(SRN_ERR_INVALID_ARG, "NULL argument");
  if (grid[0] < 1 || grid[1] < 1 || grid[2] < 1 || grid[0] * grid[1] * grid[2] != h->cfg.n_bricks)
    return fail(SRN_ERR_INVALID_ARG, "brick grid does not match n_bricks");
  if (vox < 2) return fail(SRN_ERR_INVALID_ARG, "vox < 2");
  for (int b = 0; b < h->cfg.n_bricks; ++b)
    for (int a = 0; a < 3; ++a) {
      const int64_t lo = boxes[6 * b + a], hi = boxes[6 * b + 3 + a];
      if (lo < 0 || hi >= vox || hi <= lo) return fail(SRN_ERR_INVALID_ARG, "box of brick %d invalid", b);
    }
  // voxel i of an axis with I bricks belongs to brick min(floor(I i / (vox - 1)), I - 1):
  // brick k holds [ceil(k (vox - 1) / I), ceil((k + 1)(vox - 1) / I) - 1] (the last one up to vox - 1)
  auto first = [&](int k, int I) { return (int64_t)((k * (vox - 1) + I - 1) / I); };
  unsigned char* ws = h->ws;
  srn::RenderWs w{};
  w.xyz = reinterpret_cast<float*>(ws + h->wl.r_xyz);
  w.val = reinterpret_cast<float*>(ws + h->wl.r_val);
  const srn::Model md = h->model();
  const int64_t cap = h->max_points;
  for (int bz = 0; bz < grid[2]; ++bz)
    for (int by = 0; by < grid[1]; ++by)
      for (int bx = 0; bx < grid[0]; ++bx) {
        const int b = bx + grid[0] * (by + grid[1] * bz);
        const int bc[3] = {bx, by, bz};
        int64_t lo[3], n[3];
        for (int a = 0; a < 3; ++a) {
          lo[a] = first(bc[a], grid[a]);
          const int64_t hi = bc[a] == grid[a] - 1 ? vox - 1 : first(bc[a] + 1, grid[a]) - 1;
          n[a] = hi - lo[a] + 1;
        }
        srn::DecodeChunk c{};
        c.vox = vox;
        c.brick = b;
        c.n_bricks = h->cfg.n_bricks;
        for (int a = 0; a < 3; ++a) {
          c.lo[a] = (int32_t)boxes[6 * b + a];
          c.hi[a] = (int32_t)boxes[6 * b + 3 + a];
        }
        if (n[0] <= 0 || n[1] <= 0 || n[2] <= 0) continue;
        // chunks: whole planes if they fit, else whole rows, else parts of a row
        const int64_t plane = n[0] * n[1];
        const int64_t dz = plane <= cap ? std::max<int64_t>(1, cap / plane) : 1;
        const int64_t dy = plane <= cap ? n[1] : std::max<int64_t>(1, cap / n[0]);
        const int64_t dx = n[0] <= cap ? n[0] : cap;
        for (int64_t z = 0; z < n[2]; z += dz)
          for (int64_t y = 0; y < n[1]; y += dy)
            for (int64_t x = 0; x < n[0]; x += dx) {
              c.x0 = (int32_t)(lo[0] + x); c.nx = (int32_t)std::min(dx, n[0] - x);
              c.y0 = (int32_t)(lo[1] + y); c.ny = (int32_t)std::min(dy, n[1] - y);
              c.z0 = (int32_t)(lo[2] + z); c.nz = (int32_t)std::min(dz, n[2] - z);
              cudaError_t e = srn::launch_decode_chunk(h->launch(stream), c, w, md, out);
              if (e != cudaSuccess) return cuda_fail(e, "decode");
            }
      }
  return SRN_OK;
}

}  // extern "C"

namespace {

// Checks the arguments shared by the render entry points and fills rp.
srn_status render_params(srn_handle* h, const srn_camera* cam, const float* lut, float vmin, float vmax,
                         int32_t width, int32_t height, int32_t samples, const int32_t grid[3],
                         const int64_t* boxes, int64_t vox, float* rgba, srn::RenderParams& rp) {
  srn_status s = check_handle(h);
  if (s != SRN_OK) return s;
  if (!cam || !lut || !grid || !boxes || !rgba) return fail(SRN_ERR_INVALID_ARG, "NULL argument");
  if (width < 1 || height < 1 || samples < 1) return fail(SRN_ERR_INVALID_ARG, "empty image or no samples");
  if ((int64_t)width * height > INT32_MAX) return fail(SRN_ERR_INVALID_ARG, "image of 2^31 pixels or more");
  if ((int64_t)samples > h->max_points)
    return fail(SRN_ERR_INVALID_ARG, "samples per ray %d exceed max_points", samples);
  if (!(vmax > vmin)) return fail(SRN_ERR_INVALID_ARG, "vmax must exceed vmin");
  if (grid[0] < 1 || grid[1] < 1 || grid[2] < 1 || grid[0] * grid[1] * grid[2] != h->cfg.n_bricks)
    return fail(SRN_ERR_INVALID_ARG, "brick grid does not match n_bricks");
  if (vox < 2) return fail(SRN_ERR_INVALID_ARG, "vox < 2");
  rp = srn::RenderParams{};
  rp.cam = *cam;
  rp.width = width; rp.height = height; rp.samples = samples;
  rp.order = 0;
  rp.levels = 0;
  // bundles of 8 rays x 16 samples when a batch holds at least one bundle of whole rays
  const bool bundle = 8 * (((int64_t)samples + 15) / 16 * 16) <= h->max_points;
  rp.rg = bundle ? 8 : 1;
  rp.jb = bundle ? 16 : 1;
  while ((1 << rp.levels) < std::max(width, height)) ++rp.levels;
  for (int a = 0; a < 3; ++a) rp.grid[a] = grid[a];
  rp.vox = vox; rp.vmin = vmin; rp.vmax = vmax;
  for (int b = 0; b < h->cfg.n_bricks; ++b)
    for (int a = 0; a < 3; ++a) {
      const int64_t lo = boxes[6 * b + a], hi = boxes[6 * b + 3 + a];
      if (lo < 0 || hi >= vox || hi <= lo) return fail(SRN_ERR_INVALID_ARG, "box of brick %d invalid", b);
      rp.lo[b][a] = (int32_t)lo; rp.hi[b][a] = (int32_t)hi;
    }
  return SRN_OK;
}

// Renders the pixels first .. first + count - 1 of rp's order in batches of at most
// max_points samples.
srn_status render_pixels(srn_handle* h, void* stream, const srn::RenderParams& rp, const float* lut,
                         int64_t first, int64_t count, float* rgba) {
  unsigned char* ws = h->ws;
  srn::RenderWs w;
  w.loc = reinterpret_cast<float*>(ws + h->wl.r_loc);
  w.rank = reinterpret_cast<uint32_t*>(ws + h->wl.r_rank);
  w.bid = reinterpret_cast<uint32_t*>(ws + h->wl.r_bid);
  w.pos = reinterpret_cast<uint32_t*>(ws + h->wl.r_pos);
  w.xyz = reinterpret_cast<float*>(ws + h->wl.r_xyz);
  w.val = reinterpret_cast<float*>(ws + h->wl.r_val);
  w.cnt = reinterpret_cast<uint32_t*>(ws + h->wl.r_cnt);
  w.off = reinterpret_cast<int64_t*>(ws + h->wl.r_off);
  // whole ray groups whose slots fit the workspace's max_points samples
  const int64_t spr = ((int64_t)rp.samples + rp.jb - 1) / rp.jb * rp.jb;
  const int64_t batch = h->max_points / spr / rp.rg * rp.rg;
  const srn::Model md = h->model();
  for (int64_t p0 = first; p0 < first + count; p0 += batch) {
    const int n = (int)std::min<int64_t>(batch, first + count - p0);
    cudaError_t e = srn::launch_render_batch(h->launch(stream), rp, w, (int)p0, n, md, lut, rgba);
    if (e != cudaSuccess) return cuda_fail(e, "render");
  }
  return SRN_OK;
}

}  // namespace

extern "C" {

srn_status srn_render(srn_handle* h, void* stream, const srn_camera* cam, const float* lut,
                      float vmin, float vmax, int32_t width, int32_t height, int32_t samples,
                      const int32_t grid[3], const int64_t* boxes, int64_t vox, float* rgba) {
  srn::RenderParams rp;
  srn_status s = render_params(h, cam, lut, vmin, vmax, width, height, samples, grid, boxes, vox, rgba, rp);
  if (s != SRN_OK) return s;
  return render_pixels(h, stream, rp, lut, 0, (int64_t)width * height, rgba);
}

srn_status srn_render_progressive(srn_handle* h, void* stream, const srn_camera* cam, const float* lut,
                                  float vmin, float vmax, int32_t width, int32_t height, int32_t samples,
                                  const int32_t grid[3], const int64_t* boxes, int64_t vox, int64_t first,
                                  int64_t count, float* rgba, float* preview) {
  srn::RenderParams rp;
  srn_status s = render_params(h, cam, lut, vmin, vmax, width, height, samples, grid, boxes, vox, rgba, rp);
  if (s != SRN_OK) return s;
  const int64_t npix = (int64_t)width * height;
  if (first < 0 || count < 0 || first + count > npix)
    return fail(SRN_ERR_INVALID_ARG, "pixels [%lld, %lld) outside the image of %lld", (long long)first,
                (long long)(first + count), (long long)npix);
  if (preview == rgba) return fail(SRN_ERR_INVALID_ARG, "preview_dev must not be rgba_dev");
  rp.order = 1;
  if ((s = render_pixels(h, stream, rp, lut, first, count, rgba)) != SRN_OK) return s;
  if (preview) {
    const int64_t done = first + count;
    int level = rp.levels;   // the finest level whose whole grid is among the first `done` pixels
    while (level > 0) {
      const int64_t nx = (width + (1 << (level - 1)) - 1) >> (level - 1), ny = (height + (1 << (level - 1)) - 1) >> (level - 1);
      if (nx * ny > done) break;
      --level;
    }
    cudaError_t e = srn::launch_render_preview(h->launch(stream), rp, (int)done, level, rgba, preview);
    if (e != cudaSuccess) return cuda_fail(e, "render preview");
  }
  return SRN_OK;
}

namespace {

srn_status check_tuning(const srn_tuning* t) {
  if (!t) return fail(SRN_ERR_INVALID_ARG, "tuning is NULL");
  if (t->tile_points < srn::kMinTilePoints || t->tile_points > srn::kMaxTilePoints || t->tile_points % 32)
    return fail(SRN_ERR_INVALID_ARG, "tile_points %d is not a multiple of 32 in [%d, %d]", (int)t->tile_points,
                srn::kMinTilePoints, srn::kMaxTilePoints);
  if (t->tile_level < 0 || t->tile_level > srn::kMaxTileLevel)
    return fail(SRN_ERR_INVALID_ARG, "tile_level %d outside [0, %d]", (int)t->tile_level, srn::kMaxTileLevel);
  if (t->density_ctas < 1 || t->density_ctas > srn::kMaxDensityCtas)
    return fail(SRN_ERR_INVALID_ARG, "density_ctas %d outside [1, %d]", (int)t->density_ctas,
                srn::kMaxDensityCtas);
  return SRN_OK;
}

// Installs a tuning; the CUDA graphs of srn_train_step hold launches with the old one.
void install_tuning(srn_handle* h, const srn::Tuning& t) {
  const srn::Tuning& o = h->tune;
  if (t.tile_points == o.tile_points && t.tile_level == o.tile_level && t.density_ctas == o.density_ctas) return;
  for (auto& g : h->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
  h->tune = t;
}

// Median time in milliseconds of `reps` backward passes under the handle's tuning,
// after one untimed pass (which also sets the kernels' shared-memory attributes).
srn_status time_backward(srn_handle* h, void* stream, const float* xyz, const float* target,
                         const srn::Bricks& br, uint32_t flags, int reps, cudaEvent_t t0, cudaEvent_t t1,
                         float* median) {
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  srn_status st = do_backward(h, stream, xyz, target, br, flags, nullptr);
  std::vector<float> ms((size_t)reps, 0.f);
  for (int r = 0; r < reps && st == SRN_OK; ++r) {
    cudaError_t e = cudaEventRecord(t0, cs);
    if (e != cudaSuccess) return cuda_fail(e, "autotune event");
    if ((st = do_backward(h, stream, xyz, target, br, flags, nullptr)) != SRN_OK) break;
    e = cudaEventRecord(t1, cs);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[(size_t)r], t0, t1);
    if (e != cudaSuccess) return cuda_fail(e, "autotune timing");
  }
  if (st != SRN_OK) return st;
  std::sort(ms.begin(), ms.end());
  const size_t m = (size_t)reps / 2;
  *median = reps % 2 ? ms[m] : 0.5f * (ms[m - 1] + ms[m]);
  return SRN_OK;
}

}  // namespace

srn_status srn_get_tuning(srn_handle* h, srn_tuning* out) {
  srn_status s = check_handle(h);
  if (s != SRN_OK) return s;
  if (!out) return fail(SRN_ERR_INVALID_ARG, "NULL output");
  out->tile_points = h->tune.tile_points;
  out->tile_level = h->tune.tile_level;
  out->density_ctas = h->tune.density_ctas;
  return SRN_OK;
}

srn_status srn_set_tuning(srn_handle* h, const srn_tuning* t) {
  srn_status s = check_handle(h);
  if (s != SRN_OK) return s;
  if ((s = check_tuning(t)) != SRN_OK) return s;
  install_tuning(h, srn::Tuning{t->tile_points, t->tile_level, t->density_ctas});
  return SRN_OK;
}

namespace {
// Reads the device status word into *v and clears it (synchronises the stream).
srn_status take_status(srn_handle* h, cudaStream_t cs, int32_t* v) {
  *v = 0;
  cudaError_t e = cudaMemcpyAsync(v, h->status(), sizeof *v, cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e == cudaSuccess && *v) e = cudaMemsetAsync(h->status(), 0, sizeof *v, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  return e == cudaSuccess ? SRN_OK : cuda_fail(e, "status read");
}
}  // namespace

srn_status srn_autotune(srn_handle* h, void* stream, const float* xyz, const float* target,
                        const int64_t* offsets, uint32_t flags, int32_t reps, srn_tuning* out) {
  srn_status s = check_handle(h);
  if (s != SRN_OK) return s;
  if (h->cfg.precision != SRN_BF16) return fail(SRN_ERR_UNSUPPORTED, "srn_autotune: the FP32 pass has no tiles");
  if (reps < 1 || reps > 100) return fail(SRN_ERR_INVALID_ARG, "srn_autotune: reps %d outside [1, 100]", (int)reps);
  srn::Bricks br;
  if ((s = make_bricks(h, offsets, &br)) != SRN_OK) return s;
  if ((s = check_training_counts(br)) != SRN_OK) return s;
  if (!xyz || !target) return fail(SRN_ERR_INVALID_ARG, "xyz or target is NULL");
  if (flags & ~(SRN_DENSITY | SRN_UPSTREAM | SRN_REC_DG)) return fail(SRN_ERR_INVALID_ARG, "unknown flags 0x%x", flags);
  if ((flags & SRN_DENSITY) && (flags & SRN_UPSTREAM))
    return fail(SRN_ERR_INVALID_ARG, "SRN_DENSITY needs the per-point error, which SRN_UPSTREAM lacks");
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(cs, &cap);
  if (e != cudaSuccess) return cuda_fail(e, "capture status");
  if (cap != cudaStreamCaptureStatusNone) return fail(SRN_ERR_STATE, "srn_autotune: the stream is being captured");
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  if (e != cudaSuccess) {
    if (t0) cudaEventDestroy(t0);
    return cuda_fail(e, "event create");
  }
  // candidates: tile sizes, and level caps from small blocks (small boxes, more tiles)
  // up to the largest (where the shared-memory bound on the boxes decides)
  static const int kPoints[] = {256, 512, 768, 1024};
  static const int kLevels[] = {2, 3, 4, 6, 9};
  const int32_t timing = h->timing;   // the search is not reported by the measurement hook
  h->timing = SRN_TIME_OFF;
  const srn::Tuning start = h->tune;
  srn::Tuning best = start;
  float best_ms = 0.f;
  // A pass whose decoder gave up on a tensor-core wait returns early and would look
  // fast: the status word is read (and cleared) after every timed shape, and a shape
  // that set the timeout bit is dropped.  Bits set before the call are put back.
  int32_t pre = 0, st = 0;
  s = take_status(h, cs, &pre);
  if (s == SRN_OK) s = time_backward(h, stream, xyz, target, br, flags, reps, t0, t1, &best_ms);
  if (s == SRN_OK) s = take_status(h, cs, &st);
  pre |= st & 1;
  if (s == SRN_OK && (st & 2))
    s = fail(SRN_ERR_DEVICE_TIMEOUT, "srn_autotune: the current tile shape gave up waiting for the tensor cores");
  for (int tp : kPoints) {
    for (int lv : kLevels) {
      if (s != SRN_OK || (tp == start.tile_points && lv == start.tile_level)) continue;
      h->tune = srn::Tuning{tp, lv, start.density_ctas};
      float ms = 0.f;
      if ((s = time_backward(h, stream, xyz, target, br, flags, reps, t0, t1, &ms)) != SRN_OK) break;
      if ((s = take_status(h, cs, &st)) != SRN_OK) break;
      pre |= st & 1;
      if (st & 2) continue;   // gave up: not a candidate
      if (ms < 0.99f * best_ms) {
        best = h->tune;
        best_ms = ms;
      }
    }
  }
  h->tune = start;
  h->timing = timing;
  if (pre && (e = cudaMemcpyAsync(h->status(), &pre, sizeof pre, cudaMemcpyHostToDevice, cs)) == cudaSuccess)
    e = cudaStreamSynchronize(cs);
  if (pre && e != cudaSuccess && s == SRN_OK) s = cuda_fail(e, "status restore");
  if (s == SRN_OK) {
    install_tuning(h, best);
    s = do_backward(h, stream, xyz, target, br, flags, nullptr);
  }
  if (s == SRN_OK && (e = cudaStreamSynchronize(cs)) != cudaSuccess) s = cuda_fail(e, "autotune sync");
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (s == SRN_OK && out) {
    out->tile_points = best.tile_points;
    out->tile_level = best.tile_level;
    out->density_ctas = best.density_ctas;
  }
  return s;
}

srn_status srn_get_status(srn_handle* h, void* stream) {
  srn_status s = check_handle(h);
  if (s != SRN_OK) return s;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  int32_t v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, h->status(), sizeof v, cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e == cudaSuccess && v) e = cudaMemsetAsync(h->status(), 0, sizeof v, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  if (v & 2) return fail(SRN_ERR_DEVICE_TIMEOUT, "a kernel gave up waiting for the tensor cores");
  if (v & 1) return fail(SRN_ERR_NONFINITE, "a loss was NaN or Inf");
  return SRN_OK;
}

}  // extern "C"
