// srn_sample_points_static: the batch sampler for callers that cannot allocate device
// memory.  It runs the same kernels as srn_sample_points (Philox4x32-10 draws, then a
// counting sort of each brick's points by 32^3 Morton bin), but its scratch -- each
// point's rank in its bin and the bin histograms -- lives in one file-scope __device__
// array instead of a caller-allocated workspace.
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int64_t kMaxPoints = SRN_STATIC_SAMPLER_MAX_POINTS;
constexpr int kMaxBricks = SRN_STATIC_SAMPLER_MAX_BRICKS;
constexpr size_t kRankBytes = sizeof(uint32_t) * kMaxPoints;
constexpr size_t kHistBytes = sizeof(uint32_t) * srn::kSortBins * kMaxBricks;

// One copy per device that loads the library, held until the process exits.
static __device__ __align__(256) unsigned char g_sampler_scratch[kRankBytes + kHistBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of this device's copy of the array (looked up once per device, with
// that device current; host code cannot use the array's name as a device address).
// The address is that of the runtime's primary context and is never looked up again:
// it does not follow a caller's own driver-API context, nor a cudaDeviceReset.
srn_status scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return srn::report(SRN_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return srn::report(SRN_ERR_UNSUPPORTED, "device index beyond 63");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sampler_scratch);
    if (e != cudaSuccess) return srn::report(SRN_ERR_CUDA, cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return SRN_OK;
}

}  // namespace

extern "C" srn_status srn_sample_points_static(void* stream, uint64_t seed, uint64_t step, int32_t n_bricks,
                                               const int64_t* offsets, float* xyz_dev) {
  if (n_bricks < 1 || n_bricks > kMaxBricks)
    return srn::report(SRN_ERR_INVALID_ARG, "srn_sample_points_static: n_bricks must be in [1, 8]");
  if (!offsets) return srn::report(SRN_ERR_INVALID_ARG, "srn_sample_points_static: offsets is NULL");
  if (offsets[0] != 0) return srn::report(SRN_ERR_INVALID_ARG, "srn_sample_points_static: offsets[0] must be 0");
  srn::Bricks br{};
  br.n = n_bricks;
  br.dev = nullptr;
  for (int b = 0; b <= n_bricks; ++b) {
    if (b > 0 && offsets[b] < offsets[b - 1])
      return srn::report(SRN_ERR_INVALID_ARG, "srn_sample_points_static: offsets decrease");
    br.off[b] = offsets[b];
  }
  if (br.off[n_bricks] > kMaxPoints)
    return srn::report(SRN_ERR_INVALID_ARG,
                       "srn_sample_points_static: more than SRN_STATIC_SAMPLER_MAX_POINTS (131072) points");
  if (br.off[n_bricks] == 0) return SRN_OK;
  if (!xyz_dev) return srn::report(SRN_ERR_INVALID_ARG, "srn_sample_points_static: xyz_dev is NULL");
  unsigned char* scratch = nullptr;
  srn_status st = scratch_for_current_device(&scratch);
  if (st != SRN_OK) return st;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return srn::report(SRN_ERR_CUDA, cudaGetErrorString(e));
  const srn::Launch L{static_cast<cudaStream_t>(stream), sms};
  // launch_sample clears the histograms (the only scratch that must start at zero)
  // with cudaMemsetAsync before drawing; the ranks are fully overwritten.
  e = srn::launch_sample(L, br, seed, step, nullptr, xyz_dev, reinterpret_cast<uint32_t*>(scratch),
                         reinterpret_cast<uint32_t*>(scratch + kRankBytes));
  if (e != cudaSuccess) return srn::report(SRN_ERR_CUDA, cudaGetErrorString(e));
  return SRN_OK;
}
