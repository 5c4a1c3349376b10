// fms_mean_shift_step_noalloc: one mean-shift update without any allocation.
//
// Who needs this: code that may not allocate device memory while it runs --
// for example a caller inside a real-time loop or an allocator-free runtime
// that forbids cudaMalloc/cudaFree (they synchronise the device and can stall
// other streams), or an embedding that has no memory pool to lend us.  Such a
// caller cannot provide the scratch that fms_mean_shift_step needs, so this
// entry point takes its scratch from a fixed array that is part of the
// library image instead.
//
// The array below is a static __device__ buffer: every GPU that loads the
// library reserves FMS_NOALLOC_SCRATCH_BYTES for it until the process exits.
// In host code its name only stands for the buffer; the device address that
// kernels need is fetched once per device with cudaGetSymbolAddress, with that
// device current, on the first call made on that device.
#include <math.h>

#include <mutex>

#include "../../include/fms.h"
#include "fms_internal.cuh"

using namespace fms;

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FMS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

int padded_dim_of(int d) {
  if (d <= 4) return 4;
  if (d <= 8) return 8;
  return (d + 3) / 4 * 4;
}

}  // namespace

extern "C" fms_status fms_mean_shift_step_noalloc(const float* points, int64_t n, int32_t d,
                                                  float h, const float* seeds, int64_t m,
                                                  float* out_seeds, float* out_wsum,
                                                  void* stream_) {
  if (!points || !seeds || !out_seeds || n < 1 || n > INT32_MAX || d < 1 || d > FMS_MAX_DIM ||
      m < 1 || m > INT32_MAX || !(h > 0.0f) || !isfinite(h))
    return FMS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream_);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return FMS_ERR_CUDA;

  // the same scratch layout the workspace form uses: packed points, packed
  // seeds, active list, per-chunk partial sums, control block, status word
  const int DP = padded_dim_of(d);
  const int DA = step_accumulators(d);
  const int R = step_seeds_per_warp(d);
  Tiling tl{sms * step_resident_warps_per_sm(d), step_min_chunk(d)};
  int32_t C = 0, Lc = 0;
  choose_chunks(n, (int32_t)m, R, tl, &C, &Lc);
  const size_t off_Xs = 0;
  const size_t off_Ys = off_Xs + round256((size_t)n * DP * 4);
  const size_t off_active = off_Ys + round256((size_t)m * DP * 4);
  const size_t off_part = off_active + round256((size_t)m * 4);
  const size_t off_ctl = off_part + round256((size_t)C * (size_t)m * DA * 4);
  const size_t off_status = off_ctl + round256(sizeof(IterCtl));
  const size_t total = off_status + 256;
  if (total > (size_t)FMS_NOALLOC_SCRATCH_BYTES) return FMS_ERR_WORKSPACE;

  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return FMS_ERR_CUDA;
  char* b = static_cast<char*>(base);
  float* Xs = reinterpret_cast<float*>(b + off_Xs);
  float* Ys = reinterpret_cast<float*>(b + off_Ys);
  int32_t* active = reinterpret_cast<int32_t*>(b + off_active);
  float* part = reinterpret_cast<float*>(b + off_part);
  IterCtl* ctl = reinterpret_cast<IterCtl*>(b + off_ctl);
  uint32_t* status = reinterpret_cast<uint32_t*>(b + off_status);

  const double scale = sqrt(1.4426950408889634 / (2.0 * (double)h * (double)h));
  // the status word is OR-ed into by the packing kernel: it must start at zero
  // (every other region is fully written before it is read)
  if (cudaMemsetAsync(status, 0, 4, st) != cudaSuccess) return FMS_ERR_CUDA;
  if (launch_pack_points(points, n, d, DP, (float)scale, Xs, status, st) != cudaSuccess ||
      launch_pack_points(seeds, m, d, DP, (float)scale, Ys, status, st) != cudaSuccess ||
      launch_step_setup(active, (int32_t)m, ctl, C, Lc, st) != cudaSuccess ||
      launch_ms_step(Xs, n, d, DP, Ys, active, &ctl->s, &ctl->C, &ctl->Lc, part,
                     ((tl.target_warps + 7) / 8) * 8, st, nullptr) != cudaSuccess ||
      launch_step_finish(part, ctl, seeds, d, DA, 1.0 / scale, out_seeds, out_wsum, (int)m,
                         st) != cudaSuccess)
    return FMS_ERR_CUDA;
  return FMS_OK;
}
