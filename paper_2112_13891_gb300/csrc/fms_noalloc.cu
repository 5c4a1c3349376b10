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
// kernels need is looked up with cudaGetSymbolAddress, with the calling device
// current, on every call.  The lookup enqueues no work, and looking it up each
// time (instead of caching it per device) keeps the call correct after the
// device's context has been reset or recreated, when the array may have moved.
#include <math.h>

#include "../../include/fms.h"
#include "fms_internal.cuh"

using namespace fms;

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FMS_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array in the current device's context.
cudaError_t scratch_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = p;
  return cudaSuccess;
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

  // the same scratch layout the workspace form uses (step_layout): packed
  // points, packed seeds, active list, per-chunk partial sums, control block,
  // status word
  const StepLayout L = step_layout(n, d, m, sms);
  if (L.total > (size_t)FMS_NOALLOC_SCRATCH_BYTES) return FMS_ERR_WORKSPACE;

  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return FMS_ERR_CUDA;
  char* b = static_cast<char*>(base);
  float* Xs = reinterpret_cast<float*>(b + L.off_Xs);
  float* Ys = reinterpret_cast<float*>(b + L.off_Ys);
  int32_t* active = reinterpret_cast<int32_t*>(b + L.off_active);
  float* part = reinterpret_cast<float*>(b + L.off_part);
  IterCtl* ctl = reinterpret_cast<IterCtl*>(b + L.off_ctl);
  uint32_t* status = reinterpret_cast<uint32_t*>(b + L.off_status);

  const double scale = sqrt(1.4426950408889634 / (2.0 * (double)h * (double)h));
  // the status word is OR-ed into by the packing kernel: it must start at zero
  // (every other region is fully written before it is read)
  if (cudaMemsetAsync(status, 0, 4, st) != cudaSuccess) return FMS_ERR_CUDA;
  if (launch_pack_points(points, n, d, L.DP, (float)scale, Xs, status, st) != cudaSuccess ||
      launch_pack_points(seeds, m, d, L.DP, (float)scale, Ys, status, st) != cudaSuccess ||
      launch_step_setup(active, (int32_t)m, ctl, L.C, L.Lc, st) != cudaSuccess ||
      launch_ms_step(Xs, n, d, L.DP, Ys, active, &ctl->s, &ctl->C, &ctl->Lc, part,
                     L.grid_ctas * 8, st, nullptr, nullptr, kKernelGaussian, status) != cudaSuccess ||
      launch_step_finish(part, ctl, seeds, d, L.DA, 1.0 / scale, out_seeds, out_wsum, (int)m,
                         st) != cudaSuccess)
    return FMS_ERR_CUDA;
  return FMS_OK;
}
