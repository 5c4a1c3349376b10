// Pipe-rate probes: the FP32 and SFU throughputs that the roofline of the
// evaluation kernels divides by, measured on the device in use.
//
// One CTA of 1024 threads per SM runs a fixed instruction mix with many
// independent dependency chains per thread; the SM cycle counter (clock64)
// brackets the loop, so the rates come out per clock and per SM and do not
// depend on the SM clock of the moment.  The median over SMs is reported.
//   rate[0]  FFMA:          FP32 operations per clock per SM
//   rate[1]  FFMA2 (f32x2): FP32 operations per clock per SM
//   rate[2]  MUFU.EX2:      exp2 per clock per SM
//   rate[3]  10 FFMA + 1 EX2 per unit (the exact-difference evaluation's
//            FP32 : exp2 ratio at d = 3): units per clock per SM
// and the 5th-generation tensor cores' BF16 rate (fms_probe_tensor_rates): one
// thread per SM issues back-to-back tcgen05.mma.kind::f16 (M = 128, K = 16,
// N = 16 .. 256, operands in shared memory, FP32 accumulator in tensor
// memory); the clock runs from the first issue until the MMAs' commit
// arrives on an mbarrier (bounded wait), so the rate counts completed work.
#include <algorithm>
#include <vector>

#include "../../include/fms.h"
#include "fms_internal.cuh"
#include "fms_tc.cuh"

namespace fms {
namespace {

constexpr int kProbeThreads = 1024;
constexpr int kProbeIters = 1024;

template <int MODE>
__global__ void __launch_bounds__(kProbeThreads, 1)
    pipe_probe_kernel(float a, float* __restrict__ sink, long long* __restrict__ cycles) {
  float x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = (float)threadIdx.x * 1e-3f + (float)i;
  float2 p[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) p[i] = make_float2(x[2 * i], x[2 * i + 1]);
  const float2 a2 = make_float2(a, a), b2 = make_float2(0.5f, 0.5f);
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      if constexpr (MODE == 0) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, 0.5f);
      } else if constexpr (MODE == 1) {
#pragma unroll
        for (int i = 0; i < 4; ++i) p[i] = __ffma2_rn(p[i], a2, b2);
      } else if constexpr (MODE == 2) {
        // x <- 2^-x stays in (0, 1]
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = ex2_ftz(-x[i]);
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          float t = x[i];
#pragma unroll
          for (int k = 0; k < 10; ++k) t = fmaf(t, a, 0.5f);
          x[i] = ex2_ftz(-t);
        }
      }
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
#pragma unroll
  for (int i = 0; i < 4; ++i) s += p[i].x + p[i].y;
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int MODE>
cudaError_t run_probe(int sms, float* sink, long long* cyc, std::vector<long long>& host) {
  // the second launch is the measured one (the first pays instruction-cache and clock ramp)
  for (int rep = 0; rep < 2; ++rep) {
    pipe_probe_kernel<MODE><<<sms, kProbeThreads>>>(0.999f, sink, cyc);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return e;
  return cudaMemcpy(host.data(), cyc, sizeof(long long) * sms, cudaMemcpyDeviceToHost);
}

// ---- tensor-core rate ----
constexpr int kTcProbeIters = 4096;
// dynamic shared memory requested only so that one CTA fits per SM (every CTA
// allocates all 512 tensor-memory columns)
constexpr int kTcProbeSmem = 160 * 1024;

template <int N>
__global__ void __launch_bounds__(128, 1)
    tc_rate_probe(long long* __restrict__ cycles, int n_issuers) {
  __shared__ __align__(1024) unsigned char sA[128 * 16 * 2];   // A: 128 x 16 BF16
  __shared__ __align__(1024) unsigned char sB[256 * 16 * 2];   // B: N x 16 BF16
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int e = tid; e < (int)sizeof(sA) / 4; e += blockDim.x) reinterpret_cast<uint32_t*>(sA)[e] = 0u;
  for (int e = tid; e < (int)sizeof(sB) / 4; e += blockDim.x) reinterpret_cast<uint32_t*>(sB)[e] = 0u;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc::su32(&tmem_base)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < 2; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::su32(&bar[i])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  // issuer q (lane 0 of warp q) accumulates into its own 256 columns
  const bool issuer = (tid & 31) == 0 && warp < n_issuers;
  long long t = -1;
  if (issuer) {
    const uint32_t dt = tmem_base + (uint32_t)warp * 256u;
    const uint32_t id = tc::idesc_bf16(128, N);
    const uint64_t da = tc::sdesc(tc::su32(sA), 128, 256);
    const uint64_t db = tc::sdesc(tc::su32(sB), 128, 256);
    const long long t0 = clock64();
    for (int i = 0; i < kTcProbeIters; ++i) tc::mma(dt, da, db, id, i > 0 ? 1u : 0u);
    tc::commit(&bar[warp]);
    const bool ok = tc::wait_bar(&bar[warp], 0);
    t = ok ? clock64() - t0 : -1;
    if (!ok) tc::wait_bar(&bar[warp], 0);   // once more before the columns are freed
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (issuer && warp == 0) cycles[blockIdx.x] = t;
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(512)
                 : "memory");
}

template <int N>
cudaError_t run_tc_probe(int sms, int issuers, long long* cyc, std::vector<long long>& host) {
  const cudaError_t ea = cudaFuncSetAttribute(
      tc_rate_probe<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcProbeSmem);
  if (ea != cudaSuccess) return ea;
  for (int rep = 0; rep < 2; ++rep) {
    tc_rate_probe<N><<<sms, 128, kTcProbeSmem>>>(cyc, issuers);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return e;
  return cudaMemcpy(host.data(), cyc, sizeof(long long) * sms, cudaMemcpyDeviceToHost);
}

}  // namespace
}  // namespace fms

using namespace fms;

extern "C" fms_status fms_probe_pipe_rates(double* rates, int32_t n_rates) {
  if (!rates || n_rates < 1) return FMS_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return FMS_ERR_CUDA;
  float* sink = nullptr;
  long long* cyc = nullptr;
  if (cudaMalloc(&sink, sizeof(float) * (size_t)sms * kProbeThreads) != cudaSuccess)
    return FMS_ERR_CUDA;
  if (cudaMalloc(&cyc, sizeof(long long) * (size_t)sms) != cudaSuccess) {
    cudaFree(sink);
    return FMS_ERR_CUDA;
  }
  std::vector<long long> host((size_t)sms);
  // per CTA: kProbeThreads threads x kProbeIters x 16 x (8 FFMA | 4 FFMA2 = 8 pairs | 8 EX2 | 8 units)
  const double per_cta = (double)kProbeThreads * kProbeIters * 16 * 8;
  const double ops[4] = {per_cta, per_cta, per_cta, per_cta};
  fms_status rc = FMS_OK;
  for (int m = 0; m < 4 && m < n_rates; ++m) {
    cudaError_t e = cudaSuccess;
    switch (m) {
      case 0: e = run_probe<0>(sms, sink, cyc, host); break;
      case 1: e = run_probe<1>(sms, sink, cyc, host); break;
      case 2: e = run_probe<2>(sms, sink, cyc, host); break;
      case 3: e = run_probe<3>(sms, sink, cyc, host); break;
    }
    if (e != cudaSuccess) {
      rc = FMS_ERR_CUDA;
      break;
    }
    std::vector<long long> v = host;
    std::sort(v.begin(), v.end());
    const double med = (double)v[v.size() / 2];
    rates[m] = med > 0 ? ops[m] / med : 0.0;
  }
  cudaFree(sink);
  cudaFree(cyc);
  return rc;
}

// rates[2 i] (one issuing thread) and rates[2 i + 1] (two issuing threads in
// different warps, each with its own accumulator): BF16 FLOP per clock per SM
// (2 * 128 * N * 16 per MMA, completed work) for N = 16, 32, 64, 128, 256
// (i = 0 .. 4); the median over SMs.  A negative entry: a wait gave up.
extern "C" fms_status fms_probe_tensor_rates(double* rates, int32_t n_rates) {
  if (!rates || n_rates < 1) return FMS_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return FMS_ERR_CUDA;
  long long* cyc = nullptr;
  if (cudaMalloc(&cyc, sizeof(long long) * (size_t)sms) != cudaSuccess) return FMS_ERR_CUDA;
  std::vector<long long> host((size_t)sms);
  const int Ns[5] = {16, 32, 64, 128, 256};
  fms_status rc = FMS_OK;
  for (int m = 0; m < 10 && m < n_rates; ++m) {
    const int i = m / 2, issuers = 1 + (m & 1);
    cudaError_t e = cudaSuccess;
    switch (i) {
      case 0: e = run_tc_probe<16>(sms, issuers, cyc, host); break;
      case 1: e = run_tc_probe<32>(sms, issuers, cyc, host); break;
      case 2: e = run_tc_probe<64>(sms, issuers, cyc, host); break;
      case 3: e = run_tc_probe<128>(sms, issuers, cyc, host); break;
      case 4: e = run_tc_probe<256>(sms, issuers, cyc, host); break;
    }
    if (e != cudaSuccess) {
      rc = FMS_ERR_CUDA;
      break;
    }
    std::vector<long long> v = host;
    std::sort(v.begin(), v.end());
    const double med = (double)v[v.size() / 2];
    const double flop = 2.0 * 128.0 * Ns[i] * 16.0 * kTcProbeIters * issuers;
    rates[m] = med > 0 ? flop / med : -1.0;
  }
  cudaFree(cyc);
  return rc;
}
