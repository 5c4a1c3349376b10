// ms_step on the 5th-generation tensor cores (tcgen05), for 9 <= d <= 32.
//
// For a tile of 128 seeds (rows) and a tile of 128 points, in scaled
// coordinates (w = exp2(-||y - x||^2)):
//   S = Y X^T           tcgen05.mma kind::f16, BF16 operands, FP32 in TMEM.
//                       Y and X are split into hi + lo BF16 parts and
//                       S ~= Yh Xh^T + Yh Xl^T + Yl Xh^T (three MMAs per K
//                       step), which keeps the cancellation in
//                       ||y||^2 + ||x||^2 - 2 y.x at ~2^-16 relative.
//   w = exp2(2S - ||y||^2 - ||x||^2)   epilogue: TMEM -> registers (one seed
//                       row per thread), FP32 norms, MUFU.EX2, BF16 P -> smem.
//   [W, sum w x] = P [1 | Xh | Xl]     a second MMA, accumulated in TMEM over
//                       the point tiles of the chunk.
// The chunk's partials are written as (W, sum w (x - y)) -- the layout of the
// FP32 kernels -- so the same update kernel consumes them.  This is the
// coarse ("precision") step: weights carry BF16 rounding (2^-9 relative), so
// seeds switch to the exact FP32 step before their convergence is decided.
//
// Point tiles come from a packed image per 128 points (built once per call):
//   [Xh | Xl]  B operand of the first MMA (128 rows x DPAD, K-major core
//              matrices, no swizzle); [XT] B operand of the second MMA
//   (N2 = 1 + 2 DPAD padded to 16 rows x 128 points); [nx] 128 FP32 norms
//   (+inf for padding points, so their weight is exactly 0).
// One TMA bulk copy (cp.async.bulk) per tile; every wait is bounded and sets
// an error bit instead of hanging.
#include <cuda_bf16.h>

#include "fms_internal.cuh"

namespace fms {

namespace tc {

constexpr int kM = 128;       // seeds per tile (MMA M)
constexpr int kP = 128;       // points per tile (MMA N of the first product, K of the second)
constexpr int kThreads = 128; // one warpgroup: thread r owns seed row r in the epilogue
constexpr long kSpin = 1l << 24;

template <int DPAD>
struct Geo {
  static constexpr int N2 = ((1 + 2 * DPAD) + 15) / 16 * 16;
  static constexpr int kXBytes = kP * DPAD * 2;          // one of Xh / Xl
  static constexpr int kXTBytes = N2 * kP * 2;
  static constexpr int kTileBytes = 2 * kXBytes + kXTBytes + kP * 4;
  static constexpr int kYBytes = kM * DPAD * 2;          // one of Yh / Yl
  static constexpr int kPBytes = kM * kP * 2;
  // smem: Yh, Yl, tile image, P; requested as at least 80 KB so that no more
  // than two CTAs (2 x 256 TMEM columns) share an SM
  static constexpr int kSmemUsed = 2 * kYBytes + kTileBytes + kPBytes;
  static constexpr int kSmem = kSmemUsed > 80 * 1024 ? kSmemUsed : 80 * 1024;
  static constexpr int kTmemCols = 256;                  // D1 (128) + D2 (<= 80)
};

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__host__ __device__ __forceinline__ int core_index(int r, int k, int K) {
  return ((r >> 3) * (K >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t dt, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dt),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          su32(bar))
      : "memory");
}

// bounded wait on an mbarrier phase; false when the bound ran out
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t phase) {
  for (long it = 0; it < kSpin; ++it) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(phase)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

}  // namespace tc

// Tile images of the scaled points Xs [n][DP] (DP >= d, zero padded).
template <int DPAD>
__global__ void tc_pack_tiles(const float* __restrict__ Xs, int n, int DP,
                              unsigned char* __restrict__ img) {
  using G = tc::Geo<DPAD>;
  const int t = blockIdx.x;
  unsigned char* base = img + (size_t)t * G::kTileBytes;
  __nv_bfloat16* xh = reinterpret_cast<__nv_bfloat16*>(base);
  __nv_bfloat16* xl = reinterpret_cast<__nv_bfloat16*>(base + G::kXBytes);
  __nv_bfloat16* xt = reinterpret_cast<__nv_bfloat16*>(base + 2 * G::kXBytes);
  float* nx = reinterpret_cast<float*>(base + 2 * G::kXBytes + G::kXTBytes);
  for (int e = threadIdx.x; e < tc::kP * DPAD; e += blockDim.x) {
    const int p = e / DPAD, k = e % DPAD;
    const int j = t * tc::kP + p;
    const float v = (j < n && k < DP) ? Xs[(size_t)j * DP + k] : 0.f;
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    xh[tc::core_index(p, k, DPAD)] = hi;
    xl[tc::core_index(p, k, DPAD)] = lo;
    // XT rows: 0 = ones, 1..DPAD = hi, DPAD+1..2DPAD = lo, rest zero
    xt[tc::core_index(1 + k, p, tc::kP)] = hi;
    xt[tc::core_index(1 + DPAD + k, p, tc::kP)] = lo;
  }
  for (int e = threadIdx.x; e < tc::kP; e += blockDim.x) {
    const int j = t * tc::kP + e;
    xt[tc::core_index(0, e, tc::kP)] = __float2bfloat16_rn(j < n ? 1.f : 0.f);
    for (int r = 1 + 2 * DPAD; r < G::N2; ++r) xt[tc::core_index(r, e, tc::kP)] = __float2bfloat16_rn(0.f);
    float s = INFINITY;
    if (j < n) {
      s = 0.f;
      for (int k = 0; k < DP; ++k) {
        const float v = Xs[(size_t)j * DP + k];
        s = fmaf(v, v, s);
      }
    }
    nx[e] = s;
  }
}

// The coarse step for active positions [0, count) of a list of s_total;
// chunks of Lc points (a multiple of 128); grid-stride over (seed tile,
// chunk) tasks.  Partial (c, p): part[(c * s_total + p) * DA + k], k <= DP.
template <int DPAD>
__global__ void __launch_bounds__(tc::kThreads)
    ms_step_tc(const unsigned char* __restrict__ img, int n, const float* __restrict__ y, int DP,
               int DA, const int32_t* __restrict__ active, const int32_t* __restrict__ s_total_ptr,
               const int32_t* __restrict__ count_ptr, const int32_t* __restrict__ C_ptr,
               const int32_t* __restrict__ Lc_ptr, float* __restrict__ part, uint32_t* status,
               int32_t* __restrict__ s_log) {
  using G = tc::Geo<DPAD>;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_load, bar_mma;
  __shared__ uint32_t tmem_base;
  unsigned char* sYh = smem;
  unsigned char* sYl = smem + G::kYBytes;
  unsigned char* sT = smem + 2 * G::kYBytes;
  unsigned char* sP = sT + G::kTileBytes;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int s_total = *s_total_ptr;
  const int count = *count_ptr;  // coarse seeds: positions [0, count)
  const int C = *C_ptr, Lc = *Lc_ptr;
  if (s_log && blockIdx.x == 0 && tid == 0) *s_log = count;
  if (count <= 0 || C <= 0) return;
  if (Lc <= 0 || Lc % tc::kP != 0 || count > s_total) {
    if (blockIdx.x == 0 && tid == 0) atomicOr(status, kStBadArg);
    return;
  }
  const int ntile_seed = (count + tc::kM - 1) / tc::kM;
  const long T = (long)ntile_seed * C;
  if ((long)blockIdx.x >= T) return;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::su32(&bar_load)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::su32(&bar_mma)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc::su32(&tmem_base)),
                 "r"(G::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t tD1 = tmem, tD2 = tmem + 128;
  const uint32_t id1 = tc::idesc_bf16(tc::kM, tc::kP), id2 = tc::idesc_bf16(tc::kM, G::N2);
  uint32_t ph_load = 0, ph_mma = 0;
  bool bad = false;
  const int tiles_per_chunk = Lc / tc::kP;
  const int ntiles_total = (n + tc::kP - 1) / tc::kP;

  for (long task = blockIdx.x; task < T; task += gridDim.x) {
    const int st = (int)(task % ntile_seed);
    const int c = (int)(task / ntile_seed);
    // this thread's seed row
    const int prow = st * tc::kM + tid;
    const bool valid = prow < count;
    const int64_t slot = __ldg(active + (valid ? prow : count - 1));
    float yv[DPAD];
    float ny = 0.f;
#pragma unroll
    for (int k = 0; k < DPAD; ++k) {
      yv[k] = k < DP ? __ldg(y + slot * DP + k) : 0.f;
      ny = fmaf(yv[k], yv[k], ny);
    }
    if (!valid) ny = INFINITY;
    // Y tile (hi / lo, K-major core matrices), 8 k per 16-byte store
#pragma unroll
    for (int k0 = 0; k0 < DPAD; k0 += 8) {
      uint32_t h4[4], l4[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float a = yv[k0 + 2 * q], b = yv[k0 + 2 * q + 1];
        const __nv_bfloat16 ah = __float2bfloat16_rn(a), bh = __float2bfloat16_rn(b);
        h4[q] = tc::pack_bf16(__bfloat162float(ah), __bfloat162float(bh));
        l4[q] = tc::pack_bf16(a - __bfloat162float(ah), b - __bfloat162float(bh));
      }
      const int off = tc::core_index(tid, k0, DPAD) * 2;
      *reinterpret_cast<uint4*>(sYh + off) = make_uint4(h4[0], h4[1], h4[2], h4[3]);
      *reinterpret_cast<uint4*>(sYl + off) = make_uint4(l4[0], l4[1], l4[2], l4[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc::fence_before();
    __syncthreads();
    tc::fence_after();

    const int t0 = c * tiles_per_chunk;
    const int t1 = min(ntiles_total, t0 + tiles_per_chunk);
    for (int t = t0; t < t1; ++t) {
      // tile image -> smem (TMA bulk copy)
      if (tid == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                         tc::su32(&bar_load)),
                     "r"((uint32_t)G::kTileBytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                tc::su32(sT)),
            "l"(img + (size_t)t * G::kTileBytes), "r"((uint32_t)G::kTileBytes),
            "r"(tc::su32(&bar_load))
            : "memory");
      }
      if (!tc::wait_bar(&bar_load, ph_load)) bad = true;
      ph_load ^= 1u;
      // S = Yh Xh^T + Yh Xl^T + Yl Xh^T
      if (tid == 0) {
        tc::fence_after();
        const uint32_t sbo = (DPAD / 8) * 128;
        for (int ks = 0; ks < DPAD / 16; ++ks) {
          const uint64_t ah = tc::sdesc(tc::su32(sYh) + ks * 256, 128, sbo);
          const uint64_t al = tc::sdesc(tc::su32(sYl) + ks * 256, 128, sbo);
          const uint64_t bh = tc::sdesc(tc::su32(sT) + ks * 256, 128, sbo);
          const uint64_t bl = tc::sdesc(tc::su32(sT + G::kXBytes) + ks * 256, 128, sbo);
          tc::mma(tD1, ah, bh, id1, ks > 0 ? 1u : 0u);
          tc::mma(tD1, ah, bl, id1, 1u);
          tc::mma(tD1, al, bh, id1, 1u);
        }
        tc::commit(&bar_mma);
      }
      if (!tc::wait_bar(&bar_mma, ph_mma)) bad = true;
      ph_mma ^= 1u;
      tc::fence_after();
      // epilogue: w = exp2(2 S - ny - nx) -> BF16 P[row][point]
      const float* nx = reinterpret_cast<const float*>(sT + 2 * G::kXBytes + G::kXTBytes);
#pragma unroll 1
      for (int c0 = 0; c0 < tc::kP; c0 += 32) {
        float sv[32];
        tc::ld32(tD1 + ((uint32_t)(warp * 32) << 16) + c0, sv);
#pragma unroll
        for (int j0 = 0; j0 < 32; j0 += 8) {
          uint32_t p4[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int j = j0 + 2 * q;
            const float u0 = fmaf(2.f, sv[j], -(ny + nx[c0 + j]));
            const float u1 = fmaf(2.f, sv[j + 1], -(ny + nx[c0 + j + 1]));
            p4[q] = tc::pack_bf16(ex2_ftz(u0), ex2_ftz(u1));
          }
          const int off = tc::core_index(tid, c0 + j0, tc::kP) * 2;
          *reinterpret_cast<uint4*>(sP + off) = make_uint4(p4[0], p4[1], p4[2], p4[3]);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc::fence_before();
      const int abort_now = __syncthreads_or(bad ? 1 : 0);
      tc::fence_after();
      if (abort_now) break;  // uniform: a bounded wait gave up somewhere in the CTA
      // [W, sum w x] += P [1 | Xh | Xl]
      if (tid == 0) {
        const uint32_t sbo = (tc::kP / 8) * 128;
        for (int ks = 0; ks < tc::kP / 16; ++ks) {
          const uint64_t a = tc::sdesc(tc::su32(sP) + ks * 256, 128, sbo);
          const uint64_t b = tc::sdesc(tc::su32(sT + 2 * G::kXBytes) + ks * 256, 128, sbo);
          tc::mma(tD2, a, b, id2, (t > t0 || ks > 0) ? 1u : 0u);
        }
        tc::commit(&bar_mma);
      }
      if (!tc::wait_bar(&bar_mma, ph_mma)) bad = true;
      ph_mma ^= 1u;
      tc::fence_after();
    }
    // partials of this (seed tile, chunk): W and sum w (x - y)
    if (__syncthreads_or(bad ? 1 : 0)) break;
    if (t1 > t0) {
      float acc[G::N2];
#pragma unroll
      for (int c0 = 0; c0 < G::N2; c0 += 16) {
        float v[16];
        tc::ld16(tD2 + ((uint32_t)(warp * 32) << 16) + c0, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[c0 + i] = v[i];
      }
      if (valid) {
        float* o = part + ((int64_t)c * s_total + prow) * DA;
        const float W = acc[0];
        o[0] = W;
#pragma unroll
        for (int k = 0; k < DPAD; ++k)
          if (k < DP) o[1 + k] = (acc[1 + k] + acc[1 + DPAD + k]) - yv[k] * W;
      }
    } else if (valid) {
      float* o = part + ((int64_t)c * s_total + prow) * DA;
      for (int k = 0; k <= DP; ++k) o[k] = 0.f;
    }
    tc::fence_before();
    const int abort_task = __syncthreads_or(bad ? 1 : 0);
    tc::fence_after();
    if (abort_task) break;
  }
  if (bad) {
    atomicOr(status, kStTimeout);
    // give the operations that did not signal one more bounded wait before
    // the accumulators are released
    tc::wait_bar(&bar_load, ph_load ^ 1u);
    tc::wait_bar(&bar_mma, ph_mma ^ 1u);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(G::kTmemCols)
                 : "memory");
}

size_t tc_image_bytes(int64_t n, int d) {
  const int64_t tiles = (n + tc::kP - 1) / tc::kP;
  return (size_t)tiles * (d <= 16 ? tc::Geo<16>::kTileBytes : tc::Geo<32>::kTileBytes);
}

cudaError_t launch_tc_pack(const float* Xs, int64_t n, int d, int DP, unsigned char* img,
                           cudaStream_t st) {
  const int tiles = (int)((n + tc::kP - 1) / tc::kP);
  if (d <= 16) tc_pack_tiles<16><<<tiles, 256, 0, st>>>(Xs, (int)n, DP, img);
  else tc_pack_tiles<32><<<tiles, 256, 0, st>>>(Xs, (int)n, DP, img);
  return cudaGetLastError();
}

int tc_grid(int d) {
  static int cache[2] = {0, 0};
  const int i = d <= 16 ? 0 : 1;
  if (cache[i]) return cache[i];
  int dev = 0, sms = 0, blocks = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (i == 0) {
    cudaFuncSetAttribute(ms_step_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         tc::Geo<16>::kSmem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ms_step_tc<16>, tc::kThreads,
                                                  tc::Geo<16>::kSmem);
  } else {
    cudaFuncSetAttribute(ms_step_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         tc::Geo<32>::kSmem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ms_step_tc<32>, tc::kThreads,
                                                  tc::Geo<32>::kSmem);
  }
  // at most two CTAs per SM: each holds 256 of the SM's 512 TMEM columns
  if (blocks > 2) blocks = 2;
  if (blocks < 1) blocks = 1;
  cache[i] = sms * blocks;
  return cache[i];
}

cudaError_t launch_ms_step_tc(const unsigned char* img, int64_t n, int d, int DP, int DA,
                              const float* y, const int32_t* active, const int32_t* s_total_ptr,
                              const int32_t* count_ptr, const int32_t* C_ptr,
                              const int32_t* Lc_ptr, float* part, uint32_t* status,
                              cudaStream_t st, int32_t* s_log) {
  if (d < 1 || d > kTcMaxDim || DP < d || DA < DP + 1) return cudaErrorInvalidValue;
  const int grid = tc_grid(d);
  if (d <= 16)
    ms_step_tc<16><<<grid, tc::kThreads, tc::Geo<16>::kSmem, st>>>(
        img, (int)n, y, DP, DA, active, s_total_ptr, count_ptr, C_ptr, Lc_ptr, part, status,
        s_log);
  else
    ms_step_tc<32><<<grid, tc::kThreads, tc::Geo<32>::kSmem, st>>>(
        img, (int)n, y, DP, DA, active, s_total_ptr, count_ptr, C_ptr, Lc_ptr, part, status,
        s_log);
  return cudaGetLastError();
}

}  // namespace fms
