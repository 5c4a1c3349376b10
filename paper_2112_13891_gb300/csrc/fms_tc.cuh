// tcgen05 / mbarrier helpers (inline PTX) shared by the tensor-core kernels:
// shared-memory matrix descriptors for K-major or MN-major operands in 8 x 8
// core matrices (16-byte rows, no swizzle), the BF16 instruction descriptor,
// the MMA issue and its commit to an mbarrier, bounded mbarrier waits, and
// tensor-memory loads.
#pragma once

#include <cuda_bf16.h>

#include "fms_internal.cuh"

namespace fms {
namespace tc {

constexpr long kSpin = 1l << 24;   // bound of every mbarrier wait (then: give up)

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
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t phase, long spins = kSpin) {
  for (long it = 0; it < spins; ++it) {
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

// bounded wait that also gives up when another role has set the abort flag.
// The single-thread issuers poll with the non-suspending test_wait (their
// hand-offs are on the critical path); the epilogue warps use try_wait, which
// may suspend the warp and leaves its issue slots to the other warps.
template <bool kPoll>
__device__ __forceinline__ bool wait_bar_abort(uint64_t* bar, uint32_t phase,
                                               volatile int* abort_flag, long spins = kSpin) {
  for (long it = 0; it < spins; ++it) {
    uint32_t ok;
    if (kPoll)
      asm volatile(
          "{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
          : "=r"(ok)
          : "r"(su32(bar)), "r"(phase)
          : "memory");
    else
      asm volatile(
          "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
          : "=r"(ok)
          : "r"(su32(bar)), "r"(phase)
          : "memory");
    if (ok) return true;
    if ((it & 63) == 63 && *abort_flag) return false;
  }
  return false;
}

// One bulk copy (TMA, untiled) of `bytes` from global to shared memory that
// completes a transaction count on `bar`; the issuing thread first announces
// the bytes.  Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(bar))
      : "memory");
}

// Orders this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy (bulk copy) writes to it.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void init_bar(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count));
}

// A warp walks rows [r0, r1) of a row-major global array (ROW elements of T
// per row, rows 16-byte aligned, ROW * sizeof(T) a multiple of 16) through a
// two-tile ring of its own in shared memory: lane 0 keeps up to two bulk
// copies of kRingRows rows in flight, every lane calls row_fn(row pointer) for
// each row in order.  tiles: 2 x kRingRows x ROW elements; bars: two
// mbarriers of count 1 (ring_init); use0 / use1: completed phases of each,
// carried across calls.  A wait that gives up sets kStTimeout in *status,
// waits once more for the copies in flight and returns false.
constexpr int kRingRows = 32;

__device__ __forceinline__ void ring_init(uint64_t* bars, int lane) {
  if (lane == 0) {
    init_bar(&bars[0], 1);
    init_bar(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
}

template <int ROW, typename T, typename F>
__device__ __forceinline__ bool ring_rows(const T* __restrict__ src, int r0, int r1, T* tiles,
                                          uint64_t* bars, uint32_t& use0, uint32_t& use1,
                                          int lane, uint32_t* status, F&& row_fn) {
  static_assert((ROW * sizeof(T)) % 16 == 0, "bulk copies move multiples of 16 bytes");
  constexpr int TE = kRingRows * ROW;   // elements per tile
  const int ntile = r1 > r0 ? (r1 - r0 + kRingRows - 1) / kRingRows : 0;
  auto issue = [&](int t) {
    const int a = r0 + t * kRingRows;
    const int rows = min(kRingRows, r1 - a);
    fence_proxy_async();   // the warp's reads of this stage came before (syncwarp)
    bulk_g2s(tiles + (t & 1) * TE, src + (int64_t)a * ROW, (uint32_t)(rows * ROW * sizeof(T)),
             &bars[t & 1]);
  };
  if (lane == 0) {
    if (ntile > 0) issue(0);
    if (ntile > 1) issue(1);
  }
  int t = 0;
  for (; t < ntile; ++t) {
    const int st = t & 1;
    if (!wait_bar(&bars[st], (st ? use1 : use0) & 1u)) break;
    if (st) ++use1;
    else ++use0;
    const T* tl = tiles + st * TE;
    const int rows = min(kRingRows, r1 - (r0 + t * kRingRows));
    for (int q = 0; q < rows; ++q) row_fn(tl + q * ROW);
    __syncwarp();
    if (lane == 0 && t + 2 < ntile) issue(t + 2);
  }
  if (t == ntile) return true;
  if (lane == 0) atomicOr(status, kStTimeout);
  for (int u = t; u < ntile && u < t + 2; ++u) {   // the copies issued and not consumed
    if (u & 1) {
      wait_bar(&bars[1], use1 & 1u);
      ++use1;
    } else {
      wait_bar(&bars[0], use0 & 1u);
      ++use0;
    }
  }
  return false;
}

__device__ __forceinline__ void arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
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

// tcgen05.ld of 16 columns without waiting; the registers are valid only after
// wait_ld16 on the same array (which names them as read-write operands, so no
// use can be scheduled before the wait)
__device__ __forceinline__ void ld16_issue(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ void wait_ld16(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
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
}  // namespace fms
