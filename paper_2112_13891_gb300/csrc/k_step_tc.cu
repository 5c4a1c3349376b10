// ms_step on the 5th-generation tensor cores (tcgen05), for 1 <= d <= 32.
//
// For a tile of 128 seeds (rows) and a tile of 128 points, in scaled
// coordinates (w = exp2(-||y - x||^2)):
//   S = Y X^T           tcgen05.mma kind::f16, BF16 operands, FP32 in TMEM.
//                       Y and X are split into hi + lo BF16 parts and
//                       S ~= Yh Xh^T + Yh Xl^T + Yl Xh^T (three MMAs per K
//                       step), which keeps the cancellation in
//                       ||y||^2 + ||x||^2 - 2 y.x at ~2^-16 relative.
//                       A fourth K block adds -||x||^2 / 2 to S: the tile
//                       carries it as three BF16 pieces (e0 + e1 + e2, 24
//                       significant bits) that meet a constant [0 1 1 1 0..]
//                       block of Y, so D = y.x - ||x||^2 / 2 in FP32.
//   w = exp2(2D - ||y||^2)   epilogue: TMEM -> registers, one FFMA with the
//                       seed's FP32 norm, MUFU.EX2, BF16 weights P -> smem.
//   [sum w x_hi | sum w x_lo | sum w] = P [Xh | Xl | 1]   second product, the
//                       point tile read as an MN-major B operand; accumulated
//                       in TMEM over the point tiles of the chunk.
// The chunk's partials are written as (W, sum w (x - y)) -- the layout of the
// FP32 kernels -- so the same update kernel consumes them.  This is the
// coarse ("precision") step: weights carry BF16 rounding (2^-9 relative), so
// seeds switch to the exact FP32 step before their convergence is decided.
//
// Point tiles come from a packed image per 128 points (built once per call):
//   X2 = [Xh | Xl | 1 e0 e1 e2 0 .. 0]  128 points x N2 (N2 = 2 DPAD + 16)
//              BF16, in core matrices of 8 points x 8 columns (16 B rows, no
//              swizzle); e0 + e1 + e2 = -||x||^2 / 2 (e0 = -inf, e1 = e2 = 0 for
//              padding points, so their weight is exactly 0).  Its Xh, Xl and
//              last column ranges are K-major B operands of the first product;
//              the whole of it is the MN-major B of the second (whose columns
//              2 DPAD + 1 .. are never read).
// One TMA bulk copy (cp.async.bulk) per tile; every wait is bounded and sets
// an error bit instead of hanging.
#include <cuda_bf16.h>

#include "fms_internal.cuh"
#include "fms_tc.cuh"

namespace fms {

namespace tc {

constexpr int kM = 128;       // seeds per tile (MMA M)
constexpr int kP = 128;       // points per tile (MMA N of the first product, K of the second)
constexpr int kEpiWarps = 16;  // epilogue warps: (TMEM lane quarter) x (column quarter)
constexpr int kThreads = (kEpiWarps + 2) * 32;  // + loader / S-issuer warp + P-issuer warp

template <int DPAD>
struct Geo {
  static constexpr int N2 = 2 * DPAD + 16;               // [Xh | Xl | 1 e0 e1 e2 0 ..]
  static constexpr int kX2Bytes = kP * N2 * 2;
  static constexpr int kTileBytes = kX2Bytes;
  static constexpr int kYextBytes = kM * 16 * 2;        // constant [0 1 1 1 0 ..] rows
  static constexpr int kYBytes = kM * DPAD * 2;          // one of Yh / Yl
  static constexpr int kPBytes = kM * kP * 2;
  static constexpr int kStages = 6;                      // tile ring
  // smem: Yh, Yl, Yext, P x 2, ring of kStages tile images (200 KB for DPAD = 32)
  static constexpr int kSmem = 2 * kYBytes + kYextBytes + 2 * kPBytes + kStages * kTileBytes;
  // TMEM: S accumulators D1 x 3 (3 x 128 columns), D2 = [hi sums | lo sums | W]
  static constexpr int kD2 = 3 * 128;
  static constexpr int kTmemCols = 512;
  static_assert(kSmem <= 227 * 1024, "shared memory");
  static_assert(kD2 + N2 <= kTmemCols, "tensor memory");
};
}  // namespace tc

// Tile images of the scaled points Xs [n][DP] (DP >= d, zero padded).
template <int DPAD>
__global__ void tc_pack_tiles(const float* __restrict__ Xs, int n, int DP,
                              unsigned char* __restrict__ img) {
  using G = tc::Geo<DPAD>;
  const int t = blockIdx.x;
  unsigned char* base = img + (size_t)t * G::kTileBytes;
  __nv_bfloat16* x2 = reinterpret_cast<__nv_bfloat16*>(base);
  for (int e = threadIdx.x; e < tc::kP * DPAD; e += blockDim.x) {
    const int p = e / DPAD, k = e % DPAD;
    const int j = t * tc::kP + p;
    const float v = (j < n && k < DP) ? Xs[(size_t)j * DP + k] : 0.f;
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    x2[tc::core_index(p, k, G::N2)] = hi;
    x2[tc::core_index(p, DPAD + k, G::N2)] = lo;
  }
  for (int e = threadIdx.x; e < tc::kP; e += blockDim.x) {
    const int j = t * tc::kP + e;
    // e0 + e1 + e2 = -||x||^2 / 2 (FP32 norm, split into three BF16 pieces)
    float e0 = -INFINITY, e1 = 0.f, e2 = 0.f;
    if (j < n) {
      float s = 0.f;
      for (int k = 0; k < DP; ++k) {
        const float v = Xs[(size_t)j * DP + k];
        s = fmaf(v, v, s);
      }
      const float h = -0.5f * s;
      e0 = __bfloat162float(__float2bfloat16_rn(h));
      e1 = __bfloat162float(__float2bfloat16_rn(h - e0));
      e2 = h - e0 - e1;
    }
    for (int k = 0; k < 16; ++k) {
      const float v = k == 0 ? 1.f : k == 1 ? e0 : k == 2 ? e1 : k == 3 ? e2 : 0.f;
      x2[tc::core_index(e, 2 * DPAD + k, G::N2)] = __float2bfloat16_rn(v);
    }
  }
}

// The coarse step for active positions [0, count) of a list of s_total;
// chunks of Lc points (a multiple of 128).  A persistent grid (one CTA per SM
// holding all 512 TMEM columns) walks (seed tile, chunk) tasks.
// Partial (c, p): part[(c * s_total + p) * DA + k], k <= DP.
//
// Warp roles (warp-specialised, no CTA-wide barrier inside a task).  One
// thread issues at most one tcgen05.mma per ~70-90 clocks, so the MMAs of a
// tile are split between two issuing threads:
//   warp 16, lane 0 (loader): bulk copies up to kStages tiles ahead into a
//       ring of tile buffers (a buffer is refilled once P(j) has read it), and
//       S(j+2) = Y X(j+2)^T into the one of three TMEM accumulators that the
//       epilogue of tile j-1 released.
//   warp 17, lane 0 (P issuer): P(j) = P_j [Xh | Xl | 1] into D2 as soon as
//       the epilogue of tile j has signalled.
//   warps 0..15 (epilogue): for tile j, warp w takes TMEM lanes 32 (w % 4) ..
//       +31 (seed rows) and columns 32 (w / 4) .. +31 (points): w = exp2(2S -
//       ny - nx), rounded to BF16 into P buffer j % 2 (two buffers, so the
//       epilogue of tile j+1 overlaps the product of tile j).
// mbarriers (tile / product numbers are counted across the CTA's tasks):
// bar_load[b] (copy landed), bar_s[j % 3] (S(j) done), bar_o[j % 3] (P(j)
// done: its P buffer and tile buffer are free, D2 final), bar_p[j % 3] (the
// epilogue warps wrote P of tile j and read its S accumulator; waited by both
// issuers), bar_y (the epilogue warps wrote the Y tile of a non-empty task and
// read the previous task's D2).  The loader waits for P(j-1) before it issues
// S(j+2), so no role can run two phases ahead of a waiter.  Every wait is for
// the current or the just-completed phase of its barrier (checked with a
// model of the three roles over random interleavings) and bounded; a wait
// that gives up sets kStTimeout and a shared abort flag that ends every
// role's loop.
template <int DPAD>
__global__ void __launch_bounds__(tc::kThreads, 1)
    ms_step_tc(const unsigned char* __restrict__ img, int n, const float* __restrict__ y, int DP,
               int DA, const int32_t* __restrict__ active, const int32_t* __restrict__ s_total_ptr,
               const int32_t* __restrict__ count_ptr, const int32_t* __restrict__ C_ptr,
               const int32_t* __restrict__ Lc_ptr, float* __restrict__ part, uint32_t* status,
               int32_t* __restrict__ s_log) {
  using G = tc::Geo<DPAD>;
  constexpr int S = G::kStages;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_load[S], bar_s[3], bar_o[3], bar_p[3], bar_y;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_abort;
  unsigned char* sYh = smem;
  unsigned char* sYl = smem + G::kYBytes;
  unsigned char* sYext = smem + 2 * G::kYBytes;
  unsigned char* sP = sYext + G::kYextBytes;             // P[0], P[1]
  unsigned char* sRing = sP + 2 * G::kPBytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
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

  constexpr int kCtl = tc::kEpiWarps;  // the loader warp; kCtl + 1: the P-issuer warp
  if (tid == kCtl * 32) {
    for (int i = 0; i < S; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::su32(&bar_load[i])));
    for (int i = 0; i < 3; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::su32(&bar_s[i])));
    for (int i = 0; i < 3; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::su32(&bar_o[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc::su32(&bar_p[i])),
                   "r"(tc::kEpiWarps));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc::su32(&bar_y)),
                 "r"(tc::kEpiWarps));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  // constant Y extension rows [0 1 1 1 0 .. 0] (K-major core matrices of 16 columns)
  for (int e = tid; e < tc::kM * 16; e += blockDim.x) {
    const int row = e >> 4, k = e & 15;
    reinterpret_cast<__nv_bfloat16*>(sYext)[tc::core_index(row, k, 16)] =
        __float2bfloat16_rn((k >= 1 && k <= 3) ? 1.f : 0.f);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == kCtl) {
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
  const uint32_t tD2 = tmem + G::kD2;                  // D1[i] = tmem + 128 i, i < 3
  const int tiles_per_chunk = Lc / tc::kP;
  const int ntiles_total = (n + tc::kP - 1) / tc::kP;
  bool bad = false;
  const bool issuer = warp >= kCtl;
  auto wait = [&](uint64_t* bar, uint32_t parity) -> bool {
    if (!(issuer ? tc::wait_bar_abort<true>(bar, parity, &s_abort)
                 : tc::wait_bar_abort<false>(bar, parity, &s_abort))) {
      bad = true;
      s_abort = 1;
      return false;
    }
    return true;
  };

  if (warp == kCtl) {
    if (lane == 0) {
      // ------------------------------ loader ------------------------------
      const uint32_t id1 = tc::idesc_bf16(tc::kM, tc::kP);
      const uint32_t x_row = (G::N2 / 8) * 128;        // X2: next 8-point block
      uint32_t n_load = 0, n_lw = 0, n_s = 0, n_task = 0;
      auto issue_load = [&](int t) {
        const uint32_t b = n_load % S;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                         tc::su32(&bar_load[b])),
                     "r"((uint32_t)G::kTileBytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                tc::su32(sRing + b * G::kTileBytes)),
            "l"(img + (size_t)t * G::kTileBytes), "r"((uint32_t)G::kTileBytes),
            "r"(tc::su32(&bar_load[b]))
            : "memory");
        ++n_load;
      };
      // S = Yh Xh^T + Yh Xl^T + Yl Xh^T for the tile in ring buffer `buf`
      auto issue_s = [&](uint32_t buf) {
        const unsigned char* sT = sRing + buf * G::kTileBytes;
        const uint32_t dt = tmem + (n_s % 3u) * 128u;
        const uint32_t sbo = (DPAD / 8) * 128;
#pragma unroll
        for (int ks = 0; ks < DPAD / 16; ++ks) {
          const uint64_t ah = tc::sdesc(tc::su32(sYh) + ks * 256, 128, sbo);
          const uint64_t al = tc::sdesc(tc::su32(sYl) + ks * 256, 128, sbo);
          const uint64_t bh = tc::sdesc(tc::su32(sT) + ks * 256, 128, x_row);
          const uint64_t bl = tc::sdesc(tc::su32(sT) + (DPAD / 8) * 128 + ks * 256, 128, x_row);
          tc::mma(dt, ah, bh, id1, ks > 0 ? 1u : 0u);
          tc::mma(dt, ah, bl, id1, 1u);
          tc::mma(dt, al, bh, id1, 1u);
        }
        // + [0 1 1 1 0 ..] . [1 e0 e1 e2 0 ..] = -||x||^2 / 2
        tc::mma(dt, tc::sdesc(tc::su32(sYext), 128, 256),
                tc::sdesc(tc::su32(sT) + (2 * DPAD / 8) * 128, 128, x_row), id1, 1u);
        tc::commit(&bar_s[n_s % 3u]);
        ++n_s;
      };
      auto wait_load = [&](uint32_t L) -> bool {
        const bool ok = wait(&bar_load[L % S], (L / S) & 1u);
        ++n_lw;
        return ok;
      };
      uint32_t g0 = 0;                                 // global number of the task's tile 0
      for (long task = blockIdx.x; task < T && !s_abort; task += gridDim.x) {
        const int c = (int)(task / ntile_seed);
        const int t0 = c * tiles_per_chunk;
        const int nt = max(0, min(ntiles_total, t0 + tiles_per_chunk) - t0);
        if (nt == 0) continue;                         // (no handshake for an empty task)
        if (!wait(&bar_y, n_task & 1u)) break;         // Y tile written, last D2 read
        ++n_task;
        tc::fence_after();
        const uint32_t base = n_load;                  // load number of tile 0 (== g0)
        for (int i = 0; i < nt && i < S; ++i) issue_load(t0 + i);
        if (!wait_load(base)) break;
        issue_s(base % S);
        if (nt > 1) {
          if (!wait_load(base + 1)) break;
          issue_s((base + 1) % S);
        }
        for (int j = 0; j < nt; ++j) {
          const uint32_t g = g0 + (uint32_t)j;
          if (j >= 1 && j - 1 + S < nt) {              // refill the buffer of tile j-1
            if (!wait(&bar_o[(g - 1) % 3u], ((g - 1) / 3u) & 1u)) break;  // P(j-1) read it
            issue_load(t0 + j - 1 + S);
          }
          if (j + 2 < nt) {                            // S(j+2) into the accumulator
            if (j >= 1 && !wait(&bar_p[(g - 1) % 3u], ((g - 1) / 3u) & 1u)) break;
            tc::fence_after();                         // that tile j-1 released
            if (!wait_load(base + j + 2)) break;
            issue_s((base + j + 2) % S);
          }
        }
        g0 += (uint32_t)nt;
      }
      if (bad || s_abort) {
        // one more bounded wait for every copy and product still in flight,
        // before the shared memory and the accumulators are released
        for (uint32_t L = n_lw; L < n_load; ++L) tc::wait_bar(&bar_load[L % S], (L / S) & 1u);
        if (n_s > 0) tc::wait_bar(&bar_s[(n_s - 1) % 3u], ((n_s - 1) / 3u) & 1u);
      }
    }
    __syncwarp();
  } else if (warp == kCtl + 1) {
    if (lane == 0) {
      // ---------------------------- P issuer -----------------------------
      const uint32_t id2 = tc::idesc_bf16(tc::kM, G::N2) | (1u << 16);  // B MN-major
      const uint32_t x_row = (G::N2 / 8) * 128;
      const uint32_t a_sbo = (tc::kP / 8) * 128;
      uint32_t n_o = 0;
      for (long task = blockIdx.x; task < T && !s_abort; task += gridDim.x) {
        const int c = (int)(task / ntile_seed);
        const int t0 = c * tiles_per_chunk;
        const int nt = max(0, min(ntiles_total, t0 + tiles_per_chunk) - t0);
        for (int j = 0; j < nt; ++j) {
          if (!wait(&bar_p[n_o % 3u], (n_o / 3u) & 1u)) break;  // epilogue of tile j done
          tc::fence_after();
          const unsigned char* sT = sRing + (n_o % S) * G::kTileBytes;
          const unsigned char* sPj = sP + (n_o & 1u) * G::kPBytes;
#pragma unroll
          for (int ks = 0; ks < tc::kP / 16; ++ks) {
            // MN-major B: LBO = next 8 points (K), SBO = next 8 columns (N)
            const uint64_t a = tc::sdesc(tc::su32(sPj) + ks * 256, 128, a_sbo);
            const uint64_t b = tc::sdesc(tc::su32(sT) + ks * 2 * x_row, x_row, 128);
            tc::mma(tD2, a, b, id2, (j > 0 || ks > 0) ? 1u : 0u);
          }
          tc::commit(&bar_o[n_o % 3u]);
          ++n_o;
        }
      }
      if (bad || s_abort) {
        if (n_o > 0) tc::wait_bar(&bar_o[(n_o - 1) % 3u], ((n_o - 1) / 3u) & 1u);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------ epilogue ------------------------------
    const int q = warp & 3, cq = warp >> 2;
    const int r_row = q * 32 + lane;                   // this thread's seed row
    const int c0 = cq * 32;                            // this warp's point columns
    const uint32_t row_lane = (uint32_t)(q * 32) << 16;
    uint32_t n_s = 0, n_o = 0, n_t = 0;   // S products consumed, P products, tiles
    for (long task = blockIdx.x; task < T && !s_abort; task += gridDim.x) {
      const int st = (int)(task % ntile_seed);
      const int c = (int)(task / ntile_seed);
      const int t0 = c * tiles_per_chunk;
      const int nt = max(0, min(ntiles_total, t0 + tiles_per_chunk) - t0);
      const int prow = st * tc::kM + r_row;
      const bool valid = prow < count;
      if (nt == 0) {                                   // (no handshake for an empty task)
        if (cq == 0 && valid) {
          float* o = part + ((int64_t)c * s_total + prow) * DA;
          for (int k = 0; k <= DP; ++k) o[k] = 0.f;
        }
        continue;
      }
      const int64_t slot = __ldg(active + (valid ? prow : count - 1));
      const float* yrow = y + slot * DP;
      float ny = 0.f;
      // Y tile (hi / lo, K-major core matrices): warp column quarter cq writes
      // the 8-wide k chunks k0 with k0 / 8 == cq (mod 4)
#pragma unroll
      for (int k0 = 0; k0 < DPAD; k0 += 8) {
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          v[e] = k0 + e < DP ? __ldg(yrow + k0 + e) : 0.f;
          ny = fmaf(v[e], v[e], ny);
        }
        if (((k0 >> 3) & 3) != cq) continue;
        uint32_t h4[4], l4[4];
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
          const float a = v[2 * qq], b = v[2 * qq + 1];
          const __nv_bfloat16 ah = __float2bfloat16_rn(a), bh = __float2bfloat16_rn(b);
          h4[qq] = tc::pack_bf16(__bfloat162float(ah), __bfloat162float(bh));
          l4[qq] = tc::pack_bf16(a - __bfloat162float(ah), b - __bfloat162float(bh));
        }
        const int off = tc::core_index(r_row, k0, DPAD) * 2;
        *reinterpret_cast<uint4*>(sYh + off) = make_uint4(h4[0], h4[1], h4[2], h4[3]);
        *reinterpret_cast<uint4*>(sYl + off) = make_uint4(l4[0], l4[1], l4[2], l4[3]);
      }
      if (!valid) ny = INFINITY;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::arrive(&bar_y);
      // software pipeline over 16-column halves: the TMEM load of the next half
      // (of this tile, or of tile j+1) is in flight while a half is computed
      // w = exp2(2 D - ||y||^2), D = y.x - ||x||^2 / 2 from the S accumulator
      auto compute_half = [&](int h, const uint32_t (&rr)[16], uint32_t* pk) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float u0 = fmaf(2.f, __uint_as_float(rr[2 * i]), -ny);
          const float u1 = fmaf(2.f, __uint_as_float(rr[2 * i + 1]), -ny);
          pk[8 * h + i] = tc::pack_bf16(ex2_ftz(u0), ex2_ftz(u1));
        }
      };
      uint32_t ra[16], rb[16];
      bool ok = wait(&bar_s[n_s % 3u], (n_s / 3u) & 1u);
      uint32_t d1 = tmem + (n_s % 3u) * 128u + row_lane + c0;
      if (ok) {
        tc::fence_after();
        tc::ld16_issue(d1, ra);
      }
      for (int j = 0; ok && j < nt; ++j) {
        uint32_t pk[16];
        tc::wait_ld16(ra);
        tc::ld16_issue(d1 + 16, rb);
        compute_half(0, ra, pk);
        tc::wait_ld16(rb);
        ++n_s;                                           // tile j's accumulator read
        if (j + 1 < nt) {
          if (!(ok = wait(&bar_s[n_s % 3u], (n_s / 3u) & 1u))) break;
          tc::fence_after();
          d1 = tmem + (n_s % 3u) * 128u + row_lane + c0;
          tc::ld16_issue(d1, ra);
        }
        compute_half(1, rb, pk);
        tc::fence_before();                              // S accumulator reads done
        // P buffer n_o & 1 was last read by product n_o - 2
        if (n_o >= 2 && !(ok = wait(&bar_o[(n_o - 2) % 3u], ((n_o - 2) / 3u) & 1u))) break;
        unsigned char* sPj = sP + (n_o & 1u) * G::kPBytes;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int off = tc::core_index(r_row, c0 + 8 * i, tc::kP) * 2;
          *reinterpret_cast<uint4*>(sPj + off) =
              make_uint4(pk[4 * i], pk[4 * i + 1], pk[4 * i + 2], pk[4 * i + 3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) tc::arrive(&bar_p[n_o % 3u]);
        ++n_o;                                           // P(j) follows
      }
      if (!ok) {
        tc::wait_ld16(ra);                               // no load left in flight
        tc::wait_ld16(rb);
      }
      n_t += (uint32_t)nt;
      if (s_abort) break;
      // partials of this (seed tile, chunk): W and sum w (x - y)
      {
        if (!wait(&bar_o[(n_o - 1) % 3u], ((n_o - 1) / 3u) & 1u)) break;  // last P product
        tc::fence_after();
        if (cq == 0) {
          // D2 columns: [0, DPAD) sum w x_hi, [DPAD, 2 DPAD) sum w x_lo, 2 DPAD: sum w
          float vh[16], vl[16];
          tc::ld16(tD2 + row_lane + 2 * DPAD, vh);
          const float W = vh[0];
          float* o = part + ((int64_t)c * s_total + prow) * DA;
          if (valid) o[0] = W;
#pragma unroll
          for (int k0 = 0; k0 < DPAD; k0 += 16) {
            tc::ld16(tD2 + row_lane + k0, vh);
            tc::ld16(tD2 + row_lane + DPAD + k0, vl);
#pragma unroll
            for (int e = 0; e < 16; ++e)
              if (valid && k0 + e < DP)
                o[1 + k0 + e] = (vh[e] + vl[e]) - __ldg(yrow + k0 + e) * W;
          }
        }
        tc::fence_before();                              // D2 reads done (next bar_y)
      }
    }
  }
  if (bad) atomicOr(status, kStTimeout);
  tc::fence_before();
  __syncthreads();
  if (warp == kCtl)
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

// One persistent CTA per SM: each holds all 512 TMEM columns.
int tc_grid(int d) {
  static int cache[2] = {0, 0};
  const int i = d <= 16 ? 0 : 1;
  if (cache[i]) return cache[i];
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return 1;
  cudaError_t e;
  if (i == 0)
    e = cudaFuncSetAttribute(ms_step_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             tc::Geo<16>::kSmem);
  else
    e = cudaFuncSetAttribute(ms_step_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             tc::Geo<32>::kSmem);
  if (e != cudaSuccess) return sms;
  cache[i] = sms;
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

// Self-test of the bounded waits ms_step_tc uses: one CTA waits on phase 0
// of a fresh mbarrier that nothing completes, with `spins` polls, through the
// helper `variant` selects (0: wait_bar, 1: polling wait_bar_abort, 2:
// suspending wait_bar_abort); a wait that gives up sets kStTimeout, as in
// the step kernel.  Then one arrival completes the phase and the same wait
// must succeed (kStBadArg if it does not).
__global__ void wait_selftest_kernel(uint32_t* status, long spins, int variant) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ volatile int abort_flag;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::su32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  __syncthreads();
  bool ok;
  if (variant == 1) ok = tc::wait_bar_abort<true>(&bar, 0, &abort_flag, spins);
  else if (variant == 2) ok = tc::wait_bar_abort<false>(&bar, 0, &abort_flag, spins);
  else ok = tc::wait_bar(&bar, 0, spins);
  if (!ok) atomicOr(status, kStTimeout);
  __syncthreads();
  if (threadIdx.x == 0)
    asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(tc::su32(&bar))
                 : "memory");
  __syncthreads();
  if (!tc::wait_bar(&bar, 0, spins)) atomicOr(status, kStBadArg);
}

cudaError_t launch_wait_selftest(uint32_t* status, long spins, int variant, cudaStream_t st) {
  wait_selftest_kernel<<<1, 64, 0, st>>>(status, spins, variant);
  return cudaGetLastError();
}

}  // namespace fms
