// ms_grid_round: one Seed-Selection round of Gaussian mean-shift updates
// (Eq. 6, the update of Alg. 2 under the Early Stopping of Sec. II-C) on a
// persistent grid of one CTA per SM.
//
// Decomposition.  CTA c owns a fixed, contiguous slice of the points (n / G
// points for G CTAs), staged once into shared memory by TMA bulk copies when
// it fits (else read from L2), and cut into sub-slices.  In every update each
// CTA evaluates every active seed of the round against its slice.  A warp task
// is (a group of seeds, a range of the slice); lane l takes the range's points
// l, l + 32, ...; the 32 lane sums are combined by a fixed xor tree.  That
// FP32 value -- the partial of one seed over one range -- is a leaf.  A list of
// A seeds is cut into 16 contiguous shares of A / 16 or A / 16 + 1 seeds, one
// per compute warp, each over whole sub-slices; the extra seeds go to
// consecutive warps, which sit on different SM sub-partitions, so that the
// issue load of every sub-partition is even.  Leaves are converted to 64-bit
// fixed point (2^F units, F chosen so that no sum over all n points can
// overflow) and added exactly into the update's global accumulator
// (red.global.add.u64).  Integer addition is associative, so the totals do
// not depend on which warp or CTA took which task or on the order of the
// atomics; the only rounding is that of the leaves and of one conversion to
// FP32 per total.  Four accumulators rotate.
//
// Roles and pipeline.  Phases alternate between two seed lists.  While 16
// compute warps evaluate list j, the comm warp publishes phase j - 1 (one grid
// barrier: a release-add on a counter, an acquire poll, both bounded), stages
// its totals in shared memory with one bulk copy and turns each seed's
// integer totals into the float update [W, S / W].  At the start of phase j + 1
// the compute warps apply those updates to list j - 1's seeds (the same update
// in every CTA's replicated copy of the round's seed state), ballot which stay
// live and, behind two barriers, write and read list j + 1.  Named barriers
// pass each phase between the roles.  CTA 0 writes the seed state back to
// global memory.
//
// Early Stopping.  Every CTA keeps the convergence histogram of all seeds of
// all rounds; after each update it finds t_stop, the first update count whose
// cumulative convergence count reaches ceil(gamma N), and deactivates every
// RUNNING seed that has made t_stop or more updates without converging: such
// a seed converges (if ever) after t* <= t_stop and cannot be kept.  Counts
// only grow, so the kept set is that of the synchronous rule; a stopped seed
// stays RUNNING with its update count (a later round may resume it).
#include "fms_internal.cuh"

namespace fms {

namespace {

constexpr int kGridCompWarps = 16;                  // warps that evaluate seeds
constexpr int kCommWarp = kGridCompWarps;           // the exchange warp
constexpr int kGridThreads = (kGridCompWarps + 1) * 32;
constexpr int kComp = kGridCompWarps * 32;          // compute threads
// Named barriers (0 is __syncthreads), one per parity where a phase passes
// from the compute warps to the comm warp and back.
constexpr int kBarPass = 1;     // compute -> comm: leaves of phase j issued
constexpr int kBarStaged = 3;   // comm -> compute: totals of phase j staged
constexpr int kBarComp = 5;     // among the compute warps
constexpr int kGridBufs = 4;                        // accumulators in rotation
constexpr int kGridMerge = 32;   // at most this many active seeds: one list per update
constexpr int kGridSubLen = 2048;                // longest sub-slice (points)
constexpr long long kGridSpinCycles = 4000000000LL;   // bound of one wait (~2 s)

// Shared memory carving (bytes), identical on host and device.
struct GridSmem {
  int off_bar, off_misc, off_y, off_it, off_slot, off_act, off_w, off_conv, off_list, off_ws, off_hist,
      off_stage, off_pts;
  int total;
};

__host__ __device__ inline int al16(int x) { return (x + 15) & ~15; }

// Seeds one round launch holds: two staged publications of DA accumulators
// per seed must fit in shared memory beside the seed state and the slice.
__host__ __device__ constexpr int grid_seed_cap(int DA) { return DA == 8 ? 512 : kGridMaxSeeds; }

// Seeds one compute warp takes in a phase, at most: a share of a full list.
__host__ __device__ constexpr int grid_ws(int SC) { return SC / kGridCompWarps + 4; }

__host__ __device__ inline GridSmem grid_smem(int D, int DA, int DP, int pts) {
  const int SC = grid_seed_cap(DA);
  GridSmem s{};
  int o = 0;
  s.off_bar = o;
  o += 16;
  s.off_misc = o;
  o += 256;
  s.off_y = o;
  o = al16(o + SC * D * 4);
  s.off_it = o;
  o += SC * 4;
  s.off_slot = o;
  o += SC * 4;
  s.off_act = o;   // state (kRunning, kConverged, ...)
  o += SC * 4;
  s.off_w = o;     // sum w of the latest update
  o += SC * 4;
  s.off_conv = o;  // convergence update
  o += SC * 4;
  s.off_list = o;  // two buffers of each phase list, the pool of deferred seeds
  o += 5 * SC * 4;
  s.off_ws = o;    // each compute warp's seeds of the current phase
  o += kGridCompWarps * grid_ws(SC) * 4;
  s.off_hist = o;
  o += kGridHist * 4;
  s.off_stage = o; // the staged totals of the last publication of each parity
  o += 2 * SC * DA * 8;
  s.off_pts = o;
  o += pts * DP * 4;
  s.total = o;
  return s;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void bar_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ void bar_arrive(int id, int n) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ void red_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Reduce-scatter of 32 values across the warp: lane l returns sum over lanes
// of v[l] (fixed xor tree, the same for every slot).
__device__ __forceinline__ float grid_rs32(float (&v)[32], int lane) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const float send = up ? v[i] : v[i + o];
      const float keep = up ? v[i + o] : v[i];
      v[i] = keep + __shfl_xor_sync(kFull, send, o);
    }
  }
  return v[0];
}

// Leaf partials of RR seeds (active positions a0 .. a0 + cnt - 1) over the
// points [j0, j1) of this CTA's slice (pts: shared or global memory, DP floats
// per point): exact-difference form, acc[r][0] = sum w, acc[r][1 + k] =
// sum w (x - y)_k.  The RR x DA sums are reduce-scattered over the warp in
// blocks of 32 (lane l of block q holds accumulator 32 q + l), converted to
// fixed point and added into the update's global accumulator dst[r * DA + k]
// (red.global).
template <int D, int DP, int DA, int RR, int KF, bool RES>
__device__ __forceinline__ void grid_task(const float* __restrict__ pts, int j0, int j1, int lane,
                                          const int* __restrict__ alist, int a0, int cnt,
                                          const float* __restrict__ sy,
                                          unsigned long long* dst, float fx) {
  constexpr int NV = (RR * DA + 31) / 32;
  float ys[RR][D];
#pragma unroll
  for (int r = 0; r < RR; ++r) {
    const int i = alist[a0 + (r < cnt ? r : cnt - 1)];
#pragma unroll
    for (int k = 0; k < D; ++k) ys[r][k] = sy[i * D + k];
  }
  float acc[RR][DA];
#pragma unroll
  for (int r = 0; r < RR; ++r)
#pragma unroll
    for (int k = 0; k < DA; ++k) acc[r][k] = 0.0f;
#pragma unroll 4
  for (int j = j0 + lane; j < j1; j += 32) {
    float x[D];
    const float4 p0 = RES ? *reinterpret_cast<const float4*>(pts + (size_t)j * DP)
                          : __ldg(reinterpret_cast<const float4*>(pts + (size_t)j * DP));
    float t8[8];
    t8[0] = p0.x;
    t8[1] = p0.y;
    t8[2] = p0.z;
    t8[3] = p0.w;
    if constexpr (DP == 8) {
      const float4 p1 = RES ? *reinterpret_cast<const float4*>(pts + (size_t)j * DP + 4)
                            : __ldg(reinterpret_cast<const float4*>(pts + (size_t)j * DP + 4));
      t8[4] = p1.x;
      t8[5] = p1.y;
      t8[6] = p1.z;
      t8[7] = p1.w;
    }
#pragma unroll
    for (int k = 0; k < D; ++k) x[k] = t8[k];
#pragma unroll
    for (int r = 0; r < RR; ++r) {
      float dx[D];
#pragma unroll
      for (int k = 0; k < D; ++k) dx[k] = x[k] - ys[r][k];
      float t = -dx[0] * dx[0];
#pragma unroll
      for (int k = 1; k < D; ++k) t = fmaf(-dx[k], dx[k], t);
      const float w = kweight<KF>(t);
      acc[r][0] += w;
#pragma unroll
      for (int k = 0; k < D; ++k) acc[r][1 + k] = fmaf(w, dx[k], acc[r][1 + k]);
    }
  }
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    float v[32];
#pragma unroll
    for (int e = 0; e < 32; ++e) {
      const int f = 32 * q + e;
      v[e] = f < RR * DA ? acc[f / DA][f % DA] : 0.0f;
    }
    const float s = grid_rs32(v, lane);
    const int f = 32 * q + lane;
    if (f < cnt * DA) {
      const long long qv = __float2ll_rn(s * fx);
      red_add_u64(dst + f, (unsigned long long)qv);
    }
  }
}

template <int D, int DP, int DA, int KF, bool RES, int RR>
__device__ __forceinline__ void grid_task_r(int R, const float* pts, int j0, int j1, int lane,
                                            const int* alist, int a0, int cnt, const float* sy,
                                            unsigned long long* dst, float fx) {
  if constexpr (RR >= 1) {
    if (R == RR) {
      grid_task<D, DP, DA, RR, KF, RES>(pts, j0, j1, lane, alist, a0, cnt, sy, dst, fx);
      return;
    }
    grid_task_r<D, DP, DA, KF, RES, RR - 1>(R, pts, j0, j1, lane, alist, a0, cnt, sy, dst, fx);
  }
}

// Largest seed group a warp task takes (two reduce-scatters at most).
template <int D, int DA>
constexpr int grid_rmax() {
  return DA == 2 ? 12 : (DA == 4 ? 6 : 3);
}

}  // namespace

template <int D, int DP, int DA, int KF, bool RES>
__global__ void __launch_bounds__(kGridThreads, 1) ms_grid_round_kernel(const GridRoundArgs a) {
  constexpr int RMAX = grid_rmax<D, DA>();
  constexpr int SC = grid_seed_cap(DA);
  extern __shared__ __align__(16) unsigned char smem[];
  const GridSmem L = grid_smem(D, DA, DP, RES ? a.per_cta : 0);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L.off_bar);   // [0] slice, [1] totals
  // misc: [0], [1] sizes of the even / odd phase lists, [2] the phase at
  // which the compute warps stop (0: not known yet), [3] S, [12], [13] the
  // buffer holding each parity's list, [14] the t_stop it was built with,
  // [16 .. 31] the compute warps' ballots of live entries,
  // [4] converged seeds (all rounds), [5] abort, [6] pool size, [32..63] scan
  int* misc = reinterpret_cast<int*>(smem + L.off_misc);
  float* sy = reinterpret_cast<float*>(smem + L.off_y);
  int* sit = reinterpret_cast<int*>(smem + L.off_it);
  int* sslot = reinterpret_cast<int*>(smem + L.off_slot);
  int* sst = reinterpret_cast<int*>(smem + L.off_act);
  float* sw = reinterpret_cast<float*>(smem + L.off_w);
  int* sconv = reinterpret_cast<int*>(smem + L.off_conv);
  int* lists = reinterpret_cast<int*>(smem + L.off_list);   // [parity][buffer][SC], pool[SC]
  int* pool = lists + 4 * SC;
  int* wseeds = reinterpret_cast<int*>(smem + L.off_ws);
  int* hist_s = reinterpret_cast<int*>(smem + L.off_hist);
  unsigned long long* stage = reinterpret_cast<unsigned long long*>(smem + L.off_stage);
  float* spts = reinterpret_cast<float*>(smem + L.off_pts);

  const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int N = a.rc ? a.rc->N : a.N_arg;
  const int target = a.rc ? a.rc->target : a.target_arg;
  const int cb = min(a.n, cta * a.per_cta), ce = min(a.n, cb + a.per_cta);
  const int nc = ce - cb;
  const float fx = a.fx_scale, inv_fx = a.inv_fx_scale;

  // --- barriers; stage this CTA's point slice (TMA bulk copies) ---
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar + 1)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (RES) {
      const uint32_t bytes = (uint32_t)nc * DP * 4;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)),
                   "r"(bytes)
                   : "memory");
      const char* src = reinterpret_cast<const char*>(a.Xs + (size_t)cb * DP);
      for (uint32_t off = 0; off < bytes; off += 32768u) {
        const uint32_t len = bytes - off < 32768u ? bytes - off : 32768u;
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(spts) + off),
            "l"(src + off), "r"(len), "r"(smem_u32(mbar))
            : "memory");
      }
    }
    misc[2] = 0;
    misc[4] = 0;
    misc[5] = 0;
    misc[6] = 0;
  }
  // --- the round's seeds: RUNNING slots of [0, N) in slot order (the same
  // list in every CTA) ---
  {
    int base = 0;
    for (int b = 0; b < N; b += kGridThreads) {
      const int i = b + tid;
      const int take = (i < N) && a.state[i] == kRunning;
      int tot;
      const int off = block_exclusive_scan(take, &tot, misc + 32);
      if (take && base + off < SC) {
        const int p = base + off;
        sslot[p] = i;
        sit[p] = a.it[i];
        sst[p] = kRunning;
        sw[p] = a.wlast[i];
        sconv[p] = a.conv[i];
#pragma unroll
        for (int k = 0; k < D; ++k) sy[p * D + k] = a.y[(size_t)i * DP + k];
      }
      base += tot;
    }
    if (tid == 0) misc[3] = base;
  }
  {
    int conv_total = 0;
    for (int c = tid; c < kGridHist; c += kGridThreads) {
      const int v = (c >= 1 && c <= a.max_iter) ? __ldcg(a.hist + c) : 0;
      hist_s[c] = v;
      conv_total += v;
    }
    if (conv_total) atomicAdd(misc + 4, conv_total);
  }
  __syncthreads();
  const int S = misc[3];
  if (RES) {
    // every thread waits for the slice copy (bounded); a copy that did not
    // land is flagged, and the first grid barrier sends every CTA home
    bool ok = false;
    const long long t0 = clock64();
    for (;;) {
      uint32_t r;
      asm volatile(
          "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
          : "=r"(r)
          : "r"(smem_u32(mbar)), "r"(0u)
          : "memory");
      if (r) {
        ok = true;
        break;
      }
      if (clock64() - t0 > kGridSpinCycles) break;
    }
    if (!ok && tid == 0) atomicOr(a.status, kStTimeout);
  }
  if (S > SC) {
    // the host keeps N within the capacity; a larger list is an error (every
    // CTA sees the same S and returns before the first grid barrier)
    if (cta == 0 && tid == 0) atomicOr(a.status, kStCapacity);
    return;
  }

  // t_stop (one warp): the first update count whose cumulative convergence
  // count reaches the target; INT32_MAX while fewer seeds have converged
  auto t_stop = [&]() -> int {
    int ts = INT32_MAX;
    if (misc[4] >= target) {
      int carry = 0;
      for (int b0 = 1; b0 <= a.max_iter && ts == INT32_MAX; b0 += 32) {
        const int t = b0 + lane;
        int v = t <= a.max_iter ? hist_s[t] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int u = __shfl_up_sync(kFull, v, o);
          if (lane >= o) v += u;
        }
        const unsigned hit = __ballot_sync(kFull, t <= a.max_iter && carry + v >= target);
        if (hit) ts = b0 + __ffs(hit) - 1;
        carry += __shfl_sync(kFull, v, 31);
      }
    }
    return ts;
  };
  // a seed stays in the lists while RUNNING and below t_stop (a seed that
  // has made t_stop updates without converging cannot be kept)
  auto live = [&](int p, int ts) { return sst[p] == kRunning && sit[p] < ts; };

  // first two phase lists: the live seeds alternately (one list when few)
  if (warp == kCommWarp) {
    const int ts = t_stop();
    int nl = 0;
    for (int b0 = 0; b0 < S; b0 += 32) {
      const int p = b0 + lane;
      const unsigned m = __ballot_sync(kFull, p < S && live(p, ts));
      nl += __popc(m);
    }
    const bool split = nl > kGridMerge;
    int n0 = 0, n1 = 0;
    for (int b0 = 0; b0 < S; b0 += 32) {
      const int p = b0 + lane;
      const bool t = p < S && live(p, ts);
      const unsigned m = __ballot_sync(kFull, t);
      if (t) {
        const int r = n0 + n1 + __popc(m & ((1u << lane) - 1));
        if (split && (r & 1)) lists[2 * SC + (r >> 1)] = p;
        else lists[split ? (r >> 1) : r] = p;
      }
      const int c = __popc(m);
      if (split) {
        const int tot = n0 + n1 + c;
        n0 = (tot + 1) >> 1;
        n1 = tot >> 1;
      } else {
        n0 += c;
      }
    }
    if (lane == 0) {
      misc[0] = n0;
      misc[1] = n1;
      misc[12] = 0;   // buffer of each parity's list
      misc[13] = 0;
      misc[14] = ts;  // the t_stop the lists were built with
    }
  }
  __syncthreads();
  if (misc[0] + misc[1] == 0) return;

  const int max_phase = 4 * (a.max_iter + 4);
  const size_t stride = (size_t)SC * DA;
  if (warp < kGridCompWarps) {
    // ---- compute warps.  Phase j: apply the staged updates of phase j - 2
    // (this parity) to its seeds, find which stay live, evaluate list j ----
    const int n_sub = a.n_sub, sub_len = a.sub_len;
    const float* pts = RES ? spts : a.Xs + (size_t)cb * DP;
    int* ws = wseeds + warp * grid_ws(SC);
    int q = 0;   // publications so far (non-empty phases)
    for (int j = 0; j < max_phase; ++j) {
      const int par = j & 1;
      // Work split of a list of A seeds: warp w takes a contiguous share of
      // A / 16 seeds, one more for w < A mod 16 (consecutive warps sit on
      // different SM sub-partitions, so the extra seeds spread over them), in
      // groups of at most RMAX, each over every sub-slice.
      int A, cw, aw;
      auto split = [&](int A_) {
        A = A_;
        const int per = A / kGridCompWarps, ex = A - per * kGridCompWarps;
        cw = per + (warp < ex ? 1 : 0);
        aw = warp * per + min(warp, ex);
      };
      if (j < 2) {
        const int* l0 = lists + 2 * par * SC;
        split(misc[par]);
        for (int r = lane; r < cw; r += 32) ws[r] = l0[aw + r];
        __syncwarp();
      } else {
        bar_sync(kBarStaged + par, kGridThreads);   // updates of phase j - 2 staged
        if (*(volatile int*)(misc + 5)) break;     // the exchange failed
        const int Aold = misc[par], ps = misc[6], B = misc[par ^ 1];
        const int cur = misc[12 + par], ts_old = misc[14];
        const int* lold = lists + (2 * par + cur) * SC;
        int* lnew = lists + (2 * par + (cur ^ 1)) * SC;
        const float* stg = reinterpret_cast<const float*>(stage + (size_t)par * stride);
        const bool fast = Aold <= kComp && ps <= 32;
        // the update of every seed of phase j - 2 (the same in every CTA):
        // y + S / W, staged by the comm warp as [W, S_0 / W, S_1 / W, ...]
        int pe = 0;
        bool lv = false;
        for (int e = tid; e < Aold; e += kComp) {
          const int p = lold[e];
          float f[DA];
          const float4* f4 = reinterpret_cast<const float4*>(stg + (size_t)e * 2 * DA);
#pragma unroll
          for (int k = 0; k < (DA + 3) / 4; ++k) {
            const float4 v = f4[k];
            f[4 * k] = v.x;
            if (4 * k + 1 < DA) f[4 * k + 1] = v.y;
            if (4 * k + 2 < DA) f[4 * k + 2] = v.z;
            if (4 * k + 3 < DA) f[4 * k + 3] = v.w;
          }
          const float W = f[0];
          bool ok = W > 0.0f && isfinite(W);
          float dl[D], step2 = 0.0f;
#pragma unroll
          for (int k = 0; k < D; ++k) {
            dl[k] = f[1 + k];
            step2 = fmaf(dl[k], dl[k], step2);
          }
          ok = ok && isfinite(step2);
          if (ok && a.sphere_r > 0.0f) {
            // cosine metric: the mean scaled back onto the sphere of radius
            // sphere_r; the step is the projected one
            float pp[D], nn = 0.0f;
#pragma unroll
            for (int k = 0; k < D; ++k) {
              pp[k] = sy[p * D + k] + dl[k];
              nn = fmaf(pp[k], pp[k], nn);
            }
            const float fs = a.sphere_r / sqrtf(nn);
            step2 = 0.0f;
#pragma unroll
            for (int k = 0; k < D; ++k) {
              pp[k] *= fs;
              const float d2 = pp[k] - sy[p * D + k];
              step2 = fmaf(d2, d2, step2);
            }
            ok = nn > 0.0f && isfinite(step2);
            if (ok) {
#pragma unroll
              for (int k = 0; k < D; ++k) sy[p * D + k] = pp[k];
            }
          } else if (ok) {
#pragma unroll
            for (int k = 0; k < D; ++k) sy[p * D + k] += dl[k];
          }
          const int t = sit[p] + 1;
          sit[p] = t;
          int st = kRunning;
          if (!ok) st = kFailed;
          else if (step2 <= a.tol2_s) st = kConverged;
          else if (t >= a.max_iter) st = kExhausted;
          sst[p] = st;
          // sum w of this update, at the position before its step: the
          // prune's density of a seed whose last update this is
          sw[p] = W;
          if (st == kConverged) {
            sconv[p] = t;
            if (t < kGridHist) atomicAdd(hist_s + t, 1);
            atomicAdd(misc + 4, 1);
          }
          pe = p;
          lv = st == kRunning && t < ts_old;   // live under the last t_stop
        }
        // list j: the live seeds of phase j - 2 and of the pool, or none (the
        // candidates wait in the pool) when few seeds are left and phase
        // j - 1 (evaluated, not yet applied) has some, so that the lists merge
        const unsigned m = __ballot_sync(kFull, lv);
        if (lane == 0) misc[16 + warp] = (int)m;
        const int pp = lane < ps ? pool[lane] : 0;
        const bool plv = lane < ps && live(pp, ts_old);
        const unsigned pm = __ballot_sync(kFull, plv);
        bar_sync(kBarComp, kComp);   // every update applied, every entry read, every ballot posted
        const int ts = t_stop();
        if (fast && ts == ts_old) {
          // ranks from the ballots; the owners write the new list (or the
          // pool) while the old list and the pool are no longer read
          int c = lane < kGridCompWarps ? __popc((unsigned)misc[16 + lane]) : 0;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(kFull, c, o);
            if (lane >= o) c += u;
          }
          const int nl = __shfl_sync(kFull, c, kGridCompWarps - 1);
          const int before = warp ? __shfl_sync(kFull, c, warp - 1) : 0;
          const int np = __popc(pm);
          const bool defer = B > 0 && B + nl + np <= kGridMerge;
          const int rank = before + __popc(m & ((1u << lane) - 1));
          const int prank = __popc(pm & ((1u << lane) - 1));
          if (defer) {
            if (lv) pool[np + rank] = pe;
            if (warp == 0 && plv) pool[prank] = pp;
          } else {
            if (lv) lnew[rank] = pe;
            if (warp == 0 && plv) lnew[nl + prank] = pp;
          }
          if (tid == 0) {
            misc[par] = defer ? 0 : nl + np;
            misc[6] = defer ? nl + np : 0;
            misc[12 + par] = cur ^ 1;
            // nothing left anywhere: the compute warps stop here
            if (!defer && nl + np == 0 && B == 0) misc[2] = j;
          }
        } else if (warp == 0) {
          // a list longer than one entry per thread, a long pool, or a new
          // t_stop: one warp compacts
          int nl = 0;
          for (int b0 = 0; b0 < Aold; b0 += 32) {
            const int e = b0 + lane;
            const int p = e < Aold ? lold[e] : 0;
            const bool t = e < Aold && live(p, ts);
            const unsigned mm = __ballot_sync(kFull, t);
            if (t) lnew[nl + __popc(mm & ((1u << lane) - 1))] = p;
            nl += __popc(mm);
          }
          int np = 0;
          for (int b0 = 0; b0 < ps; b0 += 32) {   // in place: writes never pass reads
            const int e = b0 + lane;
            const int p = e < ps ? pool[e] : 0;
            const bool t = e < ps && live(p, ts);
            const unsigned mm = __ballot_sync(kFull, t);
            if (t) pool[np + __popc(mm & ((1u << lane) - 1))] = p;
            np += __popc(mm);
          }
          __syncwarp();
          const bool defer = B > 0 && B + nl + np <= kGridMerge;
          int next = 0;
          if (defer) {
            for (int e = lane; e < nl; e += 32) pool[np + e] = lnew[e];
            np += nl;
          } else {
            for (int e = lane; e < np; e += 32) lnew[nl + e] = pool[e];
            next = nl + np;
            np = 0;
          }
          __syncwarp();
          if (lane == 0) {
            misc[par] = next;
            misc[6] = np;
            misc[12 + par] = cur ^ 1;
            misc[14] = ts;
            if (next == 0 && B == 0 && np == 0) misc[2] = j;
          }
        }
        bar_sync(kBarComp, kComp);   // list j written
        split(misc[par]);
        for (int r = lane; r < cw; r += 32) ws[r] = lnew[aw + r];
        __syncwarp();
        const bool done = misc[2] != 0;
        if (done) {
          bar_arrive(kBarPass + par, kGridThreads);   // releases the comm warp, which then leaves
          break;
        }
      }
      if (A > 0) {
        unsigned long long* g = a.gacc + (size_t)(q % kGridBufs) * stride;
        const int mg = (cw + RMAX - 1) / RMAX;
        const int R = mg > 0 ? (cw + mg - 1) / mg : 0;
        // one call site, so that the kernel holds one copy of each group
        // size's code
        for (int t = 0; t < mg * n_sub; ++t) {
          const int gi = t / n_sub, sb = t - gi * n_sub;
          const int a0 = gi * R, cnt = min(R, cw - gi * R);
          const int j0 = min(nc, sb * sub_len), j1 = min(nc, j0 + sub_len);
          grid_task_r<D, DP, DA, KF, RES, RMAX>(cnt, pts, j0, j1, lane, ws, a0, cnt, sy,
                                                g + (size_t)(aw + a0) * DA, fx);
        }
        ++q;
      }
      bar_arrive(kBarPass + par, kGridThreads);   // pass j done
    }
  } else if (warp == kCommWarp) {
    // ---- comm warp: publishes phase j (the grid barrier), waits for every
    // CTA's leaves, stages the totals in shared memory and turns them into
    // updates, while the compute warps run phase j + 1 ----
    int q = 0, prev_used = 0;
    unsigned long long evals = 0;
    for (int j = 0; j < max_phase; ++j) {
      const int par = j & 1;
      bar_sync(kBarPass + par, kGridThreads);   // leaves of phase j issued (or done)
      const int stop = *(volatile int*)(misc + 2);
      if (stop && j >= stop) break;
      const int A = misc[par];
      bool bad = false;
      if (A > 0) {
        const unsigned long long* g = a.gacc + (size_t)(q % kGridBufs) * stride;
        __threadfence();
        int b = 0;
        if (lane == 0) {
          red_release_add(a.gbar, 1u);
          const unsigned want = (unsigned)G * (unsigned)(q + 1);
          const long long t0 = clock64();
          for (int it = 0;; ++it) {
            if (ld_acquire(a.gbar) >= want) break;
            if ((it & 31) == 31) {
              if (*(volatile uint32_t*)a.status & kStTimeout) {
                b = 1;
                break;
              }
              if (clock64() - t0 > kGridSpinCycles) {
                atomicOr(a.status, kStTimeout);
                b = 1;
                break;
              }
            }
          }
          if (*(volatile uint32_t*)a.status & kStTimeout) b = 1;
          if (!b) {
            // the totals into shared memory: one bulk copy (async proxy)
            // after the acquire, one round trip for any A
            asm volatile("fence.proxy.async.global;" ::: "memory");
            const uint32_t bytes = (uint32_t)A * DA * 8;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                             smem_u32(mbar + 1)),
                         "r"(bytes)
                         : "memory");
            const char* src = reinterpret_cast<const char*>(g);
            const uint32_t dst = smem_u32(stage + (size_t)par * stride);
            for (uint32_t off = 0; off < bytes; off += 32768u) {
              const uint32_t len = bytes - off < 32768u ? bytes - off : 32768u;
              asm volatile(
                  "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                      dst + off),
                  "l"(src + off), "r"(len), "r"(smem_u32(mbar + 1))
                  : "memory");
            }
          }
        }
        __syncwarp();
        bad = __shfl_sync(kFull, b, 0) != 0;
        if (!bad) {
          // every CTA has read the previous publication's totals: CTA 0
          // clears that accumulator for the publication four ahead
          if (cta == 0 && q >= 1) {
            unsigned long long* gp = a.gacc + (size_t)((q - 1) % kGridBufs) * stride;
            for (int e = lane; e < prev_used * DA; e += 32) gp[e] = 0ull;
          }
          bool landed = false;
          const long long t0 = clock64();
          for (;;) {
            uint32_t r;
            asm volatile(
                "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                : "=r"(r)
                : "r"(smem_u32(mbar + 1)), "r"((uint32_t)(q & 1))
                : "memory");
            if (r) {
              landed = true;
              break;
            }
            if (clock64() - t0 > kGridSpinCycles) break;
          }
          if (!__all_sync(kFull, landed)) {
            if (lane == 0) atomicOr(a.status, kStTimeout);
            bad = true;
          }
        }
        if (!bad) {
          // each seed's update from its exact totals, in place: the entry's
          // DA integers become the floats [W, S_0 / W, S_1 / W, ...]
          unsigned long long* stg = stage + (size_t)par * stride;
          for (int e = lane; e < A; e += 32) {
            unsigned long long v[DA];
#pragma unroll
            for (int k = 0; k < DA; ++k) v[k] = stg[(size_t)e * DA + k];
            asm volatile("" ::: "memory");   // every integer read before the floats overwrite them
            float tot[DA];
#pragma unroll
            for (int k = 0; k < DA; ++k) tot[k] = __ll2float_rn((long long)v[k]) * inv_fx;
            const float W = tot[0];
            const float rW = W > 0.0f && isfinite(W) ? __frcp_rn(W) : 0.0f;
            float* fo = reinterpret_cast<float*>(stg + (size_t)e * DA);
            fo[0] = W;
#pragma unroll
            for (int k = 0; k < D; ++k) fo[1 + k] = tot[1 + k] * rW;
          }
          __syncwarp();
        }
        evals += (unsigned long long)A * (unsigned long long)a.n;
        prev_used = A;
        ++q;
      }
      if (bad && lane == 0) misc[5] = 1;
      __syncwarp();
      bar_arrive(kBarStaged + par, kGridThreads);   // totals of phase j staged
      if (bad) break;
    }
    if (cta == 0 && lane == 0 && evals) atomicAdd(a.evals, evals);
  }
  // the round's seed state and the convergence counts back to global memory
  __syncthreads();
  if (cta == 0) {
    for (int p = tid; p < S; p += kGridThreads) {
      const int slot = sslot[p];
#pragma unroll
      for (int k = 0; k < D; ++k) a.y[(size_t)slot * DP + k] = sy[p * D + k];
      a.it[slot] = sit[p];
      a.state[slot] = sst[p];
      a.wlast[slot] = sw[p];
      a.conv[slot] = sconv[p];
    }
    for (int t = 1 + tid; t <= a.max_iter; t += kGridThreads) a.hist[t] = hist_s[t];
  }
}

namespace {

// ---------------------------------------------------------------------------
// ms_grid_refine: the merged modes take more updates with FP64 positions (the
// refinement before the second prune), on the same decomposition as the
// round: CTA c owns a point slice (staged into shared memory by TMA bulk
// copies when it fits), every CTA evaluates every active mode against its
// slice with the round's warp tasks at the FP32 positions yf = fl32(ym), and
// the leaves are added exactly in 64-bit fixed point into one of three
// rotating accumulators.  One grid barrier per update (bounded; a timeout
// sets kStTimeout and every CTA leaves); after it every CTA reads the same
// totals and applies the same FP64 update to its copy of the modes:
//   ym <- ym + S/W - (ym - yf)   (= m(yf)),
// a mode stops once ||step|| <= tol (FP64) or after max_iter updates.  The
// density that orders the second prune is W of the mode's last update.  CTA
// 0 clears the accumulator of update u - 1 after barrier u (every CTA has
// read it) and writes the modes back at the end.
// ---------------------------------------------------------------------------
constexpr int kGridRefineModes = 512;   // modes one refinement launch holds
constexpr int kGridRefineWarps = 16;
constexpr int kGridRefineBufs = 3;

struct GridRefineArgs {
  const float* Xs;
  int n, per_cta, n_sub, sub_len;
  const float* y;
  const int32_t* kept;
  const int32_t* accepted;
  const int32_t* M_ptr;
  double* ym;
  float* yf;
  double* mscore;
  double tol2_s;
  int max_iter;
  int32_t* iters_out;
  unsigned long long* evals;
  unsigned long long* gacc;
  unsigned* gbar;
  uint32_t* status;
  float fx_scale;
  double inv_fx;
  double sphere_r;
};

struct RefineSmem {
  int off_bar, off_misc, off_y, off_ym, off_act, off_list, off_pts, total;
};

__host__ __device__ inline RefineSmem refine_smem(int D, int DP, int pts) {
  RefineSmem r{};
  int o = 0;
  r.off_bar = o;
  o += 16;
  r.off_misc = o;
  o += 256;
  r.off_y = o;
  o = al16(o + kGridRefineModes * D * 4);
  r.off_ym = o;
  o = al16(o + kGridRefineModes * D * 8);
  r.off_act = o;
  o += kGridRefineModes * 4;
  r.off_list = o;
  o += kGridRefineModes * 4;
  r.off_pts = o;
  o += pts * DP * 4;
  r.total = o;
  return r;
}

}  // namespace

template <int D, int DP, int DA, int KF, bool RES>
__global__ void __launch_bounds__(kGridRefineWarps * 32, 1)
    ms_grid_refine_kernel(const GridRefineArgs a) {
  constexpr int RMAX = grid_rmax<D, DA>();
  constexpr int kT = kGridRefineWarps * 32;
  extern __shared__ __align__(16) unsigned char smem[];
  const RefineSmem L = refine_smem(D, DP, RES ? a.per_cta : 0);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L.off_bar);
  int* misc = reinterpret_cast<int*>(smem + L.off_misc);   // [0] active count, [1] abort
  float* sy = reinterpret_cast<float*>(smem + L.off_y);
  double* sym = reinterpret_cast<double*>(smem + L.off_ym);
  int* sact = reinterpret_cast<int*>(smem + L.off_act);
  int* alist = reinterpret_cast<int*>(smem + L.off_list);
  float* spts = reinterpret_cast<float*>(smem + L.off_pts);
  const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int M = *a.M_ptr;
  if (M <= 0) return;
  if (M > kGridRefineModes) {   // the host keeps M within the capacity
    if (cta == 0 && tid == 0) atomicOr(a.status, kStCapacity);
    return;
  }
  const int cb = min(a.n, cta * a.per_cta), ce = min(a.n, cb + a.per_cta);
  const int nc = ce - cb;
  const float fx = a.fx_scale;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (RES) {
      const uint32_t bytes = (uint32_t)nc * DP * 4;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)),
                   "r"(bytes)
                   : "memory");
      const char* src = reinterpret_cast<const char*>(a.Xs + (size_t)cb * DP);
      for (uint32_t off = 0; off < bytes; off += 32768u) {
        const uint32_t len = bytes - off < 32768u ? bytes - off : 32768u;
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(spts) + off),
            "l"(src + off), "r"(len), "r"(smem_u32(mbar))
            : "memory");
      }
    }
    misc[1] = 0;
  }
  for (int i = tid; i < M; i += kT) {
    const int64_t src = a.kept[a.accepted[i]];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float v = a.y[src * DP + k];
      sy[i * D + k] = v;
      sym[i * D + k] = (double)v;
    }
    sact[i] = 1;
  }
  __syncthreads();
  if (RES) {
    bool ok = false;
    const long long t0 = clock64();
    for (;;) {
      uint32_t r;
      asm volatile(
          "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
          : "=r"(r)
          : "r"(smem_u32(mbar)), "r"(0u)
          : "memory");
      if (r) {
        ok = true;
        break;
      }
      if (clock64() - t0 > kGridSpinCycles) break;
    }
    if (!ok) atomicOr(a.status, kStTimeout);   // the first barrier sends every CTA home
  }
  const size_t stride = (size_t)kGridRefineModes * DA;
  const float* pts = RES ? spts : a.Xs + (size_t)cb * DP;
  int iters = 0, prev_used = 0;
  unsigned long long evals = 0;
  for (int pass = 0; pass < a.max_iter; ++pass) {
    if (warp == 0) {
      int base = 0;
      for (int b0 = 0; b0 < M; b0 += 32) {
        const int i = b0 + lane;
        const bool t = i < M && sact[i];
        const unsigned m = __ballot_sync(kFull, t);
        if (t) alist[base + __popc(m & ((1u << lane) - 1))] = i;
        base += __popc(m);
      }
      if (lane == 0) misc[0] = base;
    }
    __syncthreads();
    const int A = misc[0];
    if (A == 0) break;   // every mode has stopped (the same in every CTA)
    unsigned long long* g = a.gacc + (size_t)(pass % kGridRefineBufs) * stride;
    {
      const int m = (A + kGridRefineWarps * RMAX - 1) / (kGridRefineWarps * RMAX);
      int R = (A + kGridRefineWarps * m - 1) / (kGridRefineWarps * m);
      if (R < 1) R = 1;
      const int groups = (A + R - 1) / R;
      const int tasks = groups * a.n_sub;
      for (int t = warp; t < tasks; t += kGridRefineWarps) {
        const int gi = t / a.n_sub, sb = t - gi * a.n_sub;
        const int j0 = min(nc, sb * a.sub_len), j1 = min(nc, j0 + a.sub_len);
        const int a0 = gi * R;
        grid_task_r<D, DP, DA, KF, RES, RMAX>(R, pts, j0, j1, lane, alist, a0, min(R, A - a0),
                                              sy, g + (size_t)a0 * DA, fx);
      }
    }
    __syncthreads();   // this CTA's leaves are issued
    if (tid == 0) {
      int b = 0;
      __threadfence();
      red_release_add(a.gbar, 1u);
      const unsigned want = (unsigned)G * (unsigned)(pass + 1);
      const long long t0 = clock64();
      for (int it = 0;; ++it) {
        if (ld_acquire(a.gbar) >= want) break;
        if ((it & 31) == 31) {
          if (*(volatile uint32_t*)a.status & kStTimeout) {
            b = 1;
            break;
          }
          if (clock64() - t0 > kGridSpinCycles) {
            atomicOr(a.status, kStTimeout);
            b = 1;
            break;
          }
        }
      }
      if (*(volatile uint32_t*)a.status & kStTimeout) b = 1;
      misc[1] = b;
    }
    __syncthreads();
    if (misc[1]) break;
    // every CTA has read the previous update's totals: CTA 0 clears them
    // for the update three ahead
    if (cta == 0 && pass >= 1) {
      unsigned long long* gp = a.gacc + (size_t)((pass - 1) % kGridRefineBufs) * stride;
      for (int e = tid; e < prev_used * DA; e += kT) gp[e] = 0ull;
    }
    prev_used = A;
    evals += (unsigned long long)A * (unsigned long long)a.n;
    ++iters;
    for (int e = tid; e < A; e += kT) {
      const int i = alist[e];
      double tot[DA];
#pragma unroll
      for (int k = 0; k < DA; ++k) tot[k] = (double)(long long)__ldcg(g + (size_t)e * DA + k) * a.inv_fx;
      const double W = tot[0];
      if (cta == 0) a.mscore[i] = W;
      bool ok = W > 0.0 && isfinite(W);
      const double rW = ok ? 1.0 / W : 0.0;   // one FP64 division per mode
      double step2 = 0.0, dl[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        dl[k] = ok ? tot[1 + k] * rW - (sym[i * D + k] - (double)sy[i * D + k]) : 0.0;
        step2 += dl[k] * dl[k];
      }
      if (ok && a.sphere_r > 0.0) {
        // cosine metric: the FP64 position projected back onto the sphere
        double pp[D], nn = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          pp[k] = sym[i * D + k] + dl[k];
          nn += pp[k] * pp[k];
        }
        const double f = a.sphere_r / sqrt(nn);
        step2 = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          pp[k] *= f;
          dl[k] = pp[k] - sym[i * D + k];
          step2 += dl[k] * dl[k];
        }
        ok = nn > 0.0 && isfinite(step2);
        if (ok) {
#pragma unroll
          for (int k = 0; k < D; ++k) {
            sym[i * D + k] = pp[k];
            sy[i * D + k] = (float)pp[k];
          }
        }
      } else if (ok) {
#pragma unroll
        for (int k = 0; k < D; ++k) {
          sym[i * D + k] += dl[k];
          sy[i * D + k] = (float)sym[i * D + k];
        }
      }
      if (!ok || step2 <= a.tol2_s) sact[i] = 0;
    }
    __syncthreads();
  }
  if (cta == 0) {
    for (int e = tid; e < M * D; e += kT) {
      const int i = e / D, k = e - i * D;
      a.ym[(int64_t)i * DP + k] = sym[i * D + k];
      a.yf[(int64_t)i * DP + k] = sy[i * D + k];
    }
    if (tid == 0) {
      atomicMax(a.iters_out, iters);
      if (evals) atomicAdd(a.evals, evals);
    }
  }
}

namespace {

template <int D, int DP, int DA, int KF, bool RES>
cudaError_t launch_grid_t(const GridRoundArgs& a, int G, int smem_bytes, cudaStream_t st) {
  auto kern = ms_grid_round_kernel<D, DP, DA, KF, RES>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kGridThreads);
  cfg.dynamicSmemBytes = (size_t)smem_bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <int D, int DP, int DA, int KF, bool RES>
int occupancy_t(int smem_bytes) {
  auto kern = ms_grid_round_kernel<D, DP, DA, KF, RES>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, kGridThreads, smem_bytes) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return b;
}

int accumulators_of(int d) { return d == 1 ? 2 : (d <= 3 ? 4 : 8); }

}  // namespace

GridPlan grid_round_plan(int64_t n, int d, int sms, int max_iter) {
  GridPlan p{};
  if (d < 1 || d > 7 || sms < 1 || n < 1 || n > INT32_MAX || max_iter >= kGridHist) return p;
  const int DP = d <= 4 ? 4 : 8, DA = accumulators_of(d);
  p.G = sms;
  p.per_cta = (int)((n + sms - 1) / sms);
  p.n_sub = (p.per_cta + kGridSubLen - 1) / kGridSubLen;
  if (p.n_sub < 1) p.n_sub = 1;
  p.sub_len = ((p.per_cta + p.n_sub - 1) / p.n_sub + 31) / 32 * 32;
  int dev_max = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return GridPlan{};
  const int with_pts = grid_smem(d, DA, DP, p.per_cta).total;
  const int without = grid_smem(d, DA, DP, 0).total;
  if (with_pts <= dev_max) {
    p.resident = 1;
    p.smem = with_pts;
  } else if (without <= dev_max) {
    p.resident = 0;
    p.smem = without;
  } else {
    return GridPlan{};
  }
  int bits = 0;
  while ((1LL << bits) <= n) ++bits;
  p.fx_bits = 62 - bits;
  // one CTA of this size must fit on every SM (the cooperative launch needs
  // the whole grid resident)
  int occ = 0;
#define FMS_GRID_OCC(D_, DP_, DA_)                                                        \
  occ = p.resident ? occupancy_t<D_, DP_, DA_, kKernelGaussian, true>(p.smem)            \
                   : occupancy_t<D_, DP_, DA_, kKernelGaussian, false>(p.smem)
  switch (d) {
    case 1: FMS_GRID_OCC(1, 4, 2); break;
    case 2: FMS_GRID_OCC(2, 4, 4); break;
    case 3: FMS_GRID_OCC(3, 4, 4); break;
    case 4: FMS_GRID_OCC(4, 4, 8); break;
    case 5: FMS_GRID_OCC(5, 8, 8); break;
    case 6: FMS_GRID_OCC(6, 8, 8); break;
    case 7: FMS_GRID_OCC(7, 8, 8); break;
  }
#undef FMS_GRID_OCC
  if (occ < 1) return GridPlan{};
  p.seeds = grid_seed_cap(DA);
  p.ok = 1;
  return p;
}

size_t grid_scratch_bytes(int d) {
  // barrier counter (256 bytes) + kGridBufs accumulators [seed capacity][DA] u64
  const int DA = accumulators_of(d);
  return 256 + (size_t)kGridBufs * grid_seed_cap(DA) * DA * 8;
}

size_t grid_scratch_clear_bytes(int d) {
  // everything starts at zero (each accumulator is cleared again after use)
  return grid_scratch_bytes(d);
}

namespace {

template <int D, int DP, int DA, int KF, bool RES>
cudaError_t launch_refine_grid_t(const GridRefineArgs& a, int G, int smem_bytes, cudaStream_t st) {
  auto kern = ms_grid_refine_kernel<D, DP, DA, KF, RES>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kGridRefineWarps * 32, smem_bytes);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorCooperativeLaunchTooLarge;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kGridRefineWarps * 32);
  cfg.dynamicSmemBytes = (size_t)smem_bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

}  // namespace

int grid_refine_capacity() { return kGridRefineModes; }

cudaError_t launch_ms_grid_refine(const GridPlan& p, const float* Xs, int64_t n, int d,
                                  const float* y, const int32_t* kept, const int32_t* accepted,
                                  const int32_t* M_ptr, double* ym, float* yf, double* mscore,
                                  double tol2_s, int max_iter, int32_t* iters_out,
                                  unsigned long long* evals, uint32_t* status, void* scratch,
                                  cudaStream_t st, int kf, double sphere_r) {
  if (!p.ok) return cudaErrorInvalidValue;
  const int DP = d <= 4 ? 4 : 8, DA = accumulators_of(d);
  // the accumulators reuse the round's scratch (256-byte counter + buffers)
  if ((size_t)kGridRefineBufs * kGridRefineModes * DA * 8 + 256 > grid_scratch_bytes(d))
    return cudaErrorInvalidValue;
  int dev_max = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return cudaErrorInvalidValue;
  const int with_pts = refine_smem(d, DP, p.per_cta).total;
  const bool resident = with_pts <= dev_max;
  const int smem = resident ? with_pts : refine_smem(d, DP, 0).total;
  GridRefineArgs a{};
  a.Xs = Xs;
  a.n = (int)n;
  a.per_cta = p.per_cta;
  a.n_sub = p.n_sub;
  a.sub_len = p.sub_len;
  a.y = y;
  a.kept = kept;
  a.accepted = accepted;
  a.M_ptr = M_ptr;
  a.ym = ym;
  a.yf = yf;
  a.mscore = mscore;
  a.tol2_s = tol2_s;
  a.max_iter = max_iter;
  a.iters_out = iters_out;
  a.evals = evals;
  a.gbar = reinterpret_cast<unsigned*>(scratch);
  a.gacc = reinterpret_cast<unsigned long long*>(static_cast<char*>(scratch) + 256);
  a.status = status;
  a.fx_scale = ldexpf(1.0f, p.fx_bits);
  a.inv_fx = ldexp(1.0, -p.fx_bits);
  a.sphere_r = sphere_r;
  cudaError_t e = cudaMemsetAsync(
      scratch, 0, 256 + (size_t)kGridRefineBufs * kGridRefineModes * DA * 8, st);
  if (e != cudaSuccess) return e;
#define FMS_GRID_REF(D_, DP_, DA_)                                                                      \
  if (kf == kKernelFlat)                                                                                \
    return resident ? launch_refine_grid_t<D_, DP_, DA_, kKernelFlat, true>(a, p.G, smem, st)           \
                    : launch_refine_grid_t<D_, DP_, DA_, kKernelFlat, false>(a, p.G, smem, st);         \
  return resident ? launch_refine_grid_t<D_, DP_, DA_, kKernelGaussian, true>(a, p.G, smem, st)         \
                  : launch_refine_grid_t<D_, DP_, DA_, kKernelGaussian, false>(a, p.G, smem, st)
  switch (d) {
    case 1: FMS_GRID_REF(1, 4, 2);
    case 2: FMS_GRID_REF(2, 4, 4);
    case 3: FMS_GRID_REF(3, 4, 4);
    case 4: FMS_GRID_REF(4, 4, 8);
    case 5: FMS_GRID_REF(5, 8, 8);
    case 6: FMS_GRID_REF(6, 8, 8);
    case 7: FMS_GRID_REF(7, 8, 8);
  }
#undef FMS_GRID_REF
  return cudaErrorInvalidValue;
}

cudaError_t launch_ms_grid_round(const GridPlan& p, int d, int kf, GridRoundArgs a,
                                 void* scratch, cudaStream_t st) {
  if (!p.ok) return cudaErrorInvalidValue;
  a.per_cta = p.per_cta;
  a.n_sub = p.n_sub;
  a.sub_len = p.sub_len;
  a.gbar = reinterpret_cast<unsigned*>(scratch);
  a.gacc = reinterpret_cast<unsigned long long*>(static_cast<char*>(scratch) + 256);
  a.fx_scale = ldexpf(1.0f, p.fx_bits);
  a.inv_fx_scale = ldexpf(1.0f, -p.fx_bits);
  cudaError_t e = cudaMemsetAsync(scratch, 0, grid_scratch_clear_bytes(d), st);
  if (e != cudaSuccess) return e;
#define FMS_GRID(D_, DP_, DA_)                                                              \
  if (kf == kKernelFlat)                                                                    \
    return p.resident ? launch_grid_t<D_, DP_, DA_, kKernelFlat, true>(a, p.G, p.smem, st)  \
                      : launch_grid_t<D_, DP_, DA_, kKernelFlat, false>(a, p.G, p.smem, st); \
  return p.resident ? launch_grid_t<D_, DP_, DA_, kKernelGaussian, true>(a, p.G, p.smem, st) \
                    : launch_grid_t<D_, DP_, DA_, kKernelGaussian, false>(a, p.G, p.smem, st)
  switch (d) {
    case 1: FMS_GRID(1, 4, 2);
    case 2: FMS_GRID(2, 4, 4);
    case 3: FMS_GRID(3, 4, 4);
    case 4: FMS_GRID(4, 4, 8);
    case 5: FMS_GRID(5, 8, 8);
    case 6: FMS_GRID(6, 8, 8);
    case 7: FMS_GRID(7, 8, 8);
  }
#undef FMS_GRID
  return cudaErrorInvalidValue;
}

}  // namespace fms
