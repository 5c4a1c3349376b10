// Batched Faster Mean-shift: many independent point sets in every launch.
//
// Every phase of the single-set global path runs once for all sets: set b
// owns points [p0_b, p0_b + n_b) of the concatenated (packed) point array and
// seed slots [p0_b, p0_b + n_b) of the seed arrays (its lists -- active seeds,
// kept seeds, accepted modes, refined modes -- also start at p0_b).  Per-set
// control blocks (SetCtl) hold each set's clock, counts and chunking; a plan
// (prefix sums over sets of warp tasks, partial-sum blocks and list entries)
// lets one launch of the step / update kernels map a global task or list
// index to (set, local index) by binary search.  One CTA per set runs the
// per-set bookkeeping (compaction under the Early Stopping clock rule, kept
// list, prune, ordering); the last CTA to finish (atomic ticket, no waiting)
// rebuilds the plan for the next launch.  The whole call runs as one CUDA
// graph: the compaction, advance and refinement kernels decide on the device,
// through conditional-node handles, whether another update, another seed round
// or another refinement update follows.
#include "fms_prune_body.cuh"
#include "fms_seedperm.cuh"
#include "fms_step_body.cuh"

namespace fms {

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------
enum PlanKind : int { kPlanActive = 0, kPlanKept = 1, kPlanModes = 2 };

// (fields read through L2: other blocks of the same launch may have just
// written them)
__device__ __forceinline__ void plan_counts(const SetCtl& c, int kind, int* cnt, int* C, int* Lc) {
  if (kind == kPlanActive) {
    *cnt = __ldcg(&c.done) ? 0 : __ldcg(&c.s);
    *C = __ldcg(&c.C);
    *Lc = __ldcg(&c.Lc);
  } else if (kind == kPlanKept) {
    *cnt = __ldcg(&c.final_) ? 0 : __ldcg(&c.K);
    *C = __ldcg(&c.Ck);
    *Lc = __ldcg(&c.Lck);
  } else {
    *cnt = __ldcg(&c.rdone) ? 0 : __ldcg(&c.rs);
    *C = __ldcg(&c.rC);
    *Lc = __ldcg(&c.rLc);
  }
}

// Prefix sums over sets: task_off (warp tasks), part_off (floats of partial
// sums), list_off (list entries); totals in plan[0..1].  One block.
__device__ void build_plan(const SetCtl* __restrict__ sc, int B, int kind, int R, int DA,
                           int64_t* __restrict__ task_off, int64_t* __restrict__ part_off,
                           int64_t* __restrict__ list_off, int64_t* __restrict__ totals) {
  // serial over blocks of 1024 sets with a block scan (B is at most a few thousand)
  __shared__ int64_t carry[3];
  __shared__ int64_t wsum[3][32];
  if (threadIdx.x == 0) carry[0] = carry[1] = carry[2] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int b0 = 0; b0 < B; b0 += blockDim.x) {
    const int b = b0 + threadIdx.x;
    int64_t v[3] = {0, 0, 0};
    if (b < B) {
      int cnt, C, Lc;
      plan_counts(sc[b], kind, &cnt, &C, &Lc);
      if (cnt > 0 && C > 0) {
        const int64_t G = (cnt + R - 1) / R;
        v[0] = G * C;
        v[1] = (int64_t)C * cnt * DA;
        v[2] = cnt;
      }
    }
    int64_t inc[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      int64_t x = v[q];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
      }
      inc[q] = x;
      if (lane == 31) wsum[q][wid] = x;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        int64_t x = lane < nwarp ? wsum[q][lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int64_t y = __shfl_up_sync(kFull, x, o);
          if (lane >= o) x += y;
        }
        wsum[q][lane] = x;
      }
    }
    __syncthreads();
    if (b < B) {
      const int64_t base0 = carry[0] + (wid ? wsum[0][wid - 1] : 0) + inc[0] - v[0];
      const int64_t base1 = carry[1] + (wid ? wsum[1][wid - 1] : 0) + inc[1] - v[1];
      const int64_t base2 = carry[2] + (wid ? wsum[2][wid - 1] : 0) + inc[2] - v[2];
      task_off[b] = base0;
      part_off[b] = base1;
      list_off[b] = base2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      carry[0] += wsum[0][nwarp - 1];
      carry[1] += wsum[1][nwarp - 1];
      carry[2] += wsum[2][nwarp - 1];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    task_off[B] = carry[0];
    part_off[B] = carry[1];
    list_off[B] = carry[2];
    totals[0] = carry[0];
    totals[1] = carry[2];
  }
}

// a kernel given cond.on sets cond.h to "more work follows" when it finishes
__device__ __forceinline__ void set_cond(const BatchCond& cond, bool more,
                                         const uint32_t* status) {
  if (cond.on) {
    const bool ok = !(__ldcg(status) & kStNonFinite);   // stop early on bad input
    cudaGraphSetConditional(cond.h, (more && ok) ? 1u : 0u);
  }
}

__global__ void __launch_bounds__(1024)
    plan_kernel(const SetCtl* sc, int B, int kind, int R, int DA, int64_t* task_off,
                int64_t* part_off, int64_t* list_off, int64_t* totals, BatchCond cond,
                const uint32_t* status) {
  build_plan(sc, B, kind, R, DA, task_off, part_off, list_off, totals);
  if (threadIdx.x == 0) set_cond(cond, totals[1] > 0, status);
}

__device__ __forceinline__ int find_set(const int64_t* __restrict__ off, int B, int64_t x) {
  int lo = 0, hi = B - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// seeds
// ---------------------------------------------------------------------------
// the seeds of every set: the keyed permutation of fms_seedperm.cuh over the
// set's own points (its half width depends on the set's size)
struct BFeistel {
  uint64_t k[6];
};

__device__ __forceinline__ int64_t bpermute(int64_t r, int64_t n, const BFeistel& b) {
  FeistelKey f;
#pragma unroll
  for (int q = 0; q < 6; ++q) f.k[q] = b.k[q];
  f.hb = feistel_half_bits(n);
  return permute(r, n, f);
}

// New seeds of every set: ranks [prevN, N) -> slots p0 + rank.  A set whose
// prune result is final keeps its seeds.
__global__ void batched_seed_init(SetCtl* sc, int B, const float* __restrict__ Xs, int DP,
                                  BFeistel f, float* __restrict__ y, int32_t* __restrict__ it,
                                  int32_t* __restrict__ conv, int32_t* __restrict__ state) {
  for (int b = blockIdx.x; b < B; b += gridDim.x) {
    const SetCtl c = sc[b];
    if (c.final_) continue;
    for (int r = c.prevN + threadIdx.x; r < c.N; r += blockDim.x) {
      const int64_t idx = c.p0 + bpermute(r, c.n, f);
      const int64_t slot = c.p0 + r;
      for (int k = 0; k < DP; ++k) y[slot * DP + k] = Xs[idx * DP + k];
      it[slot] = 0;
      conv[slot] = -1;
      state[slot] = kRunning;
    }
  }
}

// ---------------------------------------------------------------------------
// Early Stopping bookkeeping per set (the clock rule of the single-set path)
// and the plan of the next update.  One CTA per set; last CTA plans.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
    batched_compact(SetCtl* sc, int B, const int32_t* __restrict__ state,
                    const int32_t* __restrict__ it, const int32_t* __restrict__ conv,
                    int32_t* __restrict__ active, int begin, int max_iter, int R, int DA,
                    Tiling tl, int64_t* task_off, int64_t* part_off, int64_t* list_off,
                    int64_t* totals, int32_t* counters, BatchCond cond,
                    const uint32_t* status) {
  __shared__ int scratch[64];
  __shared__ int sh_last;
  int32_t* blocks_done = counters + kCtrBlocksDone;
  const int b = blockIdx.x;
  SetCtl* c = sc + b;
  if (begin && c->final_) {
    if (threadIdx.x == 0) {
      c->done = 1;
      c->s = 0;
      c->C = 0;
    }
  } else if (begin || !__ldcg(&c->done)) {
    const int N = c->N, p0 = c->p0, target = c->target;
    int r = begin ? 0 : __ldcg(&c->r) + 1;
    const int prev_s = begin ? 0 : __ldcg(&c->s);
    int s = 0, convd = 0, nxt = INT32_MAX, done = 0;
    for (int guard = 0; guard <= max_iter + 2; ++guard) {
      int base = 0;
      convd = 0;
      nxt = INT32_MAX;
      for (int b0 = 0; b0 < N; b0 += blockDim.x) {
        const int i = b0 + threadIdx.x;
        int take = 0;
        if (i < N) {
          const int64_t slot = p0 + i;
          const int st = __ldcg(state + slot);
          if (st == kRunning) {
            const int ti = __ldcg(it + slot);
            if (ti == r) take = 1;
            else if (ti > r) nxt = min(nxt, ti);
          } else if (st == kConverged) {
            const int ci = __ldcg(conv + slot);
            if (ci <= r) ++convd;
            else nxt = min(nxt, ci);
          }
        }
        int tot;
        const int off = block_exclusive_scan(take, &tot, scratch);
        if (take) active[p0 + base + off] = p0 + i;
        base += tot;
      }
      convd = block_sum(convd, scratch);
      nxt = block_min(nxt, scratch);
      s = base;
      done = (convd >= target) || (r >= max_iter);
      if (!done && s == 0) {
        r = (nxt == INT32_MAX || nxt > max_iter) ? max_iter : nxt;
        continue;
      }
      break;
    }
    if (threadIdx.x == 0) {
      c->r = r;
      c->done = done;
      c->n_conv = convd;
      if (prev_s > 0) c->steps += 1;
      c->s = done ? 0 : s;
      int C = 0, Lc = 0;
      if (!done) choose_chunks(c->n, s, R, tl, &C, &Lc);
      c->C = C;
      c->Lc = Lc;
      if (!done) c->evals += (int64_t)s * c->n;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) sh_last = (atomicAdd(blocks_done, 1) == B - 1);
  __syncthreads();
  if (!sh_last) return;
  __threadfence();
  build_plan(sc, B, kPlanActive, R, DA, task_off, part_off, list_off, totals);
  if (threadIdx.x == 0) {
    *blocks_done = 0;
    if (!begin) counters[kCtrUpdates] += 1;
    set_cond(cond, totals[1] > 0, status);
  }
}

// ---------------------------------------------------------------------------
// step: one launch over the warp tasks of every set
// ---------------------------------------------------------------------------
template <int D, int DP, int DA>
__global__ void __launch_bounds__(256)
    batched_step_lowd(const float* __restrict__ Xs, const float* __restrict__ y,
                      const int32_t* __restrict__ list, const SetCtl* __restrict__ sc, int B,
                      int kind, const int64_t* __restrict__ task_off,
                      const int64_t* __restrict__ part_off, const int64_t* __restrict__ totals,
                      float* __restrict__ part) {
  constexpr int R = 32 / DA;
  const int64_t T = totals[0];
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < T; t += nw) {
    const int b = find_set(task_off, B, t);
    const SetCtl& c = sc[b];
    int cnt, C, Lc;
    plan_counts(c, kind, &cnt, &C, &Lc);
    const int64_t local = t - task_off[b];
    const int G = (cnt + R - 1) / R;
    const int g = (int)(local % G), ch = (int)(local / G);
    const int j0 = ch * Lc, j1 = min(c.n, j0 + Lc);
    lowd_task<D, DP, DA>(Xs + (int64_t)c.p0 * DP, j0, j1, y, list + c.p0, cnt, g, ch,
                         part + part_off[b], lane);
  }
}

template <int DPAD, int RG>
__global__ void __launch_bounds__(128)
    batched_step_wide(const float* __restrict__ Xs, const float* __restrict__ y,
                      const int32_t* __restrict__ list, const SetCtl* __restrict__ sc, int B,
                      int kind, const int64_t* __restrict__ task_off,
                      const int64_t* __restrict__ part_off, const int64_t* __restrict__ totals,
                      float* __restrict__ part, uint32_t* __restrict__ status) {
  extern __shared__ __align__(16) float wide_tiles[];
  __shared__ __align__(8) uint64_t wide_bars[4][2];
  constexpr int SPW = 32 * RG;
  const int64_t T = totals[0];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t* bars = wide_bars[warp];
  float* tiles = wide_tiles + warp * 2 * kWideTile * DPAD;
  tc::ring_init(bars, lane);
  uint32_t use0 = 0u, use1 = 0u;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; t < T; t += nw) {
    const int b = find_set(task_off, B, t);
    const SetCtl& c = sc[b];
    int cnt, C, Lc;
    plan_counts(c, kind, &cnt, &C, &Lc);
    const int64_t local = t - task_off[b];
    const int G = (cnt + SPW - 1) / SPW;
    const int g = (int)(local % G), ch = (int)(local / G);
    const int j0 = ch * Lc, j1 = min(c.n, j0 + Lc);
    if (!wide_task<DPAD, RG>(Xs + (int64_t)c.p0 * DPAD, j0, j1, y, list + c.p0, cnt, g, ch,
                             part + part_off[b], lane, 0, tiles, bars, use0, use1, status))
      break;
  }
}

template <int DPAD, int RG>
static void launch_bwide(int grid, const float* Xs, const float* y, const int32_t* list,
                         const SetCtl* sc, int B, int kind, const int64_t* task_off,
                         const int64_t* part_off, const int64_t* totals, float* part,
                         uint32_t* status, cudaStream_t st) {
  static bool attr = false;
  if (!attr && wide_smem_bytes<DPAD>() > 48 * 1024) {
    cudaFuncSetAttribute(batched_step_wide<DPAD, RG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         wide_smem_bytes<DPAD>());
    attr = true;
  }
  batched_step_wide<DPAD, RG><<<grid, 128, wide_smem_bytes<DPAD>(), st>>>(
      Xs, y, list, sc, B, kind, task_off, part_off, totals, part, status);
}

cudaError_t launch_batched_step(const float* Xs, int d, int DP, const float* y,
                                const int32_t* list, const SetCtl* sc, int B, int kind,
                                const int64_t* task_off, const int64_t* part_off,
                                const int64_t* totals, float* part, int target_warps,
                                uint32_t* status, cudaStream_t st) {
  const int g = (target_warps + 7) / 8;
  if (d > 7 && DP != padded_dim(d)) return cudaErrorInvalidValue;   // rows of the compiled width
  switch (d) {
    case 1: batched_step_lowd<1, 4, 2><<<g, 256, 0, st>>>(Xs, y, list, sc, B, kind, task_off, part_off, totals, part); break;
    case 2: batched_step_lowd<2, 4, 4><<<g, 256, 0, st>>>(Xs, y, list, sc, B, kind, task_off, part_off, totals, part); break;
    case 3: batched_step_lowd<3, 4, 4><<<g, 256, 0, st>>>(Xs, y, list, sc, B, kind, task_off, part_off, totals, part); break;
    case 4: batched_step_lowd<4, 4, 8><<<g, 256, 0, st>>>(Xs, y, list, sc, B, kind, task_off, part_off, totals, part); break;
    case 5: batched_step_lowd<5, 8, 8><<<g, 256, 0, st>>>(Xs, y, list, sc, B, kind, task_off, part_off, totals, part); break;
    case 6: batched_step_lowd<6, 8, 8><<<g, 256, 0, st>>>(Xs, y, list, sc, B, kind, task_off, part_off, totals, part); break;
    case 7: batched_step_lowd<7, 8, 8><<<g, 256, 0, st>>>(Xs, y, list, sc, B, kind, task_off, part_off, totals, part); break;
    default:
      if (d <= 8) launch_bwide<8, 4>(2 * g, Xs, y, list, sc, B, kind, task_off, part_off, totals, part, status, st);
      else if (d <= 16) launch_bwide<16, 2>(2 * g, Xs, y, list, sc, B, kind, task_off, part_off, totals, part, status, st);
      else if (d <= 32) launch_bwide<32, 1>(2 * g, Xs, y, list, sc, B, kind, task_off, part_off, totals, part, status, st);
      else launch_bwide<64, 1>(2 * g, Xs, y, list, sc, B, kind, task_off, part_off, totals, part, status, st);
      break;
  }
  return cudaGetLastError();
}

// Cross-chunk sums of list entry p of a set (lanes over chunks, fixed tree);
// lane k ends with accumulator k in a[k >> 5].
__device__ __forceinline__ void bsum_chunks(const float* __restrict__ part, int s, int p, int C,
                                            int DA, int d, int lane, float (&a)[3]) {
  for (int k0 = 0; k0 <= d; k0 += 4) {
    float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f;
    for (int c = lane; c < C; c += 32) {
      const float* q = part + ((int64_t)c * s + p) * DA + k0;
      if ((DA & 3) == 0) {
        const float4 t = __ldcg(reinterpret_cast<const float4*>(q));
        v0 += t.x;
        v1 += t.y;
        v2 += t.z;
        v3 += t.w;
      } else {
        const float2 t = __ldcg(reinterpret_cast<const float2*>(q));
        v0 += t.x;
        v1 += t.y;
      }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      v0 += __shfl_xor_sync(kFull, v0, o);
      v1 += __shfl_xor_sync(kFull, v1, o);
      v2 += __shfl_xor_sync(kFull, v2, o);
      v3 += __shfl_xor_sync(kFull, v3, o);
    }
    const float vals[4] = {v0, v1, v2, v3};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int k = k0 + e;
      if (k <= d && (k & 31) == lane) a[k >> 5] = vals[e];
    }
  }
}

// update of every active seed of every set (one warp per list entry)
__global__ void __launch_bounds__(256)
    batched_update(const float* __restrict__ part, const int32_t* __restrict__ active,
                   const SetCtl* __restrict__ sc, int B, const int64_t* __restrict__ list_off,
                   const int64_t* __restrict__ part_off, const int64_t* __restrict__ totals,
                   float* __restrict__ y, int32_t* __restrict__ it, int32_t* __restrict__ conv,
                   int32_t* __restrict__ state, int d, int DP, int DA, float tol2_s,
                   int max_iter) {
  const int64_t total = totals[1];
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < total;
       q += nw) {
    const int b = find_set(list_off, B, q);
    const SetCtl& c = sc[b];
    const int p = (int)(q - list_off[b]);
    const int64_t slot = active[c.p0 + p];
    float a[3] = {0.f, 0.f, 0.f};
    bsum_chunks(part + part_off[b], c.s, p, c.C, DA, d, lane, a);
    const float W = __shfl_sync(kFull, a[0], 0);
    float step2 = 0.f, delta[3] = {0.f, 0.f, 0.f};
    const bool ok = (W > 0.f) && isfinite(W);
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int k = lane + 32 * u;
      if (ok && k >= 1 && k <= d) {
        delta[u] = a[u] / W;
        step2 = fmaf(delta[u], delta[u], step2);
      }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) step2 += __shfl_xor_sync(kFull, step2, o);
    const bool finite = ok && isfinite(step2);
    if (finite) {
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int k = lane + 32 * u;
        if (k >= 1 && k <= d) y[slot * DP + (k - 1)] += delta[u];
      }
    }
    if (lane == 0) {
      const int t = it[slot] + 1;
      it[slot] = t;
      if (!finite) state[slot] = kFailed;
      else if (step2 <= tol2_s) {
        state[slot] = kConverged;
        conv[slot] = t;
      } else if (t >= max_iter) state[slot] = kExhausted;
    }
  }
}

// ---------------------------------------------------------------------------
// prune: kept lists, density pass reduce, sorted prune, doubling decision
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
    batched_kept(SetCtl* sc, int B, const int32_t* __restrict__ state,
                 const int32_t* __restrict__ conv, int keep_exhausted, int32_t* __restrict__ kept,
                 int R, int DA, Tiling tl, int64_t* task_off, int64_t* part_off,
                 int64_t* list_off, int64_t* totals, int32_t* counters) {
  __shared__ int scratch[64];
  __shared__ int sh_last;
  int32_t* blocks_done = counters + kCtrBlocksDone;
  const int b = blockIdx.x;
  SetCtl* c = sc + b;
  const int N = c->final_ ? 0 : c->N, p0 = c->p0, t_star = c->r;
  int base = 0;
  for (int b0 = 0; b0 < N; b0 += blockDim.x) {
    const int i = b0 + threadIdx.x;
    int take = 0;
    if (i < N) {
      const int st = __ldcg(state + p0 + i);
      take = keep_exhausted ? (st == kConverged || st == kExhausted)
                            : (st == kConverged && __ldcg(conv + p0 + i) <= t_star);
    }
    int tot;
    const int off = block_exclusive_scan(take, &tot, scratch);
    if (take) kept[p0 + base + off] = p0 + i;
    base += tot;
  }
  if (threadIdx.x == 0 && !c->final_) {
    c->K = base;
    c->t_star = t_star;
    int C = 0, Lc = 0;
    choose_chunks(c->n, base, R, tl, &C, &Lc);
    c->Ck = C;
    c->Lck = Lc;
    c->evals += (int64_t)base * c->n;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) sh_last = (atomicAdd(blocks_done, 1) == B - 1);
  __syncthreads();
  if (!sh_last) return;
  __threadfence();
  build_plan(sc, B, kPlanKept, R, DA, task_off, part_off, list_off, totals);
  if (threadIdx.x == 0) *blocks_done = 0;
}

// density at each kept seed: score[p0 + q] (one warp per kept seed)
__global__ void batched_score(const float* __restrict__ part, const SetCtl* __restrict__ sc, int B,
                              const int64_t* __restrict__ list_off,
                              const int64_t* __restrict__ part_off,
                              const int64_t* __restrict__ totals, int DA,
                              float* __restrict__ score) {
  const int64_t total = totals[1];
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < total;
       q += nw) {
    const int b = find_set(list_off, B, q);
    const SetCtl& c = sc[b];
    const int p = (int)(q - list_off[b]);
    const float* pb = part + part_off[b];
    float s = 0.f;
    for (int ch = lane; ch < c.Ck; ch += 32) s += __ldcg(pb + ((int64_t)ch * c.K + p) * DA);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if (lane == 0) score[c.p0 + p] = s;
  }
}

// Prune of each set (one CTA per set): the sorted visit while its sort keys
// (and, when they fit too, the accepted modes' coordinates) fit in the launch's
// smem_bytes of shared memory, else the one-block global greedy over the set's
// own region of `list`; both give the one-by-one greedy visit's result.
template <typename PT, typename ST>
__global__ void __launch_bounds__(1024)
    batched_prune(SetCtl* sc, const int32_t* __restrict__ kept, const ST* __restrict__ score,
                  const PT* __restrict__ pos, int DP, int d, PT r2, int32_t* __restrict__ accepted,
                  int32_t* __restrict__ list, int smem_bytes, int second) {
  extern __shared__ __align__(16) unsigned char smem[];
  SetCtl* c = sc + blockIdx.x;
  if (!second && c->final_) return;  // this set's prune result is already final
  const int p0 = c->p0;
  const int K = second ? c->M : c->K;
  // candidates: first prune -> kept seeds (rows = seed slots); second prune ->
  // refined modes (rows = mode slots p0 + m)
  const int32_t* rows = second ? nullptr : kept + p0;
  const PT* cpos = second ? pos + (int64_t)p0 * DP : pos;
  int32_t* M_out = second ? &c->Mr : &c->M;
  int P = 1;
  while (P < K) P <<= 1;
  if (greedy_sorted_smem<PT, ST>(K, d, P, false) <= (size_t)smem_bytes) {
    const bool acc_in_smem = greedy_sorted_smem<PT, ST>(K, d, P, true) <= (size_t)smem_bytes;
    greedy_sorted_body<PT, ST>(rows, K, score + p0, cpos, DP, d, r2, accepted + p0, M_out, P, smem,
                               acc_in_smem);
  } else {
    greedy_global_body<PT, ST>(rows, K, score + p0, cpos, DP, d, r2, list + p0, accepted + p0,
                               M_out, smem);
  }
}

// Seed-count decision of every set after its prune (Sec. II-D: double N while
// N < L*M and N < n) and the start of the next round for the sets that double
// (prevN <- N, N <- next N, target from gamma).  One CTA; it also counts the
// round and sets the round loop's condition: another round while any set doubles.
__global__ void __launch_bounds__(1024)
    batched_advance(SetCtl* sc, int B, float L, int allow, float gamma, int32_t* counters,
                    BatchCond cond, const uint32_t* status) {
  __shared__ int red[32];
  int any = 0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    SetCtl* c = sc + b;
    if (c->final_) continue;
    int next = c->N;
    if (allow && (float)c->N < L * (float)c->M && c->N < c->n) next = min(2 * c->N, c->n);
    c->next_N = next;
    if (next > c->N) {
      c->prevN = c->N;
      c->N = next;
      const int t = (int)ceil((double)gamma * (double)next);
      c->target = max(1, min(t, next));
      c->done = 0;
      any = 1;
    } else {
      c->final_ = 1;
    }
  }
  any = block_sum(any, red);
  if (threadIdx.x == 0) {
    counters[kCtrRounds] += 1;
    set_cond(cond, any > 0, status);
  }
}

// ---------------------------------------------------------------------------
// refinement (FP64 positions ym at mode slots p0 + m; yf = fl32(ym))
// ---------------------------------------------------------------------------
__global__ void batched_refine_setup(SetCtl* sc, int B, const float* __restrict__ y,
                                     const int32_t* __restrict__ kept,
                                     const int32_t* __restrict__ accepted, int DP,
                                     double* __restrict__ ym, float* __restrict__ yf,
                                     int32_t* __restrict__ ract, int32_t* __restrict__ mdone,
                                     int init_pos, int R, Tiling tl) {
  for (int b = blockIdx.x; b < B; b += gridDim.x) {
    SetCtl* c = sc + b;
    const int M = c->M, p0 = c->p0;
    for (int e = threadIdx.x; e < M * DP; e += blockDim.x) {
      const int m = e / DP, k = e % DP;
      const int64_t ms = (int64_t)p0 + m;
      if (init_pos) {
        const float v = y[(int64_t)kept[p0 + accepted[p0 + m]] * DP + k];
        ym[ms * DP + k] = (double)v;
        yf[ms * DP + k] = v;
      }
      if (k == 0) {
        ract[ms] = (int32_t)ms;
        if (init_pos) mdone[ms] = 0;
      }
    }
    if (threadIdx.x == 0) {
      int C = 0, Lc = 0;
      choose_chunks(c->n, M, R, tl, &C, &Lc);
      c->rs = M;
      c->rC = C;
      c->rLc = Lc;
      if (init_pos) c->rr = 0;
      c->rdone = M > 0 ? 0 : 1;
    }
  }
}

__global__ void __launch_bounds__(256)
    batched_refine_update(const float* __restrict__ part, const int32_t* __restrict__ ract,
                          const SetCtl* __restrict__ sc, int B,
                          const int64_t* __restrict__ list_off,
                          const int64_t* __restrict__ part_off,
                          const int64_t* __restrict__ totals, double* __restrict__ ym,
                          float* __restrict__ yf, int32_t* __restrict__ mdone,
                          double* __restrict__ mscore, int d, int DP, int DA, double tol2_s,
                          int score_only) {
  const int64_t total = totals[1];
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < total;
       q += nw) {
    const int b = find_set(list_off, B, q);
    const SetCtl& c = sc[b];
    const int p = (int)(q - list_off[b]);
    const int64_t ms = ract[c.p0 + p];
    const float* pb = part + part_off[b];
    double a[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k <= d; ++k) {
      double v = 0.0;
      for (int ch = lane; ch < c.rC; ch += 32) v += (double)__ldcg(pb + ((int64_t)ch * c.rs + p) * DA + k);
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
      if ((k & 31) == lane) a[k >> 5] = v;
    }
    const double W = __shfl_sync(kFull, a[0], 0);
    if (score_only) {
      if (lane == 0) mscore[ms] = W;
      continue;
    }
    const bool ok = W > 0.0 && isfinite(W);
    double step2 = 0.0, delta[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int k = lane + 32 * u;
      if (ok && k >= 1 && k <= d) {
        const int64_t e = ms * DP + (k - 1);
        delta[u] = a[u] / W - (ym[e] - (double)yf[e]);
        step2 += delta[u] * delta[u];
      }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) step2 += __shfl_xor_sync(kFull, step2, o);
    if (ok) {
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int k = lane + 32 * u;
        if (k >= 1 && k <= d) {
          const int64_t e = ms * DP + (k - 1);
          const double v = ym[e] + delta[u];
          ym[e] = v;
          yf[e] = (float)v;
        }
      }
    }
    if (lane == 0 && (!ok || step2 <= tol2_s)) mdone[ms] = 1;
  }
}

// modes still moving take the next refinement update (one CTA per set)
__global__ void __launch_bounds__(1024)
    batched_refine_compact(SetCtl* sc, int B, const int32_t* __restrict__ mdone,
                           int32_t* __restrict__ ract, int max_iter, int R, int DA, Tiling tl,
                           int64_t* task_off, int64_t* part_off, int64_t* list_off,
                           int64_t* totals, int32_t* counters, BatchCond cond,
                           const uint32_t* status) {
  __shared__ int scratch[64];
  __shared__ int sh_last;
  int32_t* blocks_done = counters + kCtrBlocksDone;
  SetCtl* c = sc + blockIdx.x;
  if (!__ldcg(&c->rdone)) {
    const int M = c->M, p0 = c->p0;
    int base = 0;
    for (int b0 = 0; b0 < M; b0 += blockDim.x) {
      const int m = b0 + threadIdx.x;
      const int take = (m < M && !__ldcg(mdone + p0 + m)) ? 1 : 0;
      int tot;
      const int off = block_exclusive_scan(take, &tot, scratch);
      if (take) ract[p0 + base + off] = p0 + m;
      base += tot;
    }
    if (threadIdx.x == 0) {
      const int r = c->rr + 1;
      const int done = (base == 0) || (r >= max_iter);
      c->rr = r;
      c->rdone = done;
      c->rs = done ? 0 : base;
      int C = 0, Lc = 0;
      if (!done) choose_chunks(c->n, base, R, tl, &C, &Lc);
      c->rC = C;
      c->rLc = Lc;
      if (!done) c->evals += (int64_t)base * c->n;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) sh_last = (atomicAdd(blocks_done, 1) == B - 1);
  __syncthreads();
  if (!sh_last) return;
  __threadfence();
  build_plan(sc, B, kPlanModes, R, DA, task_off, part_off, list_off, totals);
  if (threadIdx.x == 0) {
    *blocks_done = 0;
    counters[kCtrRefine] += 1;
    set_cond(cond, totals[1] > 0, status);
  }
}

// ---------------------------------------------------------------------------
// canonical order and labels
// ---------------------------------------------------------------------------
__global__ void batched_canonical(const SetCtl* __restrict__ sc, const double* __restrict__ ym,
                                  const double* __restrict__ mscore,
                                  const int32_t* __restrict__ acc2, int d, int DP,
                                  double inv_scale, float* __restrict__ out_modes, int max_modes,
                                  float* __restrict__ modes_full, int32_t* __restrict__ out_n) {
  const SetCtl& c = sc[blockIdx.x];
  const int M = c.Mr, p0 = c.p0;
  if (threadIdx.x == 0 && out_n) out_n[blockIdx.x] = M;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const int64_t ai = (int64_t)p0 + acc2[p0 + i];
    const double si = mscore[ai];
    const double* pi = ym + ai * DP;
    int rank = 0;
    for (int j = 0; j < M; ++j) {
      if (j == i) continue;
      const int64_t aj = (int64_t)p0 + acc2[p0 + j];
      const double sj = mscore[aj];
      bool less = false;
      if (sj != si) less = sj > si;
      else {
        const double* pj = ym + aj * DP;
        for (int k = 0; k < d; ++k)
          if (pj[k] != pi[k]) {
            less = pj[k] < pi[k];
            break;
          }
      }
      rank += less;
    }
    for (int k = 0; k < d; ++k) {
      const float v = (float)(pi[k] * inv_scale);
      modes_full[((int64_t)p0 + rank) * d + k] = v;
      if (out_modes && rank < max_modes)
        out_modes[((int64_t)blockIdx.x * max_modes + rank) * d + k] = v;
    }
  }
}

__global__ void __launch_bounds__(256)
    batched_label(const float* __restrict__ X, const int64_t* __restrict__ pt_off, int B, int d,
                  const SetCtl* __restrict__ sc, const float* __restrict__ modes_full,
                  int32_t* __restrict__ labels, float* __restrict__ margins, int64_t total) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < total;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int b = find_set(pt_off, B, j);
    const SetCtl& c = sc[b];
    const float* mb = modes_full + (int64_t)c.p0 * d;
    float b1 = INFINITY, b2 = INFINITY;
    int arg = -1;
    for (int m = 0; m < c.Mr; ++m) {
      float d2 = 0.f;
      for (int k = 0; k < d; ++k) {
        const float e = X[j * d + k] - mb[(int64_t)m * d + k];
        d2 = fmaf(e, e, d2);
      }
      if (d2 < b1) {
        b2 = b1;
        b1 = d2;
        arg = m;
      } else if (d2 < b2) {
        b2 = d2;
      }
    }
    labels[j] = arg;
    if (margins) margins[j] = c.Mr > 1 ? sqrtf(b2) - sqrtf(b1) : INFINITY;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static BFeistel bkey(uint64_t seed) {
  const FeistelKey k = make_key(1, seed);   // the round keys do not depend on n
  BFeistel f;
  for (int r = 0; r < 6; ++r) f.k[r] = k.k[r];
  return f;
}

cudaError_t launch_batched_seed_init(SetCtl* sc, int B, const float* Xs, int DP, uint64_t seed,
                                     float* y, int32_t* it, int32_t* conv, int32_t* state,
                                     cudaStream_t st) {
  batched_seed_init<<<B < 4096 ? B : 4096, 256, 0, st>>>(sc, B, Xs, DP, bkey(seed), y, it, conv,
                                                         state);
  return cudaGetLastError();
}

cudaError_t launch_batched_compact(SetCtl* sc, int B, const int32_t* state, const int32_t* it,
                                   const int32_t* conv, int32_t* active, int begin, int max_iter,
                                   int R, int DA, Tiling tl, int64_t* task_off, int64_t* part_off,
                                   int64_t* list_off, int64_t* totals, int32_t* counters,
                                   BatchCond cond, const uint32_t* status, cudaStream_t st) {
  batched_compact<<<B, 1024, 0, st>>>(sc, B, state, it, conv, active, begin, max_iter, R, DA, tl,
                                      task_off, part_off, list_off, totals, counters, cond,
                                      status);
  return cudaGetLastError();
}

cudaError_t launch_batched_update(const float* part, const int32_t* active, const SetCtl* sc,
                                  int B, const int64_t* list_off, const int64_t* part_off,
                                  const int64_t* totals, float* y, int32_t* it, int32_t* conv,
                                  int32_t* state, int d, int DP, int DA, float tol2_s,
                                  int max_iter, int grid, cudaStream_t st) {
  batched_update<<<grid, 256, 0, st>>>(part, active, sc, B, list_off, part_off, totals, y, it,
                                       conv, state, d, DP, DA, tol2_s, max_iter);
  return cudaGetLastError();
}

cudaError_t launch_batched_kept(SetCtl* sc, int B, const int32_t* state, const int32_t* conv,
                                int keep_exhausted, int32_t* kept, int R, int DA, Tiling tl,
                                int64_t* task_off, int64_t* part_off, int64_t* list_off,
                                int64_t* totals, int32_t* counters, cudaStream_t st) {
  batched_kept<<<B, 1024, 0, st>>>(sc, B, state, conv, keep_exhausted, kept, R, DA, tl, task_off,
                                   part_off, list_off, totals, counters);
  return cudaGetLastError();
}

cudaError_t launch_batched_score(const float* part, const SetCtl* sc, int B,
                                 const int64_t* list_off, const int64_t* part_off,
                                 const int64_t* totals, int DA, float* score, int grid,
                                 cudaStream_t st) {
  batched_score<<<grid, 256, 0, st>>>(part, sc, B, list_off, part_off, totals, DA, score);
  return cudaGetLastError();
}

// Shared memory of the per-set prune launch for sets of up to maxK candidates:
// the sorted visit's keys, indices, tiles and accepted coordinates when they
// fit in kBatchedPruneSmem, else kBatchedPruneSmem (sets whose keys do not fit
// take the global greedy).
template <typename PT, typename ST>
static size_t prune_launch_smem(int maxK, int d) {
  int P = 1;
  while (P < maxK) P <<= 1;
  size_t sm = greedy_sorted_smem<PT, ST>(maxK, d, P, true);
  if (sm > kBatchedPruneSmem) sm = kBatchedPruneSmem;
  if (sm < greedy_global_smem<PT, ST>()) sm = greedy_global_smem<PT, ST>();
  return sm;
}

template <typename PT, typename ST>
static cudaError_t launch_prune_t(SetCtl* sc, int B, const int32_t* kept, const ST* score,
                                  const PT* pos, int DP, int d, PT r2, int32_t* accepted,
                                  int32_t* list, int maxK, int second, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(
        batched_prune<PT, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchedPruneSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const size_t sm = prune_launch_smem<PT, ST>(maxK, d);
  batched_prune<PT, ST><<<B, 1024, sm, st>>>(sc, kept, score, pos, DP, d, r2, accepted, list,
                                             (int)sm, second);
  return cudaGetLastError();
}

cudaError_t launch_batched_prune_f(SetCtl* sc, int B, const int32_t* kept, const float* score,
                                   const float* pos, int DP, int d, float r2, int32_t* accepted,
                                   int32_t* list, int maxK, cudaStream_t st) {
  return launch_prune_t<float, float>(sc, B, kept, score, pos, DP, d, r2, accepted, list, maxK, 0,
                                      st);
}

cudaError_t launch_batched_prune_d(SetCtl* sc, int B, const double* score, const double* pos,
                                   int DP, int d, double r2, int32_t* accepted, int32_t* list,
                                   int maxK, cudaStream_t st) {
  return launch_prune_t<double, double>(sc, B, nullptr, score, pos, DP, d, r2, accepted, list,
                                        maxK, 1, st);
}

cudaError_t launch_batched_advance(SetCtl* sc, int B, float L, int allow, float gamma,
                                   int32_t* counters, BatchCond cond, const uint32_t* status,
                                   cudaStream_t st) {
  batched_advance<<<1, 1024, 0, st>>>(sc, B, L, allow, gamma, counters, cond, status);
  return cudaGetLastError();
}

cudaError_t launch_batched_refine_setup(SetCtl* sc, int B, const float* y, const int32_t* kept,
                                        const int32_t* accepted, int DP, double* ym, float* yf,
                                        int32_t* ract, int32_t* mdone, int init_pos, int R,
                                        Tiling tl, cudaStream_t st) {
  batched_refine_setup<<<B < 4096 ? B : 4096, 256, 0, st>>>(sc, B, y, kept, accepted, DP, ym, yf,
                                                            ract, mdone, init_pos, R, tl);
  return cudaGetLastError();
}

cudaError_t launch_plan(const SetCtl* sc, int B, int kind, int R, int DA, int64_t* task_off,
                        int64_t* part_off, int64_t* list_off, int64_t* totals, BatchCond cond,
                        const uint32_t* status, cudaStream_t st) {
  plan_kernel<<<1, 1024, 0, st>>>(sc, B, kind, R, DA, task_off, part_off, list_off, totals, cond,
                                  status);
  return cudaGetLastError();
}

cudaError_t launch_batched_refine_update(const float* part, const int32_t* ract, const SetCtl* sc,
                                         int B, const int64_t* list_off, const int64_t* part_off,
                                         const int64_t* totals, double* ym, float* yf,
                                         int32_t* mdone, double* mscore, int d, int DP, int DA,
                                         double tol2_s, int score_only, int grid,
                                         cudaStream_t st) {
  batched_refine_update<<<grid, 256, 0, st>>>(part, ract, sc, B, list_off, part_off, totals, ym,
                                              yf, mdone, mscore, d, DP, DA, tol2_s, score_only);
  return cudaGetLastError();
}

cudaError_t launch_batched_refine_compact(SetCtl* sc, int B, const int32_t* mdone, int32_t* ract,
                                          int max_iter, int R, int DA, Tiling tl,
                                          int64_t* task_off, int64_t* part_off, int64_t* list_off,
                                          int64_t* totals, int32_t* counters, BatchCond cond,
                                          const uint32_t* status, cudaStream_t st) {
  batched_refine_compact<<<B, 1024, 0, st>>>(sc, B, mdone, ract, max_iter, R, DA, tl, task_off,
                                             part_off, list_off, totals, counters, cond, status);
  return cudaGetLastError();
}

cudaError_t launch_batched_canonical(const SetCtl* sc, int B, const double* ym,
                                     const double* mscore, const int32_t* acc2, int d, int DP,
                                     double inv_scale, float* out_modes, int max_modes,
                                     float* modes_full, int32_t* out_n, cudaStream_t st) {
  batched_canonical<<<B, 256, 0, st>>>(sc, ym, mscore, acc2, d, DP, inv_scale, out_modes,
                                       max_modes, modes_full, out_n);
  return cudaGetLastError();
}

cudaError_t launch_batched_label(const float* X, const int64_t* pt_off, int B, int d,
                                 const SetCtl* sc, const float* modes_full, int32_t* labels,
                                 float* margins, int64_t total, cudaStream_t st) {
  int64_t blocks = (total + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  if (blocks < 1) blocks = 1;
  batched_label<<<(int)blocks, 256, 0, st>>>(X, pt_off, B, d, sc, modes_full, labels, margins,
                                             total);
  return cudaGetLastError();
}

}  // namespace fms
