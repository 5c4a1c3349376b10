// Prune (mode merging), the seed-count decision, FP64-accumulated refinement,
// canonical ordering and nearest-mode labelling.
#include <float.h>

#include "fms_prune_body.cuh"

namespace fms {

// ---------------------------------------------------------------------------
// Kept seeds after Early Stopping (Sec. II-C): converged by the stop update
// t* (gamma < 1), or every seed that did not fail (gamma = 1, Alg. 1).
// One CTA; slot order (= seed rank order) is preserved.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
    kept_list_kernel(const IterCtl* __restrict__ ctl, const int32_t* __restrict__ state,
                     const int32_t* __restrict__ conv, int keep_exhausted,
                     int32_t* __restrict__ kept, MergeCtl* mctl, int64_t n, int32_t R, Tiling tl,
                     const float* __restrict__ wlast, float* __restrict__ score) {
  __shared__ int scratch[64];
  const int N = ctl->N;
  const int t_star = ctl->r;
  int base = 0;
  for (int b = 0; b < N; b += blockDim.x) {
    const int i = b + threadIdx.x;
    int take = 0;
    if (i < N) {
      const int st = state[i];
      if (keep_exhausted) take = (st == kConverged) || (st == kExhausted);
      else take = (st == kConverged) && (conv[i] <= t_star);
    }
    int tot;
    const int off = block_exclusive_scan(take, &tot, scratch);
    if (take) {
      kept[base + off] = i;
      if (wlast) score[base + off] = wlast[i];
    }
    base += tot;
  }
  if (threadIdx.x == 0) {
    mctl->K = base;
    mctl->t_star = t_star;
    int C, Lc;
    choose_chunks(n, base, R, tl, &C, &Lc);
    mctl->C = C;
    mctl->Lc = Lc;
    if (!wlast) mctl->evals += (int64_t)base * n;   // the density pass the host then runs
  }
}

cudaError_t launch_kept_list(const IterCtl* ctl, const int32_t* state, const int32_t* conv,
                             int keep_exhausted, int32_t* kept, MergeCtl* mctl, int64_t n,
                             int32_t R, Tiling tl, cudaStream_t st, const float* wlast,
                             float* score) {
  kept_list_kernel<<<1, 1024, 0, st>>>(ctl, state, conv, keep_exhausted, kept, mctl, n, R, tl,
                                       wlast, score);
  return cudaGetLastError();
}

// score[q] = sum over chunks of the W partials of candidate q (one warp per
// candidate: lane l takes chunks l, l+32, ... in order, then a fixed xor tree).
__global__ void score_reduce_kernel(const float* __restrict__ part, const MergeCtl* mctl, int DA,
                                    float* __restrict__ score) {
  const int K = mctl->K, C = mctl->C;
  const int lane = threadIdx.x & 31;
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < K; q += nw) {
    float s = 0.0f;
    for (int c = lane; c < C; c += 32) s += part[((int64_t)c * K + q) * DA];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if (lane == 0) score[q] = s;
  }
}

cudaError_t launch_score_reduce(const float* part, const MergeCtl* mctl, int DA, float* score,
                                int max_K, cudaStream_t st) {
  int blocks = (max_K + 7) / 8;
  if (blocks < 1) blocks = 1;
  if (blocks > 4096) blocks = 4096;
  score_reduce_kernel<<<blocks, 256, 0, st>>>(part, mctl, DA, score);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The prune of Alg. 1 and Alg. 2: greedy radius
// suppression in order of (score descending, rank ascending).  Candidate q has
// rank q.  The sorted visit (fms_prune_body.cuh) is used while its sort keys fit
// in shared memory; larger candidate sets take the one-block global greedy.
// ---------------------------------------------------------------------------
template <typename PT, typename ST>
__global__ void __launch_bounds__(512)
    greedy_merge_kernel(const int32_t* __restrict__ cand_row, const int32_t* __restrict__ K_ptr,
                        const ST* __restrict__ score, const PT* __restrict__ pos, int DP, int d,
                        PT r2, int32_t* __restrict__ list, int32_t* __restrict__ accepted,
                        int32_t* __restrict__ M_out) {
  __shared__ __align__(16) unsigned char sm[greedy_global_smem<PT, ST>()];
  greedy_global_body<PT, ST>(cand_row, *K_ptr, score, pos, DP, d, r2, list, accepted, M_out, sm);
}

// ---------------------------------------------------------------------------
// The greedy visit on the whole GPU, for candidate sets whose sort keys do not
// fit one CTA (FP32 scores): one cooperative CTA per SM holds a contiguous
// share of the candidates in shared memory (coordinates, a 64-bit key whose
// unsigned order is the visit order -- score bits mapped to an unsigned order,
// the complemented candidate index below them -- and an alive flag).  Per
// accepted mode: every CTA posts its best alive key with one atomicMax into a
// winner slot; after one grid barrier (bounded) every CTA reads the winner,
// drops its candidates closer than r to it (the same FP32 distance as the
// one-block visit), and posts its next best into the next slot.  Three slots
// rotate; CTA 0 clears the one every CTA has finished reading.  The winners,
// in order, are the one-by-one greedy visit's accepted modes.
// ---------------------------------------------------------------------------
constexpr int kGridGreedyThreads = 512;
constexpr long long kGridGreedySpin = 4000000000LL;   // bound of one barrier wait (~2 s)

__device__ __forceinline__ unsigned long long greedy_key(float f, int q) {
  if (!(f == f)) f = -INFINITY;   // a NaN score counts as -inf (as in the sorted visit)
  if (f == 0.0f) f = 0.0f;        // -0 and +0 are equal scores
  unsigned u = __float_as_uint(f);
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return ((unsigned long long)u << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)q);
}

// bytes of shared memory for `per` candidates of DPC staged coordinates
__host__ __device__ inline size_t grid_greedy_smem(int per, int DPC) {
  return (((size_t)per * DPC * 4 + 15) / 16) * 16 + (size_t)per * 8 + (((size_t)per + 15) / 16) * 16;
}

template <int DPC>
__global__ void __launch_bounds__(kGridGreedyThreads, 1)
    greedy_grid_kernel(const int32_t* __restrict__ cand_row, const int32_t* __restrict__ K_ptr,
                       const float* __restrict__ score, const float* __restrict__ pos, int DP,
                       int d, float r2, int per, unsigned* gbar, unsigned long long* slots,
                       int32_t* __restrict__ accepted, int32_t* __restrict__ M_out,
                       uint32_t* status) {
  extern __shared__ __align__(16) unsigned char gsm[];
  __shared__ unsigned long long red[32];
  __shared__ float wpos[DPC];
  __shared__ int s_stop;
  float* spos = reinterpret_cast<float*>(gsm);
  unsigned long long* skey =
      reinterpret_cast<unsigned long long*>(gsm + (((size_t)per * DPC * 4 + 15) / 16) * 16);
  unsigned char* salive = reinterpret_cast<unsigned char*>(skey + per);
  const int K = *K_ptr;
  const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int q0 = min(K, cta * per), nq = max(0, min(K, q0 + per) - q0);
  unsigned long long best = 0ull;
  for (int e = tid; e < nq; e += kGridGreedyThreads) {
    const int q = q0 + e;
    const int64_t row = cand_row ? (int64_t)cand_row[q] : (int64_t)q;
#pragma unroll
    for (int k = 0; k < DPC; ++k) spos[(size_t)e * DPC + k] = k < d ? pos[row * DP + k] : 0.0f;
    const unsigned long long key = greedy_key(score[q], q);
    skey[e] = key;
    salive[e] = 1;
    best = key > best ? key : best;
  }
  auto block_max = [&](unsigned long long v) -> unsigned long long {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      const unsigned long long u = __shfl_xor_sync(kFull, v, o);
      v = u > v ? u : v;
    }
    if (lane == 0) red[warp] = v;
    __syncthreads();
    unsigned long long m = 0ull;
    for (int w = 0; w < kGridGreedyThreads / 32; ++w) m = red[w] > m ? red[w] : m;
    __syncthreads();
    return m;
  };
  // grid barrier number b (1, 2, ...): all CTAs have posted into the slot
  // that follows; false when the bounded wait gave up
  auto grid_barrier = [&](unsigned b) -> bool {
    if (tid == 0) {
      int stop = 0;
      __threadfence();
      asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(gbar), "r"(1u) : "memory");
      const unsigned want = (unsigned)G * b;
      const long long t0 = clock64();
      for (int it = 0;; ++it) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(gbar) : "memory");
        if (v >= want) break;
        if ((it & 31) == 31) {
          if (*(volatile uint32_t*)status & kStTimeout) {
            stop = 1;
            break;
          }
          if (clock64() - t0 > kGridGreedySpin) {
            atomicOr(status, kStTimeout);
            stop = 1;
            break;
          }
        }
      }
      s_stop = stop;
    }
    __syncthreads();
    return s_stop == 0;
  };
  best = block_max(best);
  if (tid == 0 && best) atomicMax(&slots[0], best);
  int it = 0;
  bool ok = grid_barrier(1u);
  while (ok) {
    unsigned long long W;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(W) : "l"(&slots[it % 3]) : "memory");
    if (W == 0ull) break;   // no alive candidate anywhere
    const int win = (int)(0xFFFFFFFFu - (unsigned)(W & 0xFFFFFFFFull));
    if (cta == 0 && tid == 0) accepted[it] = win;
    const int64_t wrow = cand_row ? (int64_t)cand_row[win] : (int64_t)win;
    if (tid < d) wpos[tid] = pos[wrow * DP + tid];
    __syncthreads();
    unsigned long long b = 0ull;
    for (int e = tid; e < nq; e += kGridGreedyThreads) {
      if (!salive[e]) continue;
      bool keep = q0 + e != win;
      if (keep) {
        float d2 = 0.0f;
        for (int k = 0; k < d; ++k) {
          const float dd = spos[(size_t)e * DPC + k] - wpos[k];
          d2 += dd * dd;
        }
        keep = !(d2 < r2);
      }
      if (keep) b = skey[e] > b ? skey[e] : b;
      else salive[e] = 0;
    }
    b = block_max(b);
    if (tid == 0) {
      if (b) atomicMax(&slots[(it + 1) % 3], b);
      if (cta == 0) slots[(it + 2) % 3] = 0ull;   // read by every CTA before the last barrier
    }
    ++it;
    ok = grid_barrier((unsigned)it + 1u);
  }
  if (cta == 0 && tid == 0) *M_out = it;
}

template <int DPC>
static cudaError_t launch_grid_greedy_t(const int32_t* cand_row, const int32_t* K_ptr,
                                        const float* score, const float* pos, int DP, int d,
                                        float r2, int per, int G, size_t sm, unsigned* gbar,
                                        unsigned long long* slots, int32_t* accepted,
                                        int32_t* M_out, uint32_t* status, cudaStream_t st) {
  auto kern = greedy_grid_kernel<DPC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kGridGreedyThreads, sm);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorCooperativeLaunchTooLarge;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kGridGreedyThreads);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, cand_row, K_ptr, score, pos, DP, d, r2, per, gbar, slots,
                            accepted, M_out, status);
}

// The grid visit for up to max_K FP32-scored candidates; its barrier counter
// and winner slots live in the first 64 bytes of `scratch` (cleared here).
// Returns cudaErrorInvalidValue when the candidates do not fit.
static cudaError_t launch_greedy_grid(const int32_t* cand_row, const int32_t* K_ptr,
                                      const float* score, const float* pos, int DP, int d,
                                      float r2, int32_t* scratch, int32_t* accepted,
                                      int32_t* M_out, int max_K, uint32_t* status,
                                      cudaStream_t st) {
  int dev = 0, sms = 0, dev_max = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
          cudaSuccess || sms < 1)
    return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(scratch) & 15u) != 0) return cudaErrorInvalidValue;
  const int DPC = d <= 4 ? 4 : (d <= 8 ? 8 : (d <= 16 ? 16 : (d <= 32 ? 32 : 64)));
  const int per = (max_K + sms - 1) / sms;
  const size_t sm = grid_greedy_smem(per > 0 ? per : 1, DPC);
  if (sm > (size_t)dev_max - 2048) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(scratch, 0, 64, st);
  if (e != cudaSuccess) return e;
  unsigned* gbar = reinterpret_cast<unsigned*>(scratch);
  unsigned long long* slots = reinterpret_cast<unsigned long long*>(scratch + 4);   // 16-byte offset
  switch (DPC) {
    case 4: return launch_grid_greedy_t<4>(cand_row, K_ptr, score, pos, DP, d, r2, per, sms, sm, gbar, slots, accepted, M_out, status, st);
    case 8: return launch_grid_greedy_t<8>(cand_row, K_ptr, score, pos, DP, d, r2, per, sms, sm, gbar, slots, accepted, M_out, status, st);
    case 16: return launch_grid_greedy_t<16>(cand_row, K_ptr, score, pos, DP, d, r2, per, sms, sm, gbar, slots, accepted, M_out, status, st);
    case 32: return launch_grid_greedy_t<32>(cand_row, K_ptr, score, pos, DP, d, r2, per, sms, sm, gbar, slots, accepted, M_out, status, st);
    default: return launch_grid_greedy_t<64>(cand_row, K_ptr, score, pos, DP, d, r2, per, sms, sm, gbar, slots, accepted, M_out, status, st);
  }
}

// DT > 0: d = DT at compile time (candidates in registers during the visit)
template <typename PT, typename ST, int DT>
__global__ void __launch_bounds__(1024)
    greedy_sorted_kernel(const int32_t* __restrict__ cand_row, const int32_t* __restrict__ K_ptr,
                         const ST* __restrict__ score, const PT* __restrict__ pos, int DP, int d,
                         PT r2, int32_t* __restrict__ accepted, int32_t* __restrict__ M_out,
                         int P, int acc_in_smem, int preload) {
  extern __shared__ __align__(16) unsigned char smem[];
  greedy_sorted_body<PT, ST, DT>(cand_row, *K_ptr, score, pos, DP, DT > 0 ? DT : d, r2, accepted,
                                 M_out, P, smem, acc_in_smem != 0, preload != 0);
}

template <typename PT, typename ST, int DT>
static cudaError_t launch_sorted_t(const int32_t* cand_row, const int32_t* K_ptr, const ST* score,
                                   const PT* pos, int DP, int d, PT r2, int32_t* accepted,
                                   int32_t* M_out, int P, int with_pos, int preload, size_t sm,
                                   int smem_max, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(greedy_sorted_kernel<PT, ST, DT>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
    attr = true;
  }
  greedy_sorted_kernel<PT, ST, DT><<<1, 1024, sm, st>>>(cand_row, K_ptr, score, pos, DP, d, r2,
                                                        accepted, M_out, P, with_pos, preload);
  return cudaGetLastError();
}

// Shared memory of the sorted prune for up to K candidates: sort keys and
// indices, the batch tiles, plus (preload) every candidate's coordinates and
// (with_pos) the accepted modes' coordinates.
template <typename PT, typename ST>
size_t greedy_sorted_bytes(int K, int d, int* P_out, bool with_pos, bool preload) {
  int P = 1;
  while (P < K) P <<= 1;
  *P_out = P;
  return greedy_sorted_smem<PT, ST>(K, d, P, with_pos, preload);
}

constexpr size_t kGreedySmemMax = 200 * 1024;

// The sorted prune (coordinates in shared memory when they fit, else read
// from global memory); the one-block global greedy only when even the sort
// keys do not fit.
template <typename PT, typename ST>
cudaError_t launch_greedy(const int32_t* cand_row, const int32_t* K_ptr, const ST* score,
                          const PT* pos, int DP, int d, PT r2, int32_t* alive,
                          int32_t* accepted, int32_t* M_out, int max_K, cudaStream_t st,
                          uint32_t* status = nullptr) {
  // largest layout that fits: preloaded candidates and accepted modes in
  // shared memory, then accepted modes only, then neither
  int P = 1;
  int with_pos = 1, preload = 1;
  size_t sm = greedy_sorted_bytes<PT, ST>(max_K, d, &P, true, true);
  if (sm > kGreedySmemMax) {
    preload = 0;
    sm = greedy_sorted_bytes<PT, ST>(max_K, d, &P, true, false);
  }
  if (sm > kGreedySmemMax) {
    sm = greedy_sorted_bytes<PT, ST>(max_K, d, &P, false, false);
    with_pos = 0;
  }
  if (sm <= kGreedySmemMax && d <= kPruneMaxDim) {
    const int mx = (int)kGreedySmemMax;
#define FMS_SORTED(DT_)                                                                      \
  return launch_sorted_t<PT, ST, DT_>(cand_row, K_ptr, score, pos, DP, d, r2, accepted, M_out, \
                                      P, with_pos, preload, sm, mx, st)
    if (preload && with_pos) switch (d) {
        case 1: FMS_SORTED(1);
        case 2: FMS_SORTED(2);
        case 3: FMS_SORTED(3);
        case 4: FMS_SORTED(4);
        case 5: FMS_SORTED(5);
        case 6: FMS_SORTED(6);
        case 7: FMS_SORTED(7);
        case 8: FMS_SORTED(8);
      }
    FMS_SORTED(0);
#undef FMS_SORTED
  }
  if constexpr (sizeof(ST) == 4 && sizeof(PT) == 4) {
    // FP32 scores: the visit on the whole GPU when its shares fit
    if (status && launch_greedy_grid(cand_row, K_ptr, score, pos, DP, d, r2, alive, accepted,
                                     M_out, max_K, status, st) == cudaSuccess)
      return cudaSuccess;
    cudaGetLastError();   // (a refused grid launch leaves no error behind)
  }
  greedy_merge_kernel<PT, ST><<<1, 512, 0, st>>>(cand_row, K_ptr, score, pos, DP, d, r2, alive,
                                                  accepted, M_out);
  return cudaGetLastError();
}

cudaError_t launch_greedy_merge_f(const int32_t* cand_row, const int32_t* K_ptr,
                                  const float* score, const float* pos, int DP, int d, float r2,
                                  int32_t* alive, int32_t* accepted, int32_t* M_out, int max_K,
                                  cudaStream_t st, uint32_t* status) {
  return launch_greedy<float, float>(cand_row, K_ptr, score, pos, DP, d, r2, alive, accepted,
                                     M_out, max_K, st, status);
}

cudaError_t launch_greedy_merge_d(const int32_t* K_ptr, const double* score, const double* pos,
                                  int DP, int d, double r2, int32_t* alive, int32_t* accepted,
                                  int32_t* M_out, int max_K, cudaStream_t st) {
  return launch_greedy<double, double>(nullptr, K_ptr, score, pos, DP, d, r2, alive, accepted,
                                       M_out, max_K, st);
}

// Seed-count control (Sec. II-D): double N while N < L*M (and N < n).
__global__ void doubling_kernel(MergeCtl* mctl, int32_t N, int64_t n, float L, int allow) {
  const int M = mctl->M;
  int next = N;
  if (allow && (float)N < L * (float)M && (int64_t)N < n) {
    const int64_t t = 2LL * N;
    next = (int32_t)(t < n ? t : n);
  }
  mctl->next_N = next;
}

cudaError_t launch_doubling_decision(MergeCtl* mctl, int32_t N, int64_t n, float L, int allow,
                                     cudaStream_t st) {
  doubling_kernel<<<1, 1, 0, st>>>(mctl, N, n, L, allow);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Refinement: more updates of each merged mode, run by ms_step on the FP32
// rounding yf of an FP64 position ym.  With S, W the FP32 chunk partials
// against yf, summed over chunks in FP64, the update is
//   ym <- ym + S/W - (ym - yf)        (= m(yf), in FP64)
// so positions keep FP64 resolution and the convergence test
// ||step|| <= 1e-5*h is taken in FP64.  At most 50 updates per mode.
// ---------------------------------------------------------------------------
__global__ void refine_setup_kernel(const float* __restrict__ y, const int32_t* __restrict__ kept,
                                    const int32_t* __restrict__ accepted, const int32_t* M_ptr,
                                    int DP, double* __restrict__ ym, float* __restrict__ yf,
                                    int32_t* __restrict__ active, int32_t* __restrict__ mdone,
                                    IterCtl* rctl, int init_pos, int64_t n, int32_t R, Tiling tl) {
  const int M = *M_ptr;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M * DP; e += gridDim.x * blockDim.x) {
    const int m = e / DP, k = e % DP;
    if (init_pos) {
      const float v = y[(int64_t)kept[accepted[m]] * DP + k];
      ym[e] = (double)v;
      yf[e] = v;
    }
    if (k == 0) {
      active[m] = m;
      if (init_pos) mdone[m] = 0;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int C = 0, Lc = 0;
    choose_chunks(n, M, R, tl, &C, &Lc);
    rctl->s = M;
    rctl->C = C;
    rctl->Lc = Lc;
    rctl->r = 0;
    rctl->done = M > 0 ? 0 : 1;
    rctl->N = M;
    rctl->blocks_done = 0;
    if (init_pos) rctl->steps = 0;
  }
}

cudaError_t launch_refine_setup(const float* y, const int32_t* kept, const int32_t* accepted,
                                const int32_t* M_ptr, int DP, double* ym, float* yf,
                                int32_t* active, int32_t* mdone, IterCtl* rctl, int init_pos,
                                int64_t n, int32_t R, Tiling tl, int max_M, cudaStream_t st) {
  int blocks = (max_M * DP + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 1024) blocks = 1024;
  refine_setup_kernel<<<blocks, 256, 0, st>>>(y, kept, accepted, M_ptr, DP, ym, yf, active, mdone,
                                              rctl, init_pos, n, R, tl);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256)
    refine_update_kernel(const float* __restrict__ part, int32_t* __restrict__ active,
                         IterCtl* rctl, double* __restrict__ ym, float* __restrict__ yf,
                         int32_t* __restrict__ mdone, double* __restrict__ mscore, int d, int DP,
                         int DA, double tol2_s, int max_iter, int64_t n,
                         int32_t R, Tiling tl, double sphere_r) {
  __shared__ int scratch[64];
  __shared__ int sh_last;
  __shared__ double red[8][96];
  if (__ldcg(&rctl->done)) return;
  const int s = __ldcg(&rctl->s), C = __ldcg(&rctl->C);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // many chunks: one block per mode, its 8 warps split the chunks (warp sums
  // added in warp order); else one warp per mode
  const bool block_mode = C >= kBlockReduceChunks;
  const int nw = block_mode ? gridDim.x : gridDim.x * (blockDim.x >> 5);
  const int c0 = block_mode ? wid : 0, cs = block_mode ? 8 : 1;
  for (int p = block_mode ? blockIdx.x : blockIdx.x * (blockDim.x >> 5) + wid; p < s; p += nw) {
    const int m = __ldcg(active + p);
    // lane l sums chunks c0 + cs*l, c0 + cs*(l+32), ... in FP64; fixed xor
    // tree; lane k keeps accumulator k (W for k = 0, S_{k-1} otherwise)
    double a[3] = {0.0, 0.0, 0.0};
    for (int k0 = 0; k0 <= d; k0 += 4) {
      double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
      if ((DA & 3) == 0) {
        for (int c = c0 + cs * lane; c < C; c += 32 * cs) {
          const float4 q = __ldcg(reinterpret_cast<const float4*>(part + ((int64_t)c * s + p) * DA + k0));
          v0 += (double)q.x;
          v1 += (double)q.y;
          v2 += (double)q.z;
          v3 += (double)q.w;
        }
      } else {
        for (int c = c0 + cs * lane; c < C; c += 32 * cs) {
          const float2 q = __ldcg(reinterpret_cast<const float2*>(part + ((int64_t)c * s + p) * DA));
          v0 += (double)q.x;
          v1 += (double)q.y;
        }
      }
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        v0 += __shfl_xor_sync(kFull, v0, o);
        v1 += __shfl_xor_sync(kFull, v1, o);
        v2 += __shfl_xor_sync(kFull, v2, o);
        v3 += __shfl_xor_sync(kFull, v3, o);
      }
      const double vals[4] = {v0, v1, v2, v3};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k = k0 + e;
        if (k <= d && (k & 31) == lane) a[k >> 5] = vals[e];
      }
    }
    if (block_mode) {
#pragma unroll
      for (int u = 0; u < 3; ++u) red[wid][lane + 32 * u] = a[u];
      __syncthreads();
      if (wid == 0) {
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          double t = red[0][lane + 32 * u];
          for (int w = 1; w < 8; ++w) t += red[w][lane + 32 * u];
          a[u] = t;
        }
      }
      __syncthreads();
      if (wid != 0) continue;
    }
    const double W = __shfl_sync(kFull, a[0], 0);
    // the mode's density: sum w of its latest update (the last one is at most
    // the refinement tolerance before the refined mode)
    if (lane == 0) mscore[m] = W;
    const bool ok = W > 0.0 && isfinite(W);
    double step2 = 0.0, delta[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int k = lane + 32 * u;
      if (ok && k >= 1 && k <= d) {
        const int64_t e = (int64_t)m * DP + (k - 1);
        delta[u] = a[u] / W - (ym[e] - (double)yf[e]);
        step2 += delta[u] * delta[u];
      }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) step2 += __shfl_xor_sync(kFull, step2, o);
    bool good = ok;
    if (ok && sphere_r > 0.0) {
      // cosine metric: the FP64 position scaled back onto the sphere
      double pv[3] = {0.0, 0.0, 0.0}, nn = 0.0;
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int k = lane + 32 * u;
        if (k >= 1 && k <= d) {
          pv[u] = ym[(int64_t)m * DP + (k - 1)] + delta[u];
          nn += pv[u] * pv[u];
        }
      }
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) nn += __shfl_xor_sync(kFull, nn, o);
      const double f = sphere_r / sqrt(nn);
      step2 = 0.0;
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int k = lane + 32 * u;
        if (k >= 1 && k <= d) {
          const int64_t e = (int64_t)m * DP + (k - 1);
          pv[u] *= f;
          const double dd = pv[u] - ym[e];
          step2 += dd * dd;
        }
      }
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) step2 += __shfl_xor_sync(kFull, step2, o);
      good = nn > 0.0 && isfinite(step2);
      if (good) {
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          const int k = lane + 32 * u;
          if (k >= 1 && k <= d) {
            const int64_t e = (int64_t)m * DP + (k - 1);
            ym[e] = pv[u];
            yf[e] = (float)pv[u];
          }
        }
      }
    } else if (ok) {
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int k = lane + 32 * u;
        if (k >= 1 && k <= d) {
          const int64_t e = (int64_t)m * DP + (k - 1);
          const double v = ym[e] + delta[u];
          ym[e] = v;
          yf[e] = (float)v;
        }
      }
    }
    if (lane == 0 && (!good || step2 <= tol2_s)) mdone[m] = 1;
  }
  // last block: the modes still moving take the next update
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) sh_last = (atomicAdd(&rctl->blocks_done, 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!sh_last) return;
  __threadfence();
  const int M = __ldcg(&rctl->N);
  int base = 0;
  for (int b0 = 0; b0 < M; b0 += blockDim.x) {
    const int m = b0 + threadIdx.x;
    const int take = (m < M && !__ldcg(mdone + m)) ? 1 : 0;
    int tot;
    const int off = block_exclusive_scan(take, &tot, scratch);
    if (take) active[base + off] = m;
    base += tot;
  }
  if (threadIdx.x == 0) {
    const int r = __ldcg(&rctl->r) + 1;
    const int done = (base == 0) || (r >= max_iter);
    rctl->r = r;
    rctl->steps = r;
    rctl->done = done;
    rctl->s = done ? 0 : base;
    int Cn = 0, Lcn = 0;
    if (!done) choose_chunks(n, base, R, tl, &Cn, &Lcn);
    rctl->C = Cn;
    rctl->Lc = Lcn;
    if (!done) rctl->evals += (int64_t)base * n;
    rctl->blocks_done = 0;
  }
}

cudaError_t launch_refine_update(const float* part, int32_t* active, IterCtl* rctl, double* ym,
                                 float* yf, int32_t* mdone, double* mscore, int d, int DP, int DA,
                                 double tol2_s, int max_iter, int64_t n, int32_t R,
                                 Tiling tl, int max_M, cudaStream_t st, double sphere_r) {
  int blocks = max_M;  // one block per mode (many chunks) or one warp per mode
  if (blocks < 1) blocks = 1;
  if (blocks > 1216) blocks = 1216;
  refine_update_kernel<<<blocks, 256, 0, st>>>(part, active, rctl, ym, yf, mdone, mscore, d, DP,
                                               DA, tol2_s, max_iter, n, R, tl,
                                               sphere_r);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Canonical order: score descending, ties by lexicographic coordinates.
// rank_i = #{j : key_j < key_i}; modes are written in original units.
// ---------------------------------------------------------------------------
template <typename PT>
__device__ __forceinline__ bool key_less(double sa, const PT* a, double sb, const PT* b, int d) {
  if (sa != sb) return sa > sb;
  for (int k = 0; k < d; ++k)
    if (a[k] != b[k]) return a[k] < b[k];
  return false;
}

__global__ void canonical_order_kernel(const double* __restrict__ ym,
                                       const double* __restrict__ mscore,
                                       const int32_t* __restrict__ accepted,
                                       const int32_t* __restrict__ M_ptr, int d, int DP,
                                       double inv_scale, float* __restrict__ out_modes,
                                       int32_t max_modes, float* __restrict__ modes_full,
                                       float* __restrict__ out_scores) {
  // the modes' scores are staged in shared memory (one load each instead of a
  // dependent load per comparison); coordinates are read only on equal scores
  constexpr int kStage = 1024;
  __shared__ double s_sc[kStage];
  const int M = *M_ptr;
  const bool staged = M <= kStage;
  if (staged) {
    for (int j = threadIdx.x; j < M; j += blockDim.x) s_sc[j] = mscore[accepted ? accepted[j] : j];
    __syncthreads();
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    const int ai = accepted ? accepted[i] : i;
    const double* pa = ym + (int64_t)ai * DP;
    const double sa = mscore[ai];
    int rank = 0;
    for (int j = 0; j < M; ++j) {
      if (j == i) continue;
      const double sj = staged ? s_sc[j] : mscore[accepted ? accepted[j] : j];
      if (sj != sa) {
        rank += sj > sa ? 1 : 0;
      } else {
        const int aj = accepted ? accepted[j] : j;
        if (key_less(sj, ym + (int64_t)aj * DP, sa, pa, d)) ++rank;
      }
    }
    for (int k = 0; k < d; ++k) {
      const float v = (float)(pa[k] * inv_scale);
      modes_full[(int64_t)rank * d + k] = v;
      if (out_modes && rank < max_modes) out_modes[(int64_t)rank * d + k] = v;
    }
    if (out_scores) out_scores[rank] = (float)sa;
  }
}

cudaError_t launch_canonical_order(const double* ym, const double* mscore,
                                   const int32_t* accepted, const int32_t* M_ptr, int d, int DP,
                                   double inv_scale, float* out_modes, int32_t max_modes,
                                   float* modes_full, float* out_scores, int max_M,
                                   cudaStream_t st) {
  int blocks = (max_M + 127) / 128;
  if (blocks < 1) blocks = 1;
  if (blocks > 1024) blocks = 1024;
  canonical_order_kernel<<<blocks, 128, 0, st>>>(ym, mscore, accepted, M_ptr, d, DP, inv_scale,
                                                 out_modes, max_modes, modes_full, out_scores);
  return cudaGetLastError();
}

// Positions of the accepted seeds (no refinement): FP64 copies + FP64 scores
// from the FP32 prune scores, so the same ordering kernel applies.
__global__ void unrefined_modes_kernel(const float* __restrict__ y,
                                       const int32_t* __restrict__ kept,
                                       const int32_t* __restrict__ accepted,
                                       const float* __restrict__ score, const MergeCtl* mctl,
                                       int DP, double* __restrict__ ym,
                                       double* __restrict__ mscore) {
  const int M = mctl->M;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M * DP; e += gridDim.x * blockDim.x) {
    const int m = e / DP, k = e % DP;
    const int q = accepted[m];
    ym[e] = (double)y[(int64_t)kept[q] * DP + k];
    if (k == 0) mscore[m] = (double)score[q];
  }
}

cudaError_t launch_unrefined_modes(const float* y, const int32_t* kept, const int32_t* accepted,
                                   const float* score, const MergeCtl* mctl, int DP, double* ym,
                                   double* mscore, int max_M, cudaStream_t st) {
  int blocks = (max_M * DP + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 1024) blocks = 1024;
  unrefined_modes_kernel<<<blocks, 256, 0, st>>>(y, kept, accepted, score, mctl, DP, ym, mscore);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Nearest-mode labels (the labelling of Alg. 2).  One thread per point; modes are
// staged through shared memory in tiles.  Ties go to the lowest index.
// ---------------------------------------------------------------------------
constexpr int kLabelTileFloats = 8192;

// DT > 0: the dimension at compile time (coordinates in registers); DT = 0:
// any d <= FMS_MAX_DIM_PAD, read at run time.
template <int DT>
__global__ void __launch_bounds__(256)
    label_kernel(const float* __restrict__ X, int64_t n, int d_arg, const float* __restrict__ modes,
                 const int32_t* __restrict__ M_ptr, int M_host, int32_t* __restrict__ labels,
                 float* __restrict__ margins, int unit) {
  constexpr int DX = DT > 0 ? DT : FMS_MAX_DIM_PAD;
  const int d = DT > 0 ? DT : d_arg;
  __shared__ float sm[kLabelTileFloats];
  const int M = M_ptr ? *M_ptr : M_host;
  const int tile = kLabelTileFloats / d;
  for (int64_t jb = (int64_t)blockIdx.x * blockDim.x; jb < n; jb += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = jb + threadIdx.x;
    float x[DX];
    if (j < n) {
#pragma unroll
      for (int k = 0; k < DX; ++k)
        if (k < d) x[k] = X[j * d + k];
      if (unit) {
        // cosine metric: the point's direction (in FP64, as the packing)
        double nn = 0.0;
#pragma unroll
        for (int k = 0; k < DX; ++k)
          if (k < d) nn += (double)x[k] * (double)x[k];
        const double f = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
#pragma unroll
        for (int k = 0; k < DX; ++k)
          if (k < d) x[k] = (float)((double)x[k] * f);
      }
    }
    float b1 = INFINITY, b2 = INFINITY;
    int arg = -1;
    for (int m0 = 0; m0 < M; m0 += tile) {
      const int mt = min(tile, M - m0);
      __syncthreads();
      for (int e = threadIdx.x; e < mt * d; e += blockDim.x) sm[e] = modes[(int64_t)m0 * d + e];
      __syncthreads();
      if (j < n) {
        for (int m = 0; m < mt; ++m) {
          float d2 = 0.0f;
#pragma unroll
          for (int k = 0; k < DX; ++k)
            if (k < d) {
              const float e = x[k] - sm[m * d + k];
              d2 = fmaf(e, e, d2);
            }
          if (d2 < b1) {
            b2 = b1;
            b1 = d2;
            arg = m0 + m;
          } else if (d2 < b2) {
            b2 = d2;
          }
        }
      }
    }
    if (j < n) {
      labels[j] = arg;
      if (margins) margins[j] = (M > 1) ? sqrtf(b2) - sqrtf(b1) : INFINITY;
    }
  }
}

cudaError_t launch_label(const float* X, int64_t n, int d, const float* modes,
                         const int32_t* M_dev, int32_t M_host, int32_t* labels, float* margins,
                         cudaStream_t st, int unit) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  switch (d) {
#define FMS_LABEL(D_)                                                                           \
  case D_:                                                                                      \
    label_kernel<D_><<<(int)blocks, 256, 0, st>>>(X, n, d, modes, M_dev, M_host, labels, margins, unit); \
    break;
    FMS_LABEL(1)
    FMS_LABEL(2)
    FMS_LABEL(3)
    FMS_LABEL(4)
    FMS_LABEL(5)
    FMS_LABEL(6)
    FMS_LABEL(7)
    FMS_LABEL(8)
#undef FMS_LABEL
    default:
      label_kernel<0><<<(int)blocks, 256, 0, st>>>(X, n, d, modes, M_dev, M_host, labels, margins,
                                                  unit);
  }
  return cudaGetLastError();
}

}  // namespace fms
