// Point packing, Seed Selection, the per-update seed update and the
// Early-Stopping bookkeeping that compacts the active set.
#include "fms_internal.cuh"
#include "fms_seedperm.cuh"

namespace fms {

// ---------------------------------------------------------------------------
// Packing: Xs = s * X, padded to DP floats per row; flags non-finite input.
// Xcopy (nullable) receives the rows unchanged, for later passes over the
// original points (X may be host memory read over the CPU-GPU link).
// ---------------------------------------------------------------------------
__global__ void pack_points_kernel(const float* __restrict__ X, int64_t n, int d, int DP,
                                   float scale, float* __restrict__ Xs, uint32_t* status,
                                   float* __restrict__ Xcopy) {
  const int64_t total = n * DP;
  bool bad = false;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / DP;
    const int k = (int)(e - j * DP);
    float v = 0.0f;
    if (k < d) {
      v = X[j * d + k];
      if (Xcopy) Xcopy[j * d + k] = v;
      if (!isfinite(v)) bad = true;
      v *= scale;
    }
    Xs[e] = v;
  }
  if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kStNonFinite);
}

// DP = 4 or 8: one thread per point, the padded row written with vector stores
template <int DP>
__global__ void pack_rows_kernel(const float* __restrict__ X, int n, int d, float scale,
                                 float* __restrict__ Xs, uint32_t* status,
                                 float* __restrict__ Xcopy) {
  bool bad = false;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    float v[DP];
#pragma unroll
    for (int k = 0; k < DP; ++k) {
      v[k] = 0.0f;
      if (k < d) {
        const float x = X[(int64_t)j * d + k];
        if (Xcopy) Xcopy[(int64_t)j * d + k] = x;
        if (!isfinite(x)) bad = true;
        v[k] = x * scale;
      }
    }
    float4* o = reinterpret_cast<float4*>(Xs + (int64_t)j * DP);
#pragma unroll
    for (int q = 0; q < DP / 4; ++q) o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  }
  if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kStNonFinite);
}

// Cosine metric: row j scaled to unit length, then by s; a zero row flags
// kStBadArg (it has no direction), a non-finite one kStNonFinite.
__global__ void pack_unit_rows_kernel(const float* __restrict__ X, int64_t n, int d, int DP,
                                      float scale, float* __restrict__ Xs, uint32_t* status,
                                      float* __restrict__ Xcopy) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    double nn = 0.0;
    bool bad = false;
    for (int k = 0; k < d; ++k) {
      const float v = X[j * d + k];
      if (Xcopy) Xcopy[j * d + k] = v;
      if (!isfinite(v)) bad = true;
      nn += (double)v * (double)v;
    }
    if (bad) atomicOr(status, kStNonFinite);
    else if (!(nn > 0.0)) atomicOr(status, kStBadArg);
    const double f = nn > 0.0 ? (double)scale / sqrt(nn) : 0.0;
    for (int k = 0; k < DP; ++k) Xs[j * DP + k] = k < d ? (float)((double)X[j * d + k] * f) : 0.0f;
  }
}

cudaError_t launch_pack_points(const float* X, int64_t n, int d, int DP, float scale, float* Xs,
                               uint32_t* status, cudaStream_t st, int unit, float* Xcopy) {
  if (unit) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    pack_unit_rows_kernel<<<(int)blocks, 256, 0, st>>>(X, n, d, DP, scale, Xs, status, Xcopy);
    return cudaGetLastError();
  }
  if ((DP == 4 || DP == 8) && n <= INT32_MAX && (reinterpret_cast<uintptr_t>(Xs) & 15) == 0) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    if (DP == 4)
      pack_rows_kernel<4><<<(int)blocks, 256, 0, st>>>(X, (int)n, d, scale, Xs, status, Xcopy);
    else
      pack_rows_kernel<8><<<(int)blocks, 256, 0, st>>>(X, (int)n, d, scale, Xs, status, Xcopy);
    return cudaGetLastError();
  }
  int64_t total = n * DP;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  pack_points_kernel<<<(int)blocks, 256, 0, st>>>(X, n, d, DP, scale, Xs, status, Xcopy);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Seed Selection (Alg. 2): entries of the keyed permutation of
// fms_seedperm.cuh.
// ---------------------------------------------------------------------------
__global__ void select_seeds_kernel(int64_t n, FeistelKey f, int64_t start, int64_t count,
                                    int32_t* __restrict__ out) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = (int32_t)permute(start + t, n, f);
}

cudaError_t launch_select_seeds(int64_t n, uint64_t rng_seed, int64_t start, int64_t count,
                                int32_t* out, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const FeistelKey f = make_key(n, rng_seed);
  int64_t blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  select_seeds_kernel<<<(int)blocks, 256, 0, st>>>(n, f, start, count, out);
  return cudaGetLastError();
}

// Slot `slot` takes point idx: position Xs[idx], no updates yet, state init_state.
__device__ __forceinline__ void init_seed_slot(const float* __restrict__ Xs, int DP, int64_t idx,
                                               int64_t slot, int32_t* __restrict__ seed_idx,
                                               float* __restrict__ y, int32_t* __restrict__ it,
                                               int32_t* __restrict__ conv,
                                               int32_t* __restrict__ state, int32_t init_state) {
  seed_idx[slot] = (int32_t)idx;
  for (int k = 0; k < DP; ++k) y[slot * DP + k] = Xs[idx * DP + k];
  it[slot] = 0;
  conv[slot] = -1;
  state[slot] = init_state;
}

// Initialise seed slots [slot0, slot0+count): point index from the explicit
// list or the permutation (rank0 + t), position Xs[idx], state RUNNING.
__global__ void seed_init_kernel(const float* __restrict__ Xs, int64_t n, int DP, FeistelKey f,
                                 const int32_t* __restrict__ explicit_idx, int64_t rank0,
                                 int32_t slot0, int32_t count, int32_t* __restrict__ seed_idx,
                                 float* __restrict__ y, int32_t* __restrict__ it,
                                 int32_t* __restrict__ conv, int32_t* __restrict__ state,
                                 uint32_t* status, int32_t init_state) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
    int64_t idx;
    if (explicit_idx) {
      idx = explicit_idx[t];
      if (idx < 0 || idx >= n) {
        atomicOr(status, kStBadArg);
        idx = 0;
      }
    } else {
      idx = permute(rank0 + t, n, f);
    }
    init_seed_slot(Xs, DP, idx, slot0 + t, seed_idx, y, it, conv, state, init_state);
  }
}

// ---------------------------------------------------------------------------
// Device-driven rounds (the CUDA-graph form of fms_cluster): the round's seed
// count and stop target live in RoundCtl, and round_advance takes the
// seed-count decision of Sec. II-D on the device: N <- min(2N, n) while
// N < L*M (and doubling is allowed), the new slots N..2N-1 taking the next
// entries of the same keyed permutation.  It sets the graph's loop condition
// (another round) and the condition of the post-round work (refinement,
// labels), and leaves the rest to the host (leave != 0) when the next round
// or the refinement would not fit the cluster kernels.
// ---------------------------------------------------------------------------
__global__ void round_begin_kernel(RoundCtl* rc, int32_t N, float gamma) {
  rc->N = N;
  rc->target = stop_target(gamma, N);
  rc->rounds = 0;
  rc->leave = 0;
  rc->K_last = 0;
}

cudaError_t launch_round_begin(RoundCtl* rc, int32_t N, float gamma, cudaStream_t st) {
  round_begin_kernel<<<1, 1, 0, st>>>(rc, N, gamma);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(1024)
    round_advance_kernel(RoundCtl* rc, MergeCtl* mctl, int64_t n, float L, int allow,
                         float gamma, int cap_seeds, int cap_modes, FeistelKey f,
                         const float* __restrict__ Xs, int DP, int32_t* __restrict__ seed_idx,
                         float* __restrict__ y, int32_t* __restrict__ it,
                         int32_t* __restrict__ conv, int32_t* __restrict__ state,
                         int32_t init_state, cudaGraphConditionalHandle h_loop,
                         cudaGraphConditionalHandle h_post) {
  const int N = rc->N, M = mctl->M;
  int next = N;
  if (allow && (float)N < L * (float)M && (int64_t)N < n) {
    const int64_t t2 = 2LL * N;
    next = (int32_t)(t2 < n ? t2 : n);
  }
  for (int t = threadIdx.x; t < next - N; t += blockDim.x)
    init_seed_slot(Xs, DP, permute((int64_t)N + t, n, f), (int64_t)N + t, seed_idx, y, it, conv,
                   state, init_state);
  __syncthreads();   // every thread has read rc->N
  if (threadIdx.x == 0) {
    mctl->next_N = next;
    rc->rounds += 1;
    rc->K_last = mctl->K;
    int more = 0, leave = 0;
    if (next > N) {
      rc->N = next;
      rc->target = stop_target(gamma, next);
      if (next <= cap_seeds) more = 1;
      else leave = 1;   // the next round needs the host-driven path
    } else if (M > cap_modes) {
      leave = 2;        // the refinement needs the host-driven path
    }
    rc->leave = leave;
    cudaGraphSetConditional(h_loop, more ? 1u : 0u);
    cudaGraphSetConditional(h_post, (!more && !leave) ? 1u : 0u);
  }
}

cudaError_t launch_round_advance(RoundCtl* rc, MergeCtl* mctl, int64_t n, float L, int allow,
                                 float gamma, int cap_seeds, int cap_modes, uint64_t rng_seed,
                                 const float* Xs, int DP, int32_t* seed_idx, float* y,
                                 int32_t* it, int32_t* conv, int32_t* state, int32_t init_state,
                                 cudaGraphConditionalHandle h_loop,
                                 cudaGraphConditionalHandle h_post, cudaStream_t st) {
  const FeistelKey f = make_key(n, rng_seed);
  round_advance_kernel<<<1, 1024, 0, st>>>(rc, mctl, n, L, allow, gamma, cap_seeds, cap_modes, f,
                                           Xs, DP, seed_idx, y, it, conv, state, init_state,
                                           h_loop, h_post);
  return cudaGetLastError();
}

cudaError_t launch_seed_init(const float* Xs, int64_t n, int DP, uint64_t rng_seed,
                             const int32_t* explicit_idx, int64_t rank0, int32_t slot0,
                             int32_t count, int32_t* seed_idx, float* y, int32_t* it,
                             int32_t* conv, int32_t* state, uint32_t* status, cudaStream_t st,
                             int32_t init_state) {
  if (count <= 0) return cudaSuccess;
  const FeistelKey f = make_key(n, rng_seed);
  int blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  seed_init_kernel<<<blocks, 256, 0, st>>>(Xs, n, DP, f, explicit_idx, rank0, slot0, count,
                                           seed_idx, y, it, conv, state, status, init_state);
  return cudaGetLastError();
}

// Cross-chunk sum of the partials of active position p: lane l sums chunks
// c0 + cs*l, c0 + cs*(l+32), ... in chunk order for every accumulator
// (16-byte loads), then a fixed xor tree combines the 32 lane sums.  On
// return lane k holds accumulator k (W for k = 0, S_{k-1} otherwise) in
// a[k >> 5], for k <= d.  (c0, cs) = (0, 1) sums every chunk; a block whose
// warp w takes (w, 8) splits them over 8 warps.
__device__ __forceinline__ void reduce_chunks(const float* __restrict__ part, int s, int p, int C,
                                              int DA, int d, int lane, float (&a)[3], int c0 = 0,
                                              int cs = 1) {
  for (int k0 = 0; k0 <= d; k0 += 4) {
    float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f;
    if ((DA & 3) == 0) {
#pragma unroll 4
      for (int c = c0 + cs * lane; c < C; c += 32 * cs) {
        const float4 q = __ldcg(reinterpret_cast<const float4*>(part + ((int64_t)c * s + p) * DA + k0));
        v0 += q.x;
        v1 += q.y;
        v2 += q.z;
        v3 += q.w;
      }
    } else {  // DA == 2 (d == 1)
#pragma unroll 4
      for (int c = c0 + cs * lane; c < C; c += 32 * cs) {
        const float2 q = __ldcg(reinterpret_cast<const float2*>(part + ((int64_t)c * s + p) * DA));
        v0 += q.x;
        v1 += q.y;
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

// ---------------------------------------------------------------------------
// Early Stopping bookkeeping (Sec. II-C).
//
// The clock r counts updates.  A seed takes update r+1 when it is RUNNING and
// has made exactly r updates, so seeds added by a doubling start at 0 while
// seeds left unconverged by an earlier round wait until the clock reaches
// their count: the round then behaves exactly like a fresh run over all N
// seeds.  After each update the seeds whose convergence update is <= r are
// counted and the round stops once that count reaches target =
// ceil(gamma*N), or at max_iter.  When no seed is due at r but the round goes
// on, the clock jumps to the next event (a waiting seed's count or a
// convergence update of an earlier round).  Runs on one block (any size that
// is a multiple of 32); reads bypass L1 because other blocks of the same
// launch wrote the seed states.  With the tensor-core step on, the due seeds
// are listed in two passes, COARSE ones first, so that one contiguous range
// of the list goes to each step kernel; the order within a pass is slot order.
// ---------------------------------------------------------------------------
// want: -1 lists every due running seed, else only those in state `want`.
__device__ void scan_clock(int r, int N, const int32_t* __restrict__ state,
                           const int32_t* __restrict__ it, const int32_t* __restrict__ conv,
                           int32_t* __restrict__ active, int want, int* s_out, int* conv_out,
                           int* next_event_out, int* scratch) {
  // each thread takes V consecutive seeds per block-wide step (one block scan
  // per blockDim * V seeds; V = 16 once N is large), its V state loads issued
  // together, then its V update-count loads; the list stays in slot order
  constexpr int kScanRun = 16;
  const int V = N > (int)blockDim.x * 2 ? kScanRun : 1;
  int base = 0, convd = 0, nxt = INT32_MAX;
  for (int64_t b = 0; b < N; b += (int64_t)blockDim.x * V) {
    const int64_t i0 = b + (int64_t)threadIdx.x * V;
    int stt[kScanRun], cnt_v[kScanRun];
#pragma unroll
    for (int v = 0; v < kScanRun; ++v)
      stt[v] = (v < V && i0 + v < N) ? __ldcg(state + i0 + v) : -1;
#pragma unroll
    for (int v = 0; v < kScanRun; ++v) {
      const int64_t i = i0 + v;
      cnt_v[v] = 0;
      if (stt[v] == kRunning || stt[v] == kCoarse) cnt_v[v] = __ldcg(it + i);
      else if (stt[v] == kConverged) cnt_v[v] = __ldcg(conv + i);
    }
    unsigned takes = 0;
    int cnt = 0;
#pragma unroll
    for (int v = 0; v < kScanRun; ++v) {
      if (stt[v] == kRunning || stt[v] == kCoarse) {
        const int ti = cnt_v[v];
        if (ti == r) {
          if (want < 0 || stt[v] == want) {
            takes |= 1u << v;
            ++cnt;
          }
        } else if (ti > r) {
          nxt = min(nxt, ti);
        }
      } else if (stt[v] == kConverged) {
        const int ci = cnt_v[v];
        if (ci <= r) ++convd;
        else nxt = min(nxt, ci);
      }
    }
    int tot;
    int off = block_exclusive_scan(cnt, &tot, scratch);
#pragma unroll
    for (int v = 0; v < kScanRun; ++v)
      if ((takes >> v) & 1u) active[base + off++] = (int32_t)(i0 + v);
    base += tot;
  }
  convd = block_sum(convd, scratch);
  nxt = block_min(nxt, scratch);
  *s_out = base;
  *conv_out = convd;
  *next_event_out = nxt;
}

__device__ void compaction_body(IterCtl* ctl, const int32_t* __restrict__ state,
                                const int32_t* __restrict__ it, const int32_t* __restrict__ conv,
                                int32_t* __restrict__ active, int64_t n, int32_t R, Tiling tl,
                                int begin, int N, int target, int max_iter, int* scratch) {
  int r = begin ? 0 : __ldcg(&ctl->r) + 1;
  const int prev_s = begin ? 0 : __ldcg(&ctl->s);
  int s = 0, s_c = 0, convd = 0, nxt = 0, done = 0;
  for (int guard = 0; guard <= max_iter + 2; ++guard) {
    if (tl.tc_ctas > 0) {
      int s_f = 0;
      scan_clock(r, N, state, it, conv, active, kCoarse, &s_c, &convd, &nxt, scratch);
      scan_clock(r, N, state, it, conv, active + s_c, kRunning, &s_f, &convd, &nxt, scratch);
      s = s_c + s_f;
    } else {
      scan_clock(r, N, state, it, conv, active, -1, &s, &convd, &nxt, scratch);
    }
    done = (convd >= target) || (r >= max_iter);
    if (!done && s == 0) {
      // nothing is due at r: move the clock to the next event; with no event
      // left the round ends at max_iter
      r = (nxt == INT32_MAX || nxt > max_iter) ? max_iter : nxt;
      continue;
    }
    break;
  }
  if (threadIdx.x == 0) {
    ctl->N = N;
    ctl->target = target;
    ctl->max_iter = max_iter;
    ctl->r = r;
    ctl->done = done;
    ctl->n_converged = convd;
    if (prev_s > 0) ctl->steps += 1;
    ctl->s = done ? 0 : s;
    ctl->s_tc = done ? 0 : s_c;
    int C = 0, Lc = 0;
    if (!done) {
      if (tl.tc_ctas > 0 && s_c >= s - s_c) {
        tc_choose_chunks(n, s_c, tl.tc_ctas, &C, &Lc);
      } else {
        choose_chunks(n, s - s_c, R, tl, &C, &Lc);
        if (tl.tc_ctas > 0) tc_round_chunks(n, &C, &Lc);
      }
    }
    ctl->C = C;
    ctl->Lc = Lc;
    if (!done) ctl->evals += (int64_t)s * n;
    ctl->blocks_done = 0;
  }
}

// Start of a round: the active list for update 1.
__global__ void __launch_bounds__(1024)
    iter_begin_kernel(IterCtl* ctl, const int32_t* __restrict__ state,
                      const int32_t* __restrict__ it, const int32_t* __restrict__ conv,
                      int32_t* __restrict__ active, int64_t n, int32_t R, Tiling tl, int N,
                      int target, int max_iter) {
  __shared__ int scratch[64];
  compaction_body(ctl, state, it, conv, active, n, R, tl, 1, N, target, max_iter, scratch);
}

cudaError_t launch_iter_begin(IterCtl* ctl, const int32_t* state, const int32_t* it,
                              const int32_t* conv, int32_t* active, int64_t n, int32_t R,
                              Tiling tl, int N, int target, int max_iter, cudaStream_t st) {
  iter_begin_kernel<<<1, 1024, 0, st>>>(ctl, state, it, conv, active, n, R, tl, N, target,
                                        max_iter);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Seed update: y <- y + S/W for every active seed, the convergence test
// ||S/W|| <= tol, and the seed's state.  One warp per active position.  The
// last block to finish (atomic ticket after a fence, no waiting) then runs the
// Early Stopping bookkeeping above for the next update.
//
// A COARSE seed's S/W came from the tensor-core step (BF16 weights): it moves
// by it, and once ||S/W|| <= coarse_tol (10 tol) it turns RUNNING, so the
// updates that decide convergence are always exact FP32 ones.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
    update_kernel(const float* __restrict__ part, int32_t* __restrict__ active, IterCtl* ctl,
                  float* __restrict__ y, int32_t* __restrict__ it, int32_t* __restrict__ conv,
                  int32_t* __restrict__ state, int d, int DP, int DA, float tol2_s, int64_t n,
                  int32_t R, Tiling tl, int N, int target, int max_iter, float coarse_tol2_s,
                  float sphere_r, float* __restrict__ wlast) {
  __shared__ int scratch[64];
  __shared__ int sh_last;
  __shared__ float red[8][96];
  if (__ldcg(&ctl->done)) return;  // uniform for the whole launch
  const int s = __ldcg(&ctl->s);
  const int C = __ldcg(&ctl->C);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // many chunks: one block per position, its 8 warps split the chunks and
  // the warp sums are added in warp order; else one warp per position
  const bool block_mode = C >= kBlockReduceChunks;
  const int nw = block_mode ? gridDim.x : gridDim.x * (blockDim.x >> 5);
  const int p_first = block_mode ? blockIdx.x : blockIdx.x * (blockDim.x >> 5) + wid;
  for (int p = p_first; p < s; p += nw) {
    const int64_t slot = __ldcg(active + p);
    float a[3] = {0.f, 0.f, 0.f};
    if (block_mode) {
      reduce_chunks(part, s, p, C, DA, d, lane, a, wid, 8);
#pragma unroll
      for (int u = 0; u < 3; ++u) red[wid][lane + 32 * u] = a[u];
      __syncthreads();
      if (wid == 0) {
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          float t = red[0][lane + 32 * u];
          for (int w = 1; w < 8; ++w) t += red[w][lane + 32 * u];
          a[u] = t;
        }
      }
      __syncthreads();
      if (wid != 0) continue;
    } else {
      reduce_chunks(part, s, p, C, DA, d, lane, a);
    }
    const float W = __shfl_sync(kFull, a[0], 0);
    float step2 = 0.0f;
    float delta[3] = {0.f, 0.f, 0.f};
    const bool ok = (W > 0.0f) && isfinite(W);
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int k = lane + 32 * u;  // accumulator index; coordinate k-1
      if (ok && k >= 1 && k <= d) {
        delta[u] = a[u] / W;
        step2 = fmaf(delta[u], delta[u], step2);
      }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) step2 += __shfl_xor_sync(kFull, step2, o);
    bool finite = ok && isfinite(step2);
    if (finite && sphere_r > 0.0f) {
      // cosine metric: the new position is the mean scaled back onto the
      // sphere of radius sphere_r; the step is the projected one
      float pv[3] = {0.f, 0.f, 0.f};
      float nn = 0.0f;
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int k = lane + 32 * u;
        if (k >= 1 && k <= d) {
          pv[u] = y[slot * DP + (k - 1)] + delta[u];
          nn = fmaf(pv[u], pv[u], nn);
        }
      }
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) nn += __shfl_xor_sync(kFull, nn, o);
      const float f = sphere_r / sqrtf(nn);
      step2 = 0.0f;
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int k = lane + 32 * u;
        if (k >= 1 && k <= d) {
          const float q = pv[u] * f;
          const float e = q - y[slot * DP + (k - 1)];
          step2 = fmaf(e, e, step2);
          pv[u] = q;
        }
      }
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) step2 += __shfl_xor_sync(kFull, step2, o);
      finite = nn > 0.0f && isfinite(step2);
      if (finite) {
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          const int k = lane + 32 * u;
          if (k >= 1 && k <= d) y[slot * DP + (k - 1)] = pv[u];
        }
      }
    } else if (finite) {
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int k = lane + 32 * u;
        if (k >= 1 && k <= d) y[slot * DP + (k - 1)] += delta[u];
      }
    }
    if (lane == 0) {
      // sum w of this update (at the position before it): the prune's density
      // of a seed that converges here
      if (wlast) wlast[slot] = W;
      const int t = it[slot] + 1;
      it[slot] = t;
      const bool coarse = state[slot] == kCoarse;
      if (!finite) {
        state[slot] = kFailed;
      } else if (coarse) {
        if (step2 <= coarse_tol2_s) state[slot] = kRunning;
        if (t >= max_iter) state[slot] = kExhausted;
      } else if (step2 <= tol2_s) {
        state[slot] = kConverged;
        conv[slot] = t;
      } else if (t >= max_iter) {
        state[slot] = kExhausted;
      }
    }
  }
  // last block to finish runs the bookkeeping for the next update
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) sh_last = (atomicAdd(&ctl->blocks_done, 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!sh_last) return;
  __threadfence();
  compaction_body(ctl, state, it, conv, active, n, R, tl, 0, N, target, max_iter, scratch);
}

cudaError_t launch_update(const float* part, int32_t* active, IterCtl* ctl, float* y, int32_t* it,
                          int32_t* conv, int32_t* state, int d, int DP, int DA, float tol2_s,
                          int max_iter, int64_t n, int32_t R, Tiling tl, int N, int target,
                          cudaStream_t st, int grid, float coarse_tol2_s, float sphere_r,
                          float* wlast) {
  update_kernel<<<grid, 256, 0, st>>>(part, active, ctl, y, it, conv, state, d, DP, DA, tol2_s, n,
                                      R, tl, N, target, max_iter, coarse_tol2_s, sphere_r, wlast);
  return cudaGetLastError();
}

}  // namespace fms

namespace fms {

// ---------------------------------------------------------------------------
// Stand-alone single update (fms_mean_shift_step): every seed is active.
// ---------------------------------------------------------------------------
__global__ void step_setup_kernel(int32_t* __restrict__ active, int32_t m, IterCtl* ctl, int32_t C,
                                  int32_t Lc) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    active[i] = i;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->s = m;
    ctl->C = C;
    ctl->Lc = Lc;
  }
}

cudaError_t launch_step_setup(int32_t* active, int32_t m, IterCtl* ctl, int32_t C, int32_t Lc,
                              cudaStream_t st) {
  int blocks = (m + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 1024) blocks = 1024;
  step_setup_kernel<<<blocks, 256, 0, st>>>(active, m, ctl, C, Lc);
  return cudaGetLastError();
}

// out_seeds[i] = seeds[i] + (S_i / W_i) / scale (original units), out_wsum[i] = W_i.
__global__ void step_finish_kernel(const float* __restrict__ part, const IterCtl* __restrict__ ctl,
                                   const float* __restrict__ seeds, int d, int DA, double inv_scale,
                                   float* __restrict__ out_seeds, float* __restrict__ out_wsum) {
  const int s = ctl->s, C = ctl->C;
  const int lane = threadIdx.x & 31;
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < s; p += nw) {
    float a[3] = {0.f, 0.f, 0.f};
    reduce_chunks(part, s, p, C, DA, d, lane, a);
    const float W = __shfl_sync(kFull, a[0], 0);
    // every lane reads its own coordinate before anyone writes (seeds may alias out_seeds)
    float v[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int k = lane + 32 * u;
      v[u] = (k >= 1 && k <= d) ? seeds[(int64_t)p * d + (k - 1)] : 0.0f;
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int k = lane + 32 * u;
      if (k >= 1 && k <= d)
        out_seeds[(int64_t)p * d + (k - 1)] = (float)((double)v[u] + (double)(a[u] / W) * inv_scale);
    }
    if (lane == 0 && out_wsum) out_wsum[p] = W;
  }
}

cudaError_t launch_step_finish(const float* part, const IterCtl* ctl, const float* seeds, int d,
                               int DA, double inv_scale, float* out_seeds, float* out_wsum,
                               int m, cudaStream_t st) {
  int blocks = (m + 7) / 8;
  if (blocks < 1) blocks = 1;
  if (blocks > 4096) blocks = 4096;
  step_finish_kernel<<<blocks, 256, 0, st>>>(part, ctl, seeds, d, DA, inv_scale, out_seeds,
                                             out_wsum);
  return cudaGetLastError();
}

}  // namespace fms
