// Internal declarations shared by the CUDA translation units of the library.
//
// Layout conventions on the device (all in the caller's workspace):
//   Xs      [n][DP] float   points pre-scaled by s = sqrt(log2(e) / (2 h^2)), so
//                           that the Gaussian weight exp(-||y-x||^2/(2h^2)) is
//                           exp2(-||ys - xs||^2); padded to DP floats per row
//                           (DP = 4 for d <= 4, 8 for d <= 8, else d rounded
//                           up to a multiple of 4), pad lanes are 0.
//   seeds   slot i = rank i in the seed sequence: point index, scaled position
//           y[i][DP], updates done it[i], convergence update conv[i] (-1 if
//           none) and state[i] (RUNNING / COARSE / CONVERGED / FAILED /
//           EXHAUSTED); COARSE is a running seed whose updates still take the
//           tensor-core (BF16) step.
//   active  the seed slots that take the next update, in slot order (with
//           the tensor-core step on: COARSE seeds first, then RUNNING ones).
//   part    per-(chunk, active position) partial sums [C][s][DA] float:
//           DA accumulators per seed = (sum w, sum w*(x-y)_0..d-1, pad).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fms {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;
#define FMS_MAX_DIM_PAD 64

// device status bits (OR-ed into the status word)
enum : uint32_t {
  kStNonFinite = 1u,
  kStTimeout = 2u,
  kStCapacity = 4u,
  kStBadArg = 8u,
};

// per-seed state
enum : int32_t { kRunning = 0, kConverged = 1, kFailed = 2, kExhausted = 3, kCoarse = 4 };

// Control block of one iteration loop, written by the device.
struct IterCtl {
  int32_t s;          // active seeds in the next update
  int32_t C;          // point chunks of the next update
  int32_t Lc;         // points per chunk (multiple of 32)
  int32_t r;          // global updates completed in this round
  int32_t done;       // 1: the round has stopped
  int32_t N;          // seeds in play (slots [0, N))
  int32_t target;     // ceil(gamma * N): converged seeds needed to stop
  int32_t max_iter;
  int32_t n_converged;
  int32_t n_failed;
  int32_t n_exhausted;
  int32_t steps;      // updates that had at least one active seed
  int32_t blocks_done;  // blocks of the current update launch that finished
  int32_t s_tc;       // active positions [0, s_tc) take the tensor-core step
  int64_t evals;      // seed-point evaluations issued
};

// Seed count and stop target of the device-driven rounds (CUDA-graph form).
struct RoundCtl {
  int32_t N;        // seeds in play
  int32_t target;   // ceil(gamma * N), clamped to [1, N]
  int32_t rounds;   // rounds completed
  int32_t leave;    // != 0: the host continues (1: next round, 2: refinement)
  int32_t K_last;   // prune candidates of the last round
  int32_t pad[3];
};

// ceil(gamma * N) clamped to [1, N] (the Early-Stopping count of Sec. II-C)
__host__ __device__ inline int32_t stop_target(float gamma, int32_t N) {
  int t = (int)ceil((double)gamma * (double)N);
  if (t < 1) t = 1;
  if (t > N) t = N;
  return t;
}

// Control block of the prune / refine phase.
struct MergeCtl {
  int32_t K;              // candidates of the prune (kept seeds)
  int32_t C;              // chunks of the score pass over the candidates
  int32_t Lc;
  int32_t M;              // modes accepted by the prune
  int32_t next_N;         // N of the next round (== N when not doubling)
  int32_t t_star;         // stop update of the round
  int32_t Mr;             // modes after refinement and the second prune
  int32_t Cr;             // chunks of a refinement pass (one mode per warp task)
  int32_t Lcr;
  int32_t refine_active;  // modes still moving
  int32_t refine_iters;
  int32_t pad0;
  int64_t evals;          // evaluations of prune scores and refinement
};

// Chunk count from which the cross-chunk reductions use a whole block (8
// warps) per seed instead of one warp.
constexpr int kBlockReduceChunks = 64;

// Smallest point chunk of a warp task (points): below this the per-task work
// (seed loads, the warp reduction and one store) stops being small next to
// the evaluations.
constexpr int kStepMinChunk = 512;

// Cluster-persistent rounds (k_round.cu): CTAs per cluster and the most seeds
// one cluster owns.
constexpr int kClusterCtas = 8;
constexpr int kSeedsPerCluster = 64;
constexpr int kModesPerCluster = 32;   // refinement: modes one cluster owns

// Shared memory budget of the batched per-set prune (k_batched.cu).
constexpr size_t kBatchedPruneSmem = 200 * 1024;

// Per-set control block of the batched path (k_batched.cu).
struct SetCtl {
  int32_t n;       // points of the set
  int32_t p0;      // first point, first seed slot and first list entry of the set
  int32_t N;       // seeds in play
  int32_t prevN;   // seeds before the last doubling (new seeds: ranks prevN..N-1)
  int32_t target;  // ceil(gamma * N)
  int32_t r;       // Early Stopping clock
  int32_t done;    // round finished
  int32_t s;       // active seeds of the next update
  int32_t C, Lc;   // chunks of the next update
  int32_t steps;
  int32_t n_conv;
  int32_t K;       // kept seeds (prune candidates)
  int32_t Ck, Lck; // chunks of the density pass
  int32_t M;       // modes accepted by the first prune
  int32_t next_N;
  int32_t t_star;
  int32_t final_;  // 1: no further doubling; the set's prune result is final
  int32_t rs;      // refinement: active modes
  int32_t rC, rLc;
  int32_t rr;      // refinement clock
  int32_t rdone;
  int32_t Mr;      // modes after refinement and the second prune
  int32_t pad0;
  int64_t evals;
};

// Batched call: a graph condition that a kernel sets when it finishes (on = 0:
// the kernel runs outside the graph and sets nothing), and the slots of the
// call's device counters.
struct BatchCond {
  cudaGraphConditionalHandle h;
  int32_t on;
};
enum BatchCounter : int {
  kCtrBlocksDone = 0,   // atomic ticket of the per-set kernels
  kCtrRounds = 1,       // seed rounds run
  kCtrUpdates = 2,      // seed updates run (all rounds)
  kCtrRefine = 3,       // refinement updates run
};

// Tiling of a (seed-group x point-chunk) warp-task grid.
struct Tiling {
  int32_t target_warps;   // warps the step grid runs (gridDim.x * warps per CTA)
  int32_t min_chunk;      // smallest chunk in points (multiple of 32)
  int32_t tc_ctas;        // > 0: COARSE seeds take the tensor-core step, whose grid
                          // has this many CTAs; chunks are then whole 128-point tiles
};

// Chunk count and length for s active seeds of R per warp over n points.
// The warp-task grid is G = ceil(s/R) seed groups x C chunks, run by
// target_warps persistent warps.  C is chosen to fill the last wave of warp
// tasks best (ties: fewer chunks), with chunks of at least min_chunk points.
__host__ __device__ inline void choose_chunks(int64_t n, int32_t s, int32_t R, Tiling t,
                                              int32_t* C, int32_t* Lc) {
  if (s <= 0) {
    *C = 0;
    *Lc = 0;
    return;
  }
  const int64_t G = (s + R - 1) / R;
  const int64_t TW = t.target_warps > 0 ? t.target_warps : 1;
  int64_t cmax = n / t.min_chunk;
  if (cmax < 1) cmax = 1;
  const int64_t cwant = (4 * TW + G - 1) / G;  // never more than ~4 waves of tasks
  if (cmax > cwant) cmax = cwant;
  // the best C for k waves is the largest C with G*C <= k*TW; try k = 1..4
  int64_t best_c = 1;
  int64_t best_num = -1, best_den = 1;  // efficiency as a fraction
  for (int k = 0; k <= 4; ++k) {
    int64_t c = k == 0 ? cmax : (k * TW) / G;
    if (c > cmax) c = cmax;
    if (c < 1) c = 1;
    const int64_t tasks = G * c;
    const int64_t waves = (tasks + TW - 1) / TW;
    // eff = tasks / (waves * TW); compare fractions exactly; ties -> fewer chunks
    if (tasks * best_den > best_num * (waves * TW) ||
        (tasks * best_den == best_num * (waves * TW) && c < best_c)) {
      best_num = tasks;
      best_den = waves * TW;
      best_c = c;
    }
  }
  int64_t lc = (n + best_c - 1) / best_c;
  lc = (lc + 31) / 32 * 32;
  *C = (int32_t)((n + lc - 1) / lc);
  *Lc = (int32_t)lc;
}

// Points per tile of the tensor-core step (k_step_tc.cu).
constexpr int kTcTile = 128;

// Chunks for the tensor-core step: s seeds in tiles of 128 x chunks of whole
// 128-point tiles, run by a persistent grid of `grid` CTAs.  Candidate chunk
// counts are 1..4 and the counts that make k = 1..4 full waves; the one whose
// last wave is fullest wins (ties -> fewer chunks), with at least kTcMinTiles
// tiles per chunk.  C <= max(4, 4 grid / G + 1).
constexpr int kTcMinTiles = 2;
__host__ __device__ inline void tc_choose_chunks(int64_t n, int32_t s, int32_t grid, int32_t* C,
                                                 int32_t* Lc) {
  if (s <= 0) {
    *C = 0;
    *Lc = 0;
    return;
  }
  const int64_t nt = (n + kTcTile - 1) / kTcTile;
  const int64_t G = (s + kTcTile - 1) / kTcTile;
  const int64_t P = grid > 0 ? grid : 1;
  int64_t best_tpc = nt, best_num = -1, best_den = 1, best_c = 1;
  for (int cand = 0; cand < 8; ++cand) {
    int64_t c = cand < 4 ? cand + 1 : ((cand - 3) * P) / G;
    if (c < 1) c = 1;
    int64_t tpc = (nt + c - 1) / c;
    if (tpc < kTcMinTiles) tpc = kTcMinTiles < nt ? kTcMinTiles : nt;
    c = (nt + tpc - 1) / tpc;
    const int64_t tasks = G * c;
    const int64_t waves = (tasks + P - 1) / P;
    if (tasks * best_den > best_num * (waves * P) ||
        (tasks * best_den == best_num * (waves * P) && c < best_c)) {
      best_num = tasks;
      best_den = waves * P;
      best_c = c;
      best_tpc = tpc;
    }
  }
  *C = (int32_t)best_c;
  *Lc = (int32_t)(best_tpc * kTcTile);
}

// Chunk length rounded up to whole tensor-core tiles (C recomputed).
__host__ __device__ inline void tc_round_chunks(int64_t n, int32_t* C, int32_t* Lc) {
  if (*C <= 0) return;
  const int64_t lc = ((int64_t)*Lc + kTcTile - 1) / kTcTile * kTcTile;
  *Lc = (int32_t)lc;
  *C = (int32_t)((n + lc - 1) / lc);
}

__device__ __forceinline__ float ex2_ftz(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Profile weight of a seed-point pair from t = -||ys - xs||^2 in scaled
// coordinates (xs = s x, s = sqrt(log2(e) / (2 h^2))):
//   KF = 0, Gaussian: exp(-||y - x||^2 / (2 h^2)) = exp2(t);
//   KF = 1, flat (Eq. 12): 1 inside the window ||y - x|| <= h, i.e.
//           ||ys - xs||^2 <= s^2 h^2 = log2(e) / 2 for every h, else 0.
enum : int { kKernelGaussian = 0, kKernelFlat = 1 };
constexpr float kFlatT = -0.72134752044448170f;   // -log2(e) / 2
template <int KF>
__device__ __forceinline__ float kweight(float t) {
  if constexpr (KF == kKernelFlat) return t >= kFlatT ? 1.0f : 0.0f;
  else return ex2_ftz(t);
}

// Block-wide helpers (every thread of the block must call them).
__device__ inline int block_exclusive_scan(int v, int* total, int* warp_sums) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = lane < (blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, w, o);
      if (lane >= o) w += y;
    }
    warp_sums[lane] = w;  // inclusive
  }
  __syncthreads();
  const int before = (wid > 0 ? warp_sums[wid - 1] : 0) + x - v;
  *total = warp_sums[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before;
}

__device__ inline int block_sum(int v, int* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  if (lane == 0) red[wid] = v;
  __syncthreads();
  int t = 0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  __syncthreads();
  return t;
}

__device__ inline int block_min(int v, int* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v = min(v, __shfl_xor_sync(kFull, v, o));
  if (lane == 0) red[wid] = v;
  __syncthreads();
  int t = INT32_MAX;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = min(t, red[i]);
  __syncthreads();
  return t;
}

// ---------------------------------------------------------------------------
// launchers (host functions defined in the .cu files)
// ---------------------------------------------------------------------------

// k_iter.cu
// unit != 0 (cosine metric): each row normalised to unit length first
cudaError_t launch_pack_points(const float* X, int64_t n, int d, int DP, float scale, float* Xs,
                               uint32_t* status, cudaStream_t st, int unit = 0,
                               float* Xcopy = nullptr);
cudaError_t launch_seed_init(const float* Xs, int64_t n, int DP, uint64_t rng_seed,
                             const int32_t* explicit_idx, int64_t rank0, int32_t slot0,
                             int32_t count, int32_t* seed_idx, float* y, int32_t* it,
                             int32_t* conv, int32_t* state, uint32_t* status, cudaStream_t st,
                             int32_t init_state = kRunning);
cudaError_t launch_select_seeds(int64_t n, uint64_t rng_seed, int64_t start, int64_t count,
                                int32_t* out, cudaStream_t st);
cudaError_t launch_round_begin(RoundCtl* rc, int32_t N, float gamma, cudaStream_t st);
cudaError_t launch_round_advance(RoundCtl* rc, MergeCtl* mctl, int64_t n, float L, int allow,
                                 float gamma, int cap_seeds, int cap_modes, uint64_t rng_seed,
                                 const float* Xs, int DP, int32_t* seed_idx, float* y,
                                 int32_t* it, int32_t* conv, int32_t* state, int32_t init_state,
                                 cudaGraphConditionalHandle h_loop,
                                 cudaGraphConditionalHandle h_post, cudaStream_t st);
cudaError_t launch_iter_begin(IterCtl* ctl, const int32_t* state, const int32_t* it,
                              const int32_t* conv, int32_t* active, int64_t n, int32_t R,
                              Tiling tl, int N, int target, int max_iter, cudaStream_t st);
cudaError_t launch_update(const float* part, int32_t* active, IterCtl* ctl, float* y, int32_t* it,
                          int32_t* conv, int32_t* state, int d, int DP, int DA, float tol2_s,
                          int max_iter, int64_t n, int32_t R, Tiling tl, int N, int target,
                          cudaStream_t st, int grid, float coarse_tol2_s = 0.0f,
                          float sphere_r = 0.0f,    // > 0: project onto that sphere
                          float* wlast = nullptr);  // sum w of each seed's last update
cudaError_t launch_step_setup(int32_t* active, int32_t m, IterCtl* ctl, int32_t C, int32_t Lc,
                              cudaStream_t st);
cudaError_t launch_step_finish(const float* part, const IterCtl* ctl, const float* seeds, int d,
                               int DA, double inv_scale, float* out_seeds, float* out_wsum,
                               int m, cudaStream_t st);

// k_round.cu
cudaError_t launch_ms_round(const float* Xs, int64_t n, int d, float* y, int32_t* it,
                            int32_t* conv, int32_t* state, const int32_t* list,
                            const int32_t* S_ptr, int clusters, int32_t* hist, int target,
                            int max_iter, float tol2_s, unsigned long long* evals,
                            float* wlast, cudaStream_t st, int kf = kKernelGaussian,
                            const RoundCtl* rc = nullptr,   // rc: target from the device
                            float sphere_r = 0.0f);         // > 0: project onto that sphere
// (wlast[slot]: sum w of the seed's latest update, at the position before it)
int round_max_clusters(int d);
cudaError_t launch_ms_refine(const float* Xs, int64_t n, int d, const float* y,
                             const int32_t* kept, const int32_t* accepted, const int32_t* M_ptr,
                             int clusters, double* ym, float* yf, double* mscore, double tol2_s,
                             int max_iter, int32_t* iters_out, unsigned long long* evals,
                             cudaStream_t st, int kf = kKernelGaussian,
                             double sphere_r = 0.0);
cudaError_t launch_round_list(const int32_t* state, int N, int32_t* list, int32_t* S_out,
                              cudaStream_t st, const RoundCtl* rc = nullptr);   // rc: N
cudaError_t launch_round_finish(const int32_t* hist, int target, int max_iter,
                                const int32_t* state, const int32_t* conv, int N,
                                int keep_exhausted, int32_t* kept, MergeCtl* mctl, IterCtl* ctl,
                                int64_t n, int32_t R, Tiling tl, cudaStream_t st,
                                const RoundCtl* rc = nullptr,   // rc: N and target
                                const float* wlast = nullptr,   // with score: the prune
                                float* score = nullptr);        // densities from wlast

// k_grid.cu: persistent grid rounds (one CTA per SM, cooperative launch).
// Most seeds one round launch holds (fewer for d >= 4, see GridPlan::seeds),
// and the convergence histogram entries every CTA keeps (max_iter must be
// below kGridHist).
constexpr int kGridMaxSeeds = 1024;
constexpr int kGridHist = 2048;

// Launch plan of the grid round for (n, d) on this device.
struct GridPlan {
  int ok;         // 1: the grid round can run
  int G;          // CTAs (one per SM)
  int per_cta;    // points per CTA slice
  int n_sub;      // sub-slices per CTA slice
  int sub_len;    // points per sub-slice (multiple of 32)
  int resident;   // 1: the slice is staged in shared memory
  int smem;       // dynamic shared memory per CTA (bytes)
  int fx_bits;    // fixed-point scale of the cross-CTA sums: 2^fx_bits
  int seeds;      // most seeds one launch holds
};

struct GridRoundArgs {
  const float* Xs;             // packed points [n][DP]
  int n;
  int per_cta, n_sub, sub_len; // filled by launch_ms_grid_round
  float* y;                    // seed state (slots [0, N))
  int32_t* it;
  int32_t* conv;
  int32_t* state;
  float* wlast;
  int32_t* hist;               // global convergence histogram [max_iter + 2]
  const RoundCtl* rc;          // non-null: N and target from the device
  int N_arg, target_arg;
  int max_iter;
  float tol2_s;                // squared tolerance in scaled coordinates
  float sphere_r;              // > 0: cosine metric, project onto this sphere
  unsigned long long* evals;
  unsigned long long* gacc;    // filled by launch_ms_grid_round
  unsigned* gbar;
  uint32_t* status;
  float fx_scale;              // 2^fx_bits
  float inv_fx_scale;          // 2^-fx_bits
};

GridPlan grid_round_plan(int64_t n, int d, int sms, int max_iter);
size_t grid_scratch_bytes(int d);
size_t grid_scratch_clear_bytes(int d);
// Clears the scratch's counter and first accumulator, then launches the round.
cudaError_t launch_ms_grid_round(const GridPlan& p, int d, int kf, GridRoundArgs a,
                                 void* scratch, cudaStream_t st);
// The refinement (FP64 positions, up to grid_refine_capacity() merged modes)
// on the same persistent grid; the accumulators reuse the round's scratch.
int grid_refine_capacity();
cudaError_t launch_ms_grid_refine(const GridPlan& p, const float* Xs, int64_t n, int d,
                                  const float* y, const int32_t* kept, const int32_t* accepted,
                                  const int32_t* M_ptr, double* ym, float* yf, double* mscore,
                                  double tol2_s, int max_iter, int32_t* iters_out,
                                  unsigned long long* evals, uint32_t* status, void* scratch,
                                  cudaStream_t st, int kf, double sphere_r);

// k_unroll.cu: unrolled steps and their adjoint
struct UGeom {
  int B, n, m, d, DP;  // DP: padded row length of the packed copies (4, 8, 16 or 32)
  int Cp, Lp;          // point chunks of the seed-major passes (Lp points each)
  int Cs, Ls;          // seed chunks of the point-major pass (Ls seeds each)
};
// One forward update (T = float, or double for checking gradients); Wout (W_t)
// and Sh (the weight shift of seeds whose W underflowed, 0 otherwise) may be
// null; rlist [B m] and rcount (zero on entry, zero again on return) are
// scratch; status receives kStTimeout if a staged-row wait gives up (the
// affected outputs are then NaN).
template <typename T>
cudaError_t unroll_fwd_step(const T* X, const T* Y, const UGeom& g, T c, T* part, T* Ynext,
                            T* Wout, T* Sh, int32_t* rlist, int32_t* rcount, int grid,
                            uint32_t* status, cudaStream_t st);
// The adjoint of one update; SD is scratch of [B m] x (2 DP + 4) values.
template <typename T>
cudaError_t unroll_bwd_step(const T* X, const T* Y, const T* MU, const T* G, const T* Wt,
                            const T* Sh, const UGeom& g, T c, T inv_h2, T inv_h3, T* part_s,
                            T* part_p, T* SD, T* dh_part, T* Gprev, T* dX, double* dh, int grid,
                            uint32_t* status, cudaStream_t st);
template <typename T>
cudaError_t unroll_pack_rows(const T* src, int64_t rows, int d, int DP, T* dst, cudaStream_t st);
template <typename T>
cudaError_t unroll_unpack_rows(const T* src, int64_t rows, int d, int DP, T* dst,
                               cudaStream_t st);

// k_step.cu: one update's partial sums for the active seeds
// status: the call's status word (kStTimeout when a staged-tile wait gives up;
// required for d > 8)
cudaError_t launch_ms_step(const float* Xs, int64_t n, int d, int DP, const float* y,
                           const int32_t* active, const int32_t* s_ptr, const int32_t* C_ptr,
                           const int32_t* Lc_ptr, float* part, int target_warps,
                           cudaStream_t st, int32_t* s_log = nullptr,
                           const int32_t* p_lo_ptr = nullptr, int kf = kKernelGaussian,
                           uint32_t* status = nullptr);
int step_seeds_per_warp(int d);
int batched_seeds_per_warp(int d);   // the batched step's wide tasks (32 lanes x RG seeds)
int step_resident_warps_per_sm(int d);
// smallest chunk (points) of a warp task: the low-d kernel splits a chunk over
// 32 lanes, the quad kernel (d = 8) over 4 point lanes, the wide kernel
// (d > 8) gives every point to all 32 lanes
inline int step_min_chunk(int d) { return d <= 7 ? kStepMinChunk : (d <= 8 ? 256 : 64); }
int step_accumulators(int d);

// Scratch layout of one stand-alone update (fms_mean_shift_step and its
// allocation-free variant): packed points, packed seeds, active list,
// per-chunk partial sums, control block, status word; every region 256-byte
// aligned.
struct StepLayout {
  size_t off_Xs, off_Ys, off_active, off_part, off_ctl, off_status, total;
  int DP, DA, R, grid_ctas, C, Lc;
};

// Row width of the packed copies: the padded dimension the step kernels are
// compiled for (4, 8, 16, 32 or 64), so their row loads need no bounds test;
// the padding coordinates are zero for points and seeds alike.
inline int padded_dim(int d) {
  if (d <= 4) return 4;
  if (d <= 8) return 8;
  if (d <= 16) return 16;
  if (d <= 32) return 32;
  return 64;
}

inline size_t align256(size_t x) { return (x + 255) / 256 * 256; }

inline StepLayout step_layout(int64_t n, int d, int64_t m, int sms) {
  StepLayout L{};
  L.DP = padded_dim(d);
  L.DA = step_accumulators(d);
  L.R = step_seeds_per_warp(d);
  Tiling tl{(sms > 0 ? sms : 1) * step_resident_warps_per_sm(d), step_min_chunk(d)};
  L.grid_ctas = (tl.target_warps + 7) / 8;
  choose_chunks(n, (int32_t)m, L.R, tl, &L.C, &L.Lc);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at_ = o;
    o += align256(bytes > 0 ? bytes : 1);
    return at_;
  };
  L.off_Xs = take((size_t)n * L.DP * 4);
  L.off_Ys = take((size_t)m * L.DP * 4);
  L.off_active = take((size_t)m * 4);
  L.off_part = take((size_t)L.C * (size_t)m * L.DA * 4);
  L.off_ctl = take(sizeof(IterCtl));
  L.off_status = take(64);
  L.total = o;
  return L;
}

// k_step_tc.cu: the coarse step on the tensor cores (1 <= d <= 32).  The
// point tile images are built once per call by launch_tc_pack; the step
// handles active positions [0, *count_ptr) of a list whose partials have the
// stride *s_total_ptr, with chunks of *Lc_ptr (a multiple of 128) points.
constexpr int kTcMaxDim = 32;
size_t tc_image_bytes(int64_t n, int d);
cudaError_t launch_tc_pack(const float* Xs, int64_t n, int d, int DP, unsigned char* img,
                           cudaStream_t st);
int tc_grid(int d);
cudaError_t launch_ms_step_tc(const unsigned char* img, int64_t n, int d, int DP, int DA,
                              const float* y, const int32_t* active, const int32_t* s_total_ptr,
                              const int32_t* count_ptr, const int32_t* C_ptr,
                              const int32_t* Lc_ptr, float* part, uint32_t* status,
                              cudaStream_t st, int32_t* s_log = nullptr);

// k_merge.cu
cudaError_t launch_kept_list(const IterCtl* ctl, const int32_t* state, const int32_t* conv,
                             int keep_exhausted, int32_t* kept, MergeCtl* mctl, int64_t n,
                             int32_t R, Tiling tl, cudaStream_t st,
                             const float* wlast = nullptr,   // gather the prune's scores from
                             float* score = nullptr);        // each kept seed's last update
cudaError_t launch_score_reduce(const float* part, const MergeCtl* mctl, int DA, float* score,
                                int max_K, cudaStream_t st);
// status: the call's status word; with it, candidate sets too large for one
// CTA's sorted visit take the grid visit (kStTimeout if a barrier gives up)
cudaError_t launch_greedy_merge_f(const int32_t* cand_row, const int32_t* K_ptr,
                                  const float* score, const float* pos, int DP, int d, float r2,
                                  int32_t* alive, int32_t* accepted, int32_t* M_out, int max_K,
                                  cudaStream_t st, uint32_t* status = nullptr);
cudaError_t launch_greedy_merge_d(const int32_t* K_ptr, const double* score, const double* pos,
                                  int DP, int d, double r2, int32_t* alive, int32_t* accepted,
                                  int32_t* M_out, int max_K, cudaStream_t st);
cudaError_t launch_doubling_decision(MergeCtl* mctl, int32_t N, int64_t n, float L, int allow,
                                     cudaStream_t st);
cudaError_t launch_refine_setup(const float* y, const int32_t* kept, const int32_t* accepted,
                                const int32_t* M_ptr, int DP, double* ym, float* yf,
                                int32_t* active, int32_t* mdone, IterCtl* rctl, int init_pos,
                                int64_t n, int32_t R, Tiling tl, int max_M, cudaStream_t st);
cudaError_t launch_refine_update(const float* part, int32_t* active, IterCtl* rctl, double* ym,
                                 float* yf, int32_t* mdone, double* mscore, int d, int DP, int DA,
                                 double tol2_s, int max_iter, int64_t n, int32_t R,
                                 Tiling tl, int max_M, cudaStream_t st,
                                 double sphere_r = 0.0);
cudaError_t launch_canonical_order(const double* ym, const double* mscore,
                                   const int32_t* accepted, const int32_t* M_ptr, int d, int DP,
                                   double inv_scale, float* out_modes, int32_t max_modes,
                                   float* modes_full, float* out_scores, int max_M,
                                   cudaStream_t st);
cudaError_t launch_unrefined_modes(const float* y, const int32_t* kept, const int32_t* accepted,
                                   const float* score, const MergeCtl* mctl, int DP, double* ym,
                                   double* mscore, int max_M, cudaStream_t st);
cudaError_t launch_label(const float* X, int64_t n, int d, const float* modes,
                         const int32_t* M_dev, int32_t M_host, int32_t* labels, float* margins,
                         cudaStream_t st,
                         int unit = 0);   // unit: compare the points' directions

}  // namespace fms
