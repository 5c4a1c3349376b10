/*
 * fms.h -- C ABI of the GB300 (sm_103a) Faster Mean-shift library.
 *
 * Gaussian-kernel mean-shift clustering with the Euclidean metric, after
 * "GPU-accelerated Faster Mean Shift with euclidean distance metrics"
 * (arXiv 2112.13891):
 *   - the update of every seed y is the Gaussian-weighted mean over ALL n
 *     points, m(y) = sum_j w_j x_j / sum_j w_j, w_j = exp(-||y - x_j||^2/(2h^2))
 *     (Sec. II-A Eq. 6 and Eq. 9-10 read with the Gaussian profile; Sec. II-B,
 *     the update of Alg. 2 and the prose after Eq. 11: no window search);
 *   - Seed Selection: N = 128 seeds drawn from the points, doubled while
 *     N < L*M with L = 8 (Alg. 2, Sec. II-C Eq. 15, Sec. II-D);
 *   - Early Stopping: iteration ends once ceil(gamma*N) seeds have converged;
 *     seeds not converged by then are discarded (Sec. II-C);
 *   - modes are pruned (the prune of Alg. 2) and every point is labelled by its
 *     nearest mode (the labelling of Alg. 2);
 *   - options select the flat kernel of Eq. 12-15 instead of the Gaussian,
 *     and the cosine metric of the sibling method the paper cites.
 *
 * Conventions (all entry points):
 *   - Array arguments are DEVICE pointers unless marked "host".  Points are
 *     row-major float32 [n x d], contiguous.  The caller owns every buffer.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All device work is issued on it, in order.
 *   - Nothing throws across the ABI.  Every call returns an fms_status; device
 *     detected errors (non-finite input, exhausted capacity, a wait that timed
 *     out) come back through a status word the call reads before returning.
 *   - Calls that return host-visible results (counts, stats) synchronise the
 *     stream once before returning; this is stated per call.
 *   - Calls on the same device and stream are serialised by the stream; calls
 *     that share one workspace must not overlap.
 */
#ifndef FMS_H
#define FMS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fms_status {
  FMS_OK = 0,
  FMS_ERR_INVALID_ARG = 1,  /* a size, pointer or option is out of range          */
  FMS_ERR_NONFINITE = 2,    /* a point coordinate is NaN or +-inf                  */
  FMS_ERR_CAPACITY = 3,     /* more modes than max_modes (count still reported)    */
  FMS_ERR_TIMEOUT = 4,      /* a bounded device wait gave up                       */
  FMS_ERR_CUDA = 5,         /* a CUDA runtime call failed                          */
  FMS_ERR_WORKSPACE = 6,    /* workspace too small or misaligned                   */
  FMS_ERR_UNSUPPORTED = 7   /* dimension or mode not built into this library       */
} fms_status;

/* Largest point dimension the library accepts. */
#define FMS_MAX_DIM 64

/*
 * Options.  A zero-initialised struct selects the defaults shown.
 */
typedef struct fms_options {
  int32_t all_seeds;        /* 0: Seed Selection + Early Stopping (Alg. 2).
                               1: every point is a seed, gamma = 1, no doubling
                                  (plain mean shift, Alg. 1).                    */
  int32_t n_initial;        /* initial seed count N; 0 -> 128 (Sec. II-D)        */
  float L;                  /* doubling factor: double N while N < L*M; 0 -> 8   */
  float gamma;              /* Early Stopping fraction in (0, 1]; 0 -> 0.95.
                               The paper gives no value (Sec. II-C).             */
  float merge_radius;       /* prune radius in point units; 0 -> h               */
  int32_t skip_refine;      /* 0: refine every merged mode with FP64-accumulated
                               updates until the step is <= 1e-5*h (at most 50
                               updates) and merge again; 1: report the merged
                               seeds as they are.                                */
  uint64_t rng_seed;        /* key of the seed permutation (see fms_select_seeds) */
  const int32_t* seed_indices; /* optional DEVICE list of seed point indices; when
                               non-NULL it replaces Seed Selection and doubling   */
  int32_t n_seed_indices;   /* its length                                         */
  int32_t profile;          /* 1: time every ms_step launch with CUDA events and
                               report it in fms_stats (adds event records)        */
  int32_t precision;        /* arithmetic of the seed updates (FMS_PRECISION_*):
                               AUTO (0) = TENSOR for 9 <= d <= 32, else FP32.
                               FP32 (1): every update evaluates the weights in
                                  FP32 from exact differences.
                               TENSOR (2, 8 <= d <= 32; FP32 elsewhere): a
                                  seed's updates take the coarse tensor-core
                                  step (BF16 weights, FP32 sums; see
                                  fms_mean_shift_step_coarse) until one moves
                                  it by <= 10*tol, then FP32 updates, so
                                  convergence is always decided by an FP32
                                  update.  Modes agree with FP32 within the
                                  tolerance; a seed's update count may differ. */
  int32_t kernel;           /* profile of the weights (FMS_KERNEL_*):
                               GAUSSIAN (0): w = exp(-||y-x||^2 / (2h^2)) over all
                                  points (the reading of Sec. II-B used throughout).
                               FLAT (1): the uniform kernel of Eq. 12-15: the
                                  update is the mean of the points within
                                  distance h (inclusive), the density of a mode
                                  the number of such points; a seed whose window
                                  is empty fails.  FP32 updates only (precision is
                                  ignored); not available in fms_cluster_batched. */
  int32_t metric;           /* distance (FMS_METRIC_*):
                               EUCLIDEAN (0): the paper's metric.
                               COSINE (1): the sibling method the paper cites
                                  (its formulation is not printed there): the
                                  points are normalised to the unit sphere (a
                                  zero point is an invalid argument), the weight
                                  is the kernel of the chord distance ||x - y||
                                  between unit vectors (Gaussian: exp((x.y - 1)
                                  / h^2)), and every update is projected back
                                  onto the sphere.  h, tol, merge_radius and the
                                  margins are chord distances; modes are unit
                                  vectors.  FP32 updates only; not available in
                                  fms_cluster_batched.                          */
  int32_t reserved[3];      /* must be zero                                       */
} fms_options;

#define FMS_KERNEL_GAUSSIAN 0
#define FMS_KERNEL_FLAT 1
#define FMS_METRIC_EUCLIDEAN 0
#define FMS_METRIC_COSINE 1

#define FMS_PRECISION_AUTO 0
#define FMS_PRECISION_FP32 1
#define FMS_PRECISION_TENSOR 2

/* Statistics of one clustering call (host struct, filled when non-NULL). */
typedef struct fms_stats {
  int32_t iterations;       /* global mean-shift iterations over all rounds       */
  int32_t rounds;           /* 1 + number of seed doublings                       */
  int32_t n_seeds_final;    /* N at the end                                       */
  int32_t n_converged;      /* seeds converged by the final stop iteration        */
  int32_t n_discarded;      /* seeds dropped by Early Stopping or failed (sum w=0) */
  int32_t n_kept;           /* seeds that entered the final prune                 */
  int32_t n_modes;          /* M                                                  */
  int32_t refine_iterations;/* FP64-accumulated refinement updates                */
  int32_t t_star_last;      /* stop iteration of the last round                   */
  int32_t kernel_launches;  /* CUDA kernels this call launched                    */
  int64_t evals;            /* seed-point kernel evaluations in mean-shift updates */
  int64_t score_evals;      /* evaluations spent on prune scores and refinement   */
  uint64_t workspace_bytes; /* bytes of workspace the call used                   */
  /* filled when opt->profile = 1 (else zero): */
  double step_kernel_ms;    /* summed device time of ms_step launches that had work */
  int32_t step_launches;    /* ms_step launches that had work                     */
  int32_t coarse_launches;  /* tensor-core coarse step launches that had work     */
  int64_t step_evals;       /* seed-point evaluations of those launches           */
  double round_kernel_ms;   /* summed device time of the cluster round launches   */
  int64_t round_evals;      /* evaluations of those launches                      */
  int32_t round_launches;
  int32_t graph;            /* 1: the call ran as one cached CUDA graph (the same
                               kernels as the host-driven path, one host sync) */
  double phase_ms[4];       /* device time of: seed rounds (selection, updates,
                               stop), prunes + doubling, refinement + ordering,
                               labels                                            */
  double coarse_kernel_ms;  /* summed device time of those coarse step launches   */
  int64_t coarse_evals;     /* evaluations of those launches                      */
} fms_stats;

/* Human-readable name of a status code (static storage). */
const char* fms_strerror(fms_status status);

/*
 * Self-test of the bounded waits the tensor-core step uses on its mbarriers
 * (failure detection without a GPU fault; no counterpart in the paper): one
 * CTA waits on a phase that nothing completes, polling at most `spins` times
 * through the wait helper `variant` selects (0: try_wait, 1: polling
 * test_wait with an abort flag, 2: suspending try_wait with an abort flag).
 * A wait that gives up sets the FMS_ERR_TIMEOUT bit of the status word and
 * returns, as in the step kernel; the phase is then completed and the same
 * wait must succeed.  *out_status (host) receives the status word: 2 =
 * timed out as expected, 8 = the completed phase was not seen.  Returns
 * FMS_ERR_TIMEOUT when the first wait gave up.  Synchronises `stream`.
 */
fms_status fms_selftest_bounded_wait(int32_t variant, int64_t spins, uint32_t* out_status,
                                     void* stream);

/* Fill *opt with the explicit default values listed in fms_options. */
void fms_options_default(fms_options* opt);

/*
 * Workspace bytes fms_cluster needs for n points of dimension d with the
 * given options (NULL = defaults).  Returns 0 for invalid sizes.
 */
size_t fms_workspace_size(int64_t n, int32_t d, const fms_options* opt);

/*
 * Faster Mean-shift clustering (Alg. 2, Sec. II-C/D) or plain mean shift
 * (Alg. 1, opt->all_seeds = 1) of n points in R^d.
 *
 *   points       [n x d] float32, device.  1 <= d <= FMS_MAX_DIM, n >= 1.
 *   h            Gaussian bandwidth, > 0.
 *   tol          convergence radius: a seed has converged when one update
 *                moves it by at most tol (in point units); 0 -> 1e-3*h.
 *   max_iter     cap on updates per seed (> 0).
 *   out_modes    [max_modes x d] float32, device: the modes, in canonical
 *                order: density descending (sum w of the mode's last
 *                refinement update, one step of at most 1e-5*h before the
 *                mode, so within O(1e-10) relative of the KDE value at the
 *                mode), ties by coordinates.
 *   out_n_modes  host int32: M.  If M > max_modes, FMS_ERR_CAPACITY is
 *                returned, *out_n_modes = M and out_modes holds the first
 *                max_modes modes; labels are still written.
 *   out_labels   [n] int32, device: index of the nearest mode (ties -> lowest).
 *   out_margins  [n] float32, device, nullable: distance to the second-nearest
 *                mode minus distance to the nearest (+inf when M = 1).
 *   workspace    device buffer of >= fms_workspace_size(n, d, opt) bytes,
 *                256-byte aligned; NULL -> the call allocates one with
 *                cudaMallocAsync on `stream` and frees it before returning.
 *   stats        host, nullable.
 * Synchronises `stream` once per seed round and once at the end; a call
 * repeated with the same pointers, sizes, scalars and options and a caller
 * workspace runs as one cached CUDA graph and synchronises once
 * (stats->graph = 1).
 */
fms_status fms_cluster(const float* points, int64_t n, int32_t d, float h, float tol,
                       int32_t max_iter, const fms_options* opt, float* out_modes,
                       int32_t max_modes, int32_t* out_n_modes, int32_t* out_labels,
                       float* out_margins, void* workspace, size_t workspace_bytes,
                       fms_stats* stats, void* stream);

/*
 * fms_cluster with HOST input and output buffers (the same clustering, Alg. 2
 * or Alg. 1): the call copies the points to the device, clusters them and
 * copies the labels, margins and modes back, with the copy-backs queued on
 * `stream` before the call's final synchronisation (one synchronisation in
 * the CUDA-graph form).  Page-locked host buffers make the copies
 * asynchronous; pageable ones work but are staged by the driver.
 *
 *   points       HOST [n x d] float32.
 *   out_modes    HOST [max_modes x d] float32 (the first min(M, max_modes)
 *                rows are the modes in canonical order); nullable when
 *                max_modes = 0.
 *   out_n_modes  host int32: M (FMS_ERR_CAPACITY as in fms_cluster).
 *   out_labels   HOST [n] int32; out_margins HOST [n] float32, nullable.
 *   workspace    DEVICE buffer of >= fms_cluster_host_workspace_size(n, d,
 *                max_modes, opt) bytes, 256-byte aligned (it holds the
 *                clustering workspace and device copies of the inputs and
 *                outputs); NULL -> allocated with cudaMallocAsync and freed.
 * The host output buffers are written when the call returns FMS_OK or
 * FMS_ERR_CAPACITY.  Page-locked (pinned) host buffers are used in place: the
 * packing and label kernels read the points and write the labels and margins
 * through their mapped addresses instead of staging copies (after an error
 * such buffers may hold partial results); pageable buffers are copied.
 */
size_t fms_cluster_host_workspace_size(int64_t n, int32_t d, int32_t max_modes,
                                       const fms_options* opt);
fms_status fms_cluster_host(const float* points, int64_t n, int32_t d, float h, float tol,
                            int32_t max_iter, const fms_options* opt, float* out_modes,
                            int32_t max_modes, int32_t* out_n_modes, int32_t* out_labels,
                            float* out_margins, void* workspace, size_t workspace_bytes,
                            fms_stats* stats, void* stream);

/*
 * Batched Faster Mean-shift: B independent point sets of uneven size
 * clustered together, every phase of Alg. 2 (Sec. II-C/D) one launch for all
 * sets (the sets share h, tol, max_iter and the options).  The paper clusters
 * one set per call; batching has no counterpart there.
 *
 *   points       [offsets[B] x d] float32, device: set b is rows
 *                offsets[b] .. offsets[b+1]-1.
 *   offsets      HOST int64[B+1], offsets[0] = 0, strictly increasing.
 *   out_modes    [B x max_modes x d] float32, device: set b's modes at
 *                out_modes + b*max_modes*d, canonical order.
 *   out_n_modes  DEVICE int32[B]: each set's mode count (FMS_ERR_CAPACITY if
 *                any exceeds max_modes; the counts are still written).
 *   out_labels   [offsets[B]] int32, device: index of the nearest mode of the
 *                point's own set; out_margins as in fms_cluster (nullable).
 *   workspace    fms_batched_workspace_size(offsets, B, d, opt) bytes or NULL.
 * opt->seed_indices must be NULL.  Any set size and seed count is accepted:
 * a set's prune runs in shared memory while its candidates' sort keys fit
 * there and in global memory beyond that (same result).
 * The whole call is one CUDA graph launched on `stream`: its updates, seed
 * rounds and refinement updates are conditional WHILE nodes whose conditions
 * the kernels set, so no host decision interrupts it; the call synchronises
 * `stream` once, at the end, to read the status and the statistics
 * (stats->graph = 1; stats->kernel_launches counts the kernels the graph ran).
 * The graph is built on the first call with a given (pointers, B, total,
 * largest set, d, h, tol, max_iter, max_modes, options) and reused by later
 * calls with the same values; the per-set sizes are copied in before every
 * launch.  The step kernel's tiling is chosen by a built-in autotuner the
 * first time a shape (d, size class of the total, size class of B) is seen
 * on a device: it times one update with each candidate tiling (synchronising
 * on each) and keeps the fastest.
 * Errors: FMS_ERR_INVALID_ARG (bad sizes, offsets or options),
 * FMS_ERR_WORKSPACE (workspace too small or not 256-byte aligned),
 * FMS_ERR_NONFINITE (a non-finite point), FMS_ERR_CAPACITY (see out_n_modes),
 * FMS_ERR_CUDA (a CUDA call failed, including the graph's construction).
 */
size_t fms_batched_workspace_size(const int64_t* offsets, int32_t B, int32_t d,
                                  const fms_options* opt);
fms_status fms_cluster_batched(const float* points, const int64_t* offsets, int32_t B, int32_t d,
                               float h, float tol, int32_t max_iter, const fms_options* opt,
                               float* out_modes, int32_t max_modes, int32_t* out_n_modes,
                               int32_t* out_labels, float* out_margins, void* workspace,
                               size_t workspace_bytes, fms_stats* stats, void* stream);

/*
 * Faster Mean-shift over a sequence of F frames of n points each (Sec. II-D,
 * the video / tracking use).  Frame f is clustered exactly as fms_cluster with
 * opt->n_initial = N_f (doubling inside the frame while N < L*M as usual),
 * N_0 = opt->n_initial (0 -> 128).  When frame f ends with N seeds and M
 * modes, the next frame starts with N_{f+1} = N - M if N > H*M, else N (the
 * paper's seed reduction for nearly identical consecutive frames).
 *   frames          [F][n][d] float32, device.
 *   H               seed-reduction factor; <= 0 -> 32 (the paper's value).
 *   out_modes       [F][max_modes][d] device; out_n_modes [F] host;
 *   out_labels      [F][n] device; out_margins [F][n] device, nullable;
 *   out_seed_counts [F] host, nullable: N_f, the seed count frame f started with.
 *   workspace       >= fms_workspace_size(n, d, opt) bytes (reused by every
 *                   frame) or NULL (allocated once on `stream`).
 *   stats           nullable: iterations, rounds, evaluations and launches
 *                   summed over the frames; the other fields of the last frame.
 * opt->all_seeds and opt->seed_indices fix N and are rejected.  The call
 * synchronises once per frame: the next frame's seed count is decided on the
 * host, as in the paper's flowchart.  FMS_ERR_CAPACITY if any frame had more
 * than max_modes modes (all frames are still processed).
 */
fms_status fms_cluster_frames(const float* frames, int32_t F, int64_t n, int32_t d, float h,
                              float tol, int32_t max_iter, const fms_options* opt, float H,
                              float* out_modes, int32_t max_modes, int32_t* out_n_modes,
                              int32_t* out_labels, float* out_margins, int32_t* out_seed_counts,
                              void* workspace, size_t workspace_bytes, fms_stats* stats,
                              void* stream);

/*
 * Seed Selection (Alg. 2): writes entries [start, start+count) of a
 * keyed pseudo-random permutation pi of [0, n) to out_indices (device int32).
 * pi(i) applies a balanced 6-round Feistel network on 2*hb bits (4^hb the
 * smallest power of four >= n, hb >= 1) whose round r XORs the left half with
 * the low hb bits of mix64(k_r ^ right), and repeats it while the result is
 * >= n (cycle walking).  mix64 is the SplitMix64 output function and k_r
 * (r = 0..5) are the first six SplitMix64 outputs of the stream seeded with
 * rng_seed.  Requires 1 <= n < 2^31, 0 <= start, start+count <= n.
 * Asynchronous.
 */
fms_status fms_select_seeds(int64_t n, uint64_t rng_seed, int64_t start, int64_t count,
                            int32_t* out_indices, void* stream);

/*
 * One Gaussian mean-shift update of m seeds against all n points (Eq. 6 with
 * the Gaussian weight; the update of Alg. 2):
 *   out_seeds[i] = sum_j w_ij x_j / sum_j w_ij,  w_ij = exp(-||seeds_i - x_j||^2/(2h^2)).
 *   seeds, out_seeds  [m x d] float32, device (may alias).
 *   out_wsum     [m] float32, device, nullable: sum_j w_ij.
 *   workspace    >= fms_step_workspace_size(n, d, m) bytes or NULL (allocated).
 * Asynchronous unless workspace is NULL.
 */
size_t fms_step_workspace_size(int64_t n, int32_t d, int64_t m);
fms_status fms_mean_shift_step(const float* points, int64_t n, int32_t d, float h,
                               const float* seeds, int64_t m, float* out_seeds,
                               float* out_wsum, void* workspace, size_t workspace_bytes,
                               void* stream);

/*
 * One coarse mean-shift update on the tensor cores, for 1 <= d <= 32
 * (FMS_ERR_UNSUPPORTED above): the same update as fms_mean_shift_step with the
 * weights evaluated at reduced precision.  In scaled coordinates
 * (u = s*x, s = sqrt(log2(e)/(2h^2)), so w = 2^-||u_y - u_x||^2), the cross
 * term u_y.u_x is a tensor-core product of BF16 hi/lo splits of both
 * operands (hi*hi + hi*lo + lo*hi, FP32 accumulation), the squared norms are
 * FP32, w = 2^(2 u_y.u_x - ||u_y||^2 - ||u_x||^2) is rounded to BF16, and
 * sum w and sum w*x are a second tensor-core product of those weights with
 * the BF16 hi/lo split of the points (FP32 accumulation).  The result agrees
 * with the FP32 update to about 2^-8 relative in each weight; it is the
 * "coarse" step that fms_cluster's FMS_PRECISION_TENSOR uses until a seed's
 * move drops to 10*tol.  The paper (Sec. II-B) evaluates every weight in full
 * precision; this step is the library's tensor-core formulation of the same
 * sums.  Arguments as fms_mean_shift_step; workspace
 * >= fms_coarse_step_workspace_size(n, d, m) bytes (0 for unsupported sizes)
 * or NULL.  FMS_ERR_TIMEOUT if a bounded wait for the tensor cores gave up
 * (reported only when workspace is NULL, i.e. when the call synchronises).
 */
size_t fms_coarse_step_workspace_size(int64_t n, int32_t d, int64_t m);
fms_status fms_mean_shift_step_coarse(const float* points, int64_t n, int32_t d, float h,
                                      const float* seeds, int64_t m, float* out_seeds,
                                      float* out_wsum, void* workspace, size_t workspace_bytes,
                                      void* stream);

/*
 * One mean-shift update, as fms_mean_shift_step, for callers that cannot
 * allocate device memory: real-time or allocator-free runtimes where
 * cudaMalloc / cudaFree (which may synchronise the device) are not allowed
 * while work is in flight, and hosts that have no memory pool to lend the
 * library a workspace.  The paper has no counterpart; this is a deployment
 * convenience.
 *
 * The call allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine).  Its scratch is one fixed array of FMS_NOALLOC_SCRATCH_BYTES that
 * is part of the library image, so every GPU on which the library is loaded
 * holds that much device memory until the process exits.  A request whose
 * scratch would not fit -- fms_step_workspace_size(n, d, m) larger than
 * FMS_NOALLOC_SCRATCH_BYTES -- is refused with FMS_ERR_WORKSPACE before any
 * device work.  Every call looks up the array's device address in the
 * current device's context (cudaGetSymbolAddress, which enqueues no work), so
 * the call stays valid after that context has been reset or recreated.  The
 * first call on a device may load the library's device code; make that first
 * call before capturing the stream into a graph.
 *
 * All calls share the one array and it keeps the previous call's contents:
 * the call clears what must start at zero itself, but calls that overlap on
 * the GPU (other streams, other host threads) race on the array and must be
 * serialised by the caller.
 *   points [n x d], seeds/out_seeds [m x d] float32, device; out_wsum [m] or
 *   NULL.  Asynchronous on `stream`; non-finite input is not reported (the
 *   outputs are then not finite).
 */
#define FMS_NOALLOC_SCRATCH_BYTES (16u << 20)
fms_status fms_mean_shift_step_noalloc(const float* points, int64_t n, int32_t d, float h,
                                       const float* seeds, int64_t m, float* out_seeds,
                                       float* out_wsum, void* stream);

/*
 * Measured pipe rates of the current device, per clock and per SM (median
 * over SMs, SM cycle counter around a fixed instruction mix on every SM).
 * The paper has no counterpart: these are the throughputs that the roofline
 * of the evaluation kernels divides by, measured rather than taken from data
 * sheets.  rates[0] FFMA FP32 ops, [1] packed FFMA2 (f32x2) FP32 ops,
 * [2] MUFU ex2, [3] units of 10 FFMA + 1 ex2 (the exact-difference evaluation
 * mix at d = 3); the first min(n_rates, 4) are written.  Synchronous; takes
 * a few milliseconds and allocates (a diagnostic, not for hot paths).
 */
fms_status fms_probe_pipe_rates(double* rates, int32_t n_rates);

/*
 * Measured BF16 tensor-core rate of the current device (tcgen05.mma.kind::f16,
 * M = 128, K = 16, FP32 accumulation in tensor memory), from one bounded
 * launch per configuration with one CTA per SM (bounded mbarrier waits; the
 * tensor memory is freed before the CTA exits).  rates[2 i] (one issuing
 * thread per SM) and rates[2 i + 1] (two issuing threads in different warps)
 * are FLOP per clock per SM of completed MMAs for N = 16, 32, 64, 128, 256
 * (i = 0 .. 4), the median over SMs; multiply by the SM clock and the SM
 * count for FLOP/s.  Writes min(n_rates, 10) entries; a negative entry means
 * a wait gave up.  Synchronises the device.  FMS_ERR_INVALID_ARG (null or
 * n_rates < 1), FMS_ERR_CUDA.
 */
fms_status fms_probe_tensor_rates(double* rates, int32_t n_rates);

/*
 * Nearest-mode labelling (the labelling of Alg. 2): labels[j] = argmin_k
 * ||x_j - modes_k|| (ties -> lowest k) and, if margins is non-NULL,
 * margins[j] = second-nearest minus nearest distance (+inf when M = 1).
 * points [n x d], modes [M x d] float32, device; M >= 1.  Asynchronous.
 */
fms_status fms_label_points(const float* points, int64_t n, int32_t d, const float* modes,
                            int32_t M, int32_t* labels, float* margins, void* stream);

/*
 * Differentiable unrolled mean shift: T Gaussian updates of every seed of B
 * independent sets (no Seed Selection, no stopping; all seeds move T times),
 * and the adjoint of that map, for training embeddings through the
 * clustering.  The paper has no counterpart; the update is Eq. 6 with the
 * Gaussian weight.  With p_ij = w_ij / sum_j w_ij, mu_i = sum_j p_ij x_j,
 * g_i = dL/dmu_i and a_ij = g_i . (x_j - mu_i), one update contributes
 *   dL/dy_i  = (1/h^2) sum_j p_ij a_ij (x_j - mu_i)
 *   dL/dx_j += p_ij [g_i - a_ij (x_j - y_i)/h^2]
 *   dL/dh   += (1/h^3) sum_ij p_ij ||y_i - x_j||^2 a_ij.
 * Weights are recomputed tile by tile (nothing of size m x n is stored); the
 * forward stores the positions every k updates and at the end (Y_T), and each
 * update's W_i and weight shift (one value per seed), in `ckpt`; the backward
 * recomputes the positions between two checkpoints one segment at a time.
 * A seed whose sum of weights underflows (every point farther than ~13 h in
 * FP32) is recomputed with its weights taken relative to its nearest point.
 *
 *   points  [B x n x d], seeds0 [B x m x d], out_seeds [B x m x d]: float32,
 *           device, row-major; 1 <= d <= 32.  h > 0, T >= 1, k >= 1.
 *   ckpt    opaque device buffer of fms_unrolled_ckpt_size() bytes (16-byte
 *           aligned), written by the forward and read by the backward.
 *   ws      device workspace of fms_unrolled_workspace_size() bytes, 256-byte
 *           aligned (the same size serves both directions).
 *   grad_out [B x m x d] = dL/dY_T; grad_points [B x n x d] and grad_seeds0
 *           [B x m x d] are overwritten; grad_h [B] (float64, device) receives
 *           dL/dh of each set.
 * Both calls are asynchronous on `stream`.  Errors: FMS_ERR_INVALID_ARG (null
 * pointer, sizes out of range, h not finite and positive), FMS_ERR_WORKSPACE
 * (buffers too small or misaligned), FMS_ERR_CUDA (a launch failed).  The
 * pair kernels stage rows in shared memory with bulk copies whose waits are
 * bounded; a wait that gives up turns the affected outputs into NaN (the
 * calls do not synchronise, so it is reported through the results).
 *
 * The *_f64 entry points are the same computation in FP64 (double pointers,
 * h as double; `ckpt` and `ws` sized by the *_f64 size functions), for
 * checking gradients by finite differences on the GPU; the FP32 entry points
 * are the fast path.
 */
size_t fms_unrolled_ckpt_size(int32_t B, int64_t n, int64_t m, int32_t d, int32_t T, int32_t k);
size_t fms_unrolled_workspace_size(int32_t B, int64_t n, int64_t m, int32_t d, int32_t T,
                                   int32_t k);
fms_status fms_unrolled_forward(const float* points, const float* seeds0, int32_t B, int64_t n,
                                int64_t m, int32_t d, float h, int32_t T, int32_t k,
                                float* out_seeds, void* ckpt, size_t ckpt_bytes, void* ws,
                                size_t ws_bytes, void* stream);
fms_status fms_unrolled_backward(const float* points, int32_t B, int64_t n, int64_t m, int32_t d,
                                 float h, int32_t T, int32_t k, const void* ckpt,
                                 size_t ckpt_bytes, const float* grad_out, float* grad_points,
                                 float* grad_seeds0, double* grad_h, void* ws, size_t ws_bytes,
                                 void* stream);
size_t fms_unrolled_ckpt_size_f64(int32_t B, int64_t n, int64_t m, int32_t d, int32_t T,
                                  int32_t k);
size_t fms_unrolled_workspace_size_f64(int32_t B, int64_t n, int64_t m, int32_t d, int32_t T,
                                       int32_t k);
fms_status fms_unrolled_forward_f64(const double* points, const double* seeds0, int32_t B,
                                    int64_t n, int64_t m, int32_t d, double h, int32_t T,
                                    int32_t k, double* out_seeds, void* ckpt, size_t ckpt_bytes,
                                    void* ws, size_t ws_bytes, void* stream);
fms_status fms_unrolled_backward_f64(const double* points, int32_t B, int64_t n, int64_t m,
                                     int32_t d, double h, int32_t T, int32_t k, const void* ckpt,
                                     size_t ckpt_bytes, const double* grad_out,
                                     double* grad_points, double* grad_seeds0, double* grad_h,
                                     void* ws, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FMS_H */
