// C ABI of the batched clustering (fms_cluster_batched): many independent
// point sets, every phase one launch for all sets (k_batched.cu), the whole
// call one CUDA graph whose loops (updates, seed rounds, refinement) are
// conditional WHILE nodes driven by the kernels, plus the project's tile
// autotuner for the batched step kernel.
#include <math.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/fms.h"
#include "fms_internal.cuh"

namespace fms {
cudaError_t launch_batched_seed_init(SetCtl* sc, int B, const float* Xs, int DP, uint64_t seed,
                                     float* y, int32_t* it, int32_t* conv, int32_t* state,
                                     cudaStream_t st);
cudaError_t launch_batched_compact(SetCtl* sc, int B, const int32_t* state, const int32_t* it,
                                   const int32_t* conv, int32_t* active, int begin, int max_iter,
                                   int R, int DA, Tiling tl, int64_t* task_off, int64_t* part_off,
                                   int64_t* list_off, int64_t* totals, int32_t* counters,
                                   BatchCond cond, const uint32_t* status, cudaStream_t st);
cudaError_t launch_batched_step(const float* Xs, int d, int DP, const float* y,
                                const int32_t* list, const SetCtl* sc, int B, int kind,
                                const int64_t* task_off, const int64_t* part_off,
                                const int64_t* totals, float* part, int target_warps,
                                uint32_t* status, cudaStream_t st);
cudaError_t launch_batched_update(const float* part, const int32_t* active, const SetCtl* sc,
                                  int B, const int64_t* list_off, const int64_t* part_off,
                                  const int64_t* totals, float* y, int32_t* it, int32_t* conv,
                                  int32_t* state, int d, int DP, int DA, float tol2_s,
                                  int max_iter, int grid, cudaStream_t st);
cudaError_t launch_batched_kept(SetCtl* sc, int B, const int32_t* state, const int32_t* conv,
                                int keep_exhausted, int32_t* kept, int R, int DA, Tiling tl,
                                int64_t* task_off, int64_t* part_off, int64_t* list_off,
                                int64_t* totals, int32_t* counters, cudaStream_t st);
cudaError_t launch_batched_score(const float* part, const SetCtl* sc, int B,
                                 const int64_t* list_off, const int64_t* part_off,
                                 const int64_t* totals, int DA, float* score, int grid,
                                 cudaStream_t st);
cudaError_t launch_batched_prune_f(SetCtl* sc, int B, const int32_t* kept, const float* score,
                                   const float* pos, int DP, int d, float r2, int32_t* accepted,
                                   int32_t* list, int maxK, cudaStream_t st);
cudaError_t launch_batched_prune_d(SetCtl* sc, int B, const double* score, const double* pos,
                                   int DP, int d, double r2, int32_t* accepted, int32_t* list,
                                   int maxK, cudaStream_t st);
cudaError_t launch_batched_advance(SetCtl* sc, int B, float L, int allow, float gamma,
                                   int32_t* counters, BatchCond cond, const uint32_t* status,
                                   cudaStream_t st);
cudaError_t launch_batched_refine_setup(SetCtl* sc, int B, const float* y, const int32_t* kept,
                                        const int32_t* accepted, int DP, double* ym, float* yf,
                                        int32_t* ract, int32_t* mdone, int init_pos, int R,
                                        Tiling tl, cudaStream_t st);
cudaError_t launch_plan(const SetCtl* sc, int B, int kind, int R, int DA, int64_t* task_off,
                        int64_t* part_off, int64_t* list_off, int64_t* totals, BatchCond cond,
                        const uint32_t* status, cudaStream_t st);
cudaError_t launch_batched_refine_update(const float* part, const int32_t* ract, const SetCtl* sc,
                                         int B, const int64_t* list_off, const int64_t* part_off,
                                         const int64_t* totals, double* ym, float* yf,
                                         int32_t* mdone, double* mscore, int d, int DP, int DA,
                                         double tol2_s, int score_only, int grid,
                                         cudaStream_t st);
cudaError_t launch_batched_refine_compact(SetCtl* sc, int B, const int32_t* mdone, int32_t* ract,
                                          int max_iter, int R, int DA, Tiling tl,
                                          int64_t* task_off, int64_t* part_off, int64_t* list_off,
                                          int64_t* totals, int32_t* counters, BatchCond cond,
                                          const uint32_t* status, cudaStream_t st);
cudaError_t launch_batched_canonical(const SetCtl* sc, int B, const double* ym,
                                     const double* mscore, const int32_t* acc2, int d, int DP,
                                     double inv_scale, float* out_modes, int max_modes,
                                     float* modes_full, int32_t* out_n, cudaStream_t st);
cudaError_t launch_batched_label(const float* X, const int64_t* pt_off, int B, int d,
                                 const SetCtl* sc, const float* modes_full, int32_t* labels,
                                 float* margins, int64_t total, cudaStream_t st);
}  // namespace fms

using namespace fms;

namespace {

constexpr int kTwMultMax = 2;  // largest warp multiplier the autotuner tries
constexpr int kRefineMax = 50;
enum : int { kPlanActive = 0, kPlanKept = 1, kPlanModes = 2 };

size_t a256(size_t x) { return (x + 255) / 256 * 256; }

int padded(int d) { return padded_dim(d); }

int sms_now() {
  int dev = 0, s = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return s;
}

struct BLayout {
  size_t Xs, y, it, conv, state, active, kept, acc1, acc2, plist, score, ym, yf, ract, mdone,
      mscore, modes_full, part, sc, task_off, part_off, list_off, totals, counters, pt_off, status,
      total;
  int DP, DA, R, TW;
  Tiling tl;
};

// Partial-sum capacity: per set C_b * cnt_b * DA with C_b from choose_chunks
// (<= 4 * tl.target_warps / G_b + 1), so sum_b <= (4 * TWb * B + total_groups) * R * DA.
BLayout make_blayout(int64_t total, int B, int d, int sms, int tw_mult, int min_chunk) {
  BLayout L{};
  L.DP = padded(d);
  L.DA = step_accumulators(d);
  L.R = batched_seeds_per_warp(d);
  L.TW = (sms > 0 ? sms : 1) * step_resident_warps_per_sm(d);
  // every set gets a share of the GPU's warps for its chunking (all sets run
  // in the same launches)
  int twb = (L.TW * tw_mult) / (B > 0 ? B : 1);
  if (twb < 32) twb = 32;
  L.tl.target_warps = twb;
  L.tl.min_chunk = min_chunk;
  // partial sums sized for the largest autotuner candidate, so that every
  // candidate tiling fits the same layout
  int twb_max = (L.TW * kTwMultMax) / (B > 0 ? B : 1);
  if (twb_max < 32) twb_max = 32;
  const int64_t groups = total / L.R + B;
  const size_t part_floats = (size_t)(4 * (int64_t)twb_max * B + groups + 1) * L.R * L.DA;
  size_t o = 0;
  auto take = [&](size_t b) {
    size_t at = o;
    o += a256(b > 0 ? b : 1);
    return at;
  };
  L.Xs = take((size_t)total * L.DP * 4);
  L.y = take((size_t)total * L.DP * 4);
  L.it = take((size_t)total * 4);
  L.conv = take((size_t)total * 4);
  L.state = take((size_t)total * 4);
  L.active = take((size_t)total * 4);
  L.kept = take((size_t)total * 4);
  L.acc1 = take((size_t)total * 4);
  L.acc2 = take((size_t)total * 4);
  L.plist = take((size_t)total * 4);
  L.score = take((size_t)total * 4);
  L.ym = take((size_t)total * L.DP * 8);
  L.yf = take((size_t)total * L.DP * 4);
  L.ract = take((size_t)total * 4);
  L.mdone = take((size_t)total * 4);
  L.mscore = take((size_t)total * 8);
  L.modes_full = take((size_t)total * d * 4);
  L.part = take(part_floats * 4);
  L.sc = take((size_t)B * sizeof(SetCtl));
  L.task_off = take((size_t)(B + 1) * 8);
  L.part_off = take((size_t)(B + 1) * 8);
  L.list_off = take((size_t)(B + 1) * 8);
  L.totals = take(64);
  L.counters = take(64);
  L.pt_off = take((size_t)(B + 1) * 8);
  L.status = take(64);
  L.total = o;
  return L;
}

// Autotuner state: best (tw_mult, min_chunk) per (device, d, log2 total, B bucket).
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_tuned;
const int kTwMults[2] = {1, 2};
const int kMinChunksLow[3] = {256, 512, 1024};
const int kMinChunksWide[3] = {32, 64, 128};

template <typename T>
T* at(void* base, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}

int ilog2(int64_t x) {
  int r = 0;
  while ((int64_t(1) << (r + 1)) <= x) ++r;
  return r;
}

// ---------------------------------------------------------------------------
// The call as one CUDA graph.  A graph bakes in its pointers, launch shapes
// and scalars, so it is kept per (arguments, options, tiling, device); the
// per-set control blocks and point offsets are copied in before every launch,
// so sets of other sizes with the same count, total and largest size reuse it.
// ---------------------------------------------------------------------------
struct BGraphKey {
  const void* points;
  const void* modes;
  const void* n_modes;
  const void* labels;
  const void* margins;
  const void* ws;
  int64_t total;
  int32_t B, d, max_iter, max_modes, max_n, dev, tw_mult, min_chunk;
  float h, tol;
  unsigned char opts[sizeof(fms_options)];
};

struct BGraphCache {
  static constexpr int kEntries = 4;
  BGraphKey key[kEntries];
  cudaGraphExec_t exec[kEntries] = {};
  int used = 0, next = 0;
  ~BGraphCache() {
    for (int i = 0; i < used; ++i)
      if (exec[i]) cudaGraphExecDestroy(exec[i]);
  }
};

BGraphCache& bgraph_cache() {
  thread_local BGraphCache c;
  return c;
}

// Private capture streams (per device; one per nesting level), kept for the
// thread's life.
cudaStream_t bcapture_stream(int dev, int level) {
  constexpr int kMaxDevices = 64;
  thread_local cudaStream_t s[kMaxDevices][3] = {};
  if (dev < 0 || dev >= kMaxDevices || level < 0 || level > 2) return nullptr;
  if (!s[dev][level] &&
      cudaStreamCreateWithFlags(&s[dev][level], cudaStreamNonBlocking) != cudaSuccess)
    s[dev][level] = nullptr;
  return s[dev][level];
}

// During capture on `cs`: a WHILE node after the captured work; capture of its
// body (returned in *body) begins on `body_cs`; further capture on `cs`
// depends on the node.
cudaError_t begin_while(cudaStream_t cs, cudaGraphConditionalHandle h, cudaStream_t body_cs,
                        cudaGraph_t* body) {
  cudaStreamCaptureStatus cst;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  if (cst != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, cg, deps, nullptr, nd, &np);
  if (e != cudaSuccess) return e;
  e = cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) return e;
  *body = np.conditional.phGraph_out[0];
  return cudaStreamBeginCaptureToGraph(body_cs, *body, nullptr, nullptr, 0,
                                       cudaStreamCaptureModeThreadLocal);
}

cudaError_t end_body(cudaStream_t body_cs, cudaError_t e) {
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(body_cs, &g);
  return e != cudaSuccess ? e : e2;
}

}  // namespace

extern "C" {


size_t fms_batched_workspace_size(const int64_t* offsets, int32_t B, int32_t d,
                                  const fms_options* opt) {
  (void)opt;
  if (!offsets || B < 1 || d < 1 || d > FMS_MAX_DIM) return 0;
  const int64_t total = offsets[B] - offsets[0];
  if (total < 1 || total > INT32_MAX) return 0;
  return make_blayout(total, B, d, sms_now(), kTwMults[0], 32).total;
}

fms_status fms_cluster_batched(const float* points, const int64_t* offsets, int32_t B, int32_t d,
                               float h, float tol, int32_t max_iter, const fms_options* opt_in,
                               float* out_modes, int32_t max_modes, int32_t* out_n_modes,
                               int32_t* out_labels, float* out_margins, void* workspace,
                               size_t workspace_bytes, fms_stats* stats, void* stream_) {
  fms_options o;
  fms_options_default(&o);
  if (opt_in) {
    o.all_seeds = opt_in->all_seeds;
    if (opt_in->n_initial > 0) o.n_initial = opt_in->n_initial;
    if (opt_in->L > 0.f) o.L = opt_in->L;
    if (opt_in->gamma > 0.f) o.gamma = opt_in->gamma;
    if (opt_in->merge_radius > 0.f) o.merge_radius = opt_in->merge_radius;
    o.skip_refine = opt_in->skip_refine;
    o.rng_seed = opt_in->rng_seed;
    o.seed_indices = opt_in->seed_indices;
    o.profile = opt_in->profile;
    o.kernel = opt_in->kernel;
    o.metric = opt_in->metric;
  }
  if (stats) memset(stats, 0, sizeof(*stats));
  if (o.kernel != FMS_KERNEL_GAUSSIAN) return FMS_ERR_UNSUPPORTED;   // (flat: fms_cluster only)
  if (o.metric != FMS_METRIC_EUCLIDEAN) return FMS_ERR_UNSUPPORTED;   // (cosine: fms_cluster only)
  if (!points || !offsets || B < 1 || d < 1 || d > FMS_MAX_DIM || !(h > 0.f) || !isfinite(h) ||
      !(tol >= 0.f) || max_iter < 1 || !out_labels || !out_n_modes || max_modes < 0 ||
      (max_modes > 0 && !out_modes) || o.seed_indices || !(o.gamma > 0.f && o.gamma <= 1.f))
    return FMS_ERR_INVALID_ARG;
  if (offsets[0] != 0) return FMS_ERR_INVALID_ARG;
  for (int b = 0; b < B; ++b)
    if (offsets[b + 1] <= offsets[b]) return FMS_ERR_INVALID_ARG;
  const int64_t total = offsets[B];
  if (total > INT32_MAX) return FMS_ERR_INVALID_ARG;
  if (tol == 0.f) tol = 1e-3f * h;
  if (o.all_seeds) o.gamma = 1.f;
  cudaStream_t st = static_cast<cudaStream_t>(stream_);
  const int sms = sms_now();
  if (sms <= 0) return FMS_ERR_CUDA;

  // tuned tiling for this shape (or the first candidate until tuned)
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_tuple(dev, (int)d, ilog2(total), ilog2(B));
  bool tuned = false;
  std::pair<int, int> cfg{kTwMults[0], d <= 7 ? kMinChunksLow[1] : kMinChunksWide[1]};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto itc = g_tuned.find(key);
    if (itc != g_tuned.end()) {
      cfg = itc->second;
      tuned = true;
    }
  }
  BLayout Lo = make_blayout(total, B, d, sms, cfg.first, cfg.second);
  const size_t need = Lo.total;  // identical for every candidate tiling
  bool owns = false;
  void* ws = workspace;
  if (ws) {
    if (workspace_bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255u)) return FMS_ERR_WORKSPACE;
  } else {
    if (cudaMallocAsync(&ws, need, st) != cudaSuccess) return FMS_ERR_CUDA;
    owns = true;
  }
  fms_status rc = FMS_OK;
  std::vector<SetCtl> hsc(B);
  int32_t hcnt[4] = {0, 0, 0, 0};
  uint32_t hstatus = 0;
#define BC(call)                \
  do {                          \
    if ((call) != cudaSuccess) { \
      rc = FMS_ERR_CUDA;        \
      goto done;                \
    }                           \
  } while (0)
  {
    const int DP = Lo.DP, DA = Lo.DA, R = Lo.R;
    float* Xs = at<float>(ws, Lo.Xs);
    float* y = at<float>(ws, Lo.y);
    int32_t* it = at<int32_t>(ws, Lo.it);
    int32_t* conv = at<int32_t>(ws, Lo.conv);
    int32_t* state = at<int32_t>(ws, Lo.state);
    int32_t* active = at<int32_t>(ws, Lo.active);
    int32_t* kept = at<int32_t>(ws, Lo.kept);
    int32_t* acc1 = at<int32_t>(ws, Lo.acc1);
    int32_t* acc2 = at<int32_t>(ws, Lo.acc2);
    int32_t* plist = at<int32_t>(ws, Lo.plist);
    float* score = at<float>(ws, Lo.score);
    double* ym = at<double>(ws, Lo.ym);
    float* yf = at<float>(ws, Lo.yf);
    int32_t* ract = at<int32_t>(ws, Lo.ract);
    int32_t* mdone = at<int32_t>(ws, Lo.mdone);
    double* mscore = at<double>(ws, Lo.mscore);
    float* modes_full = at<float>(ws, Lo.modes_full);
    float* part = at<float>(ws, Lo.part);
    SetCtl* sc = at<SetCtl>(ws, Lo.sc);
    int64_t* task_off = at<int64_t>(ws, Lo.task_off);
    int64_t* part_off = at<int64_t>(ws, Lo.part_off);
    int64_t* list_off = at<int64_t>(ws, Lo.list_off);
    int64_t* totals = at<int64_t>(ws, Lo.totals);
    int32_t* counters = at<int32_t>(ws, Lo.counters);
    int64_t* pt_off = at<int64_t>(ws, Lo.pt_off);
    uint32_t* status = at<uint32_t>(ws, Lo.status);
    const double scale = sqrt(1.4426950408889634 / (2.0 * (double)h * (double)h));
    const double tol_s = (double)tol * scale;
    const float tol2_s = (float)(tol_s * tol_s);
    const double r_merge = o.merge_radius > 0.f ? (double)o.merge_radius : (double)h;
    const double r2_s = (r_merge * scale) * (r_merge * scale);
    const int grid_upd = sms * 8;
    const BatchCond no_cond{0, 0};
    int max_n = 1;

    for (int b = 0; b < B; ++b) {
      SetCtl& c = hsc[b];
      memset(&c, 0, sizeof(c));
      c.n = (int32_t)(offsets[b + 1] - offsets[b]);
      c.p0 = (int32_t)offsets[b];
      c.N = o.all_seeds ? c.n : (o.n_initial < c.n ? o.n_initial : c.n);
      c.prevN = 0;
      const int t = (int)ceil((double)o.gamma * (double)c.N);
      c.target = t < 1 ? 1 : (t > c.N ? c.N : t);
      if (c.n > max_n) max_n = c.n;
    }
    BC(cudaMemcpyAsync(sc, hsc.data(), (size_t)B * sizeof(SetCtl), cudaMemcpyHostToDevice, st));
    BC(cudaMemcpyAsync(pt_off, offsets, (size_t)(B + 1) * 8, cudaMemcpyHostToDevice, st));

    // --- autotune the step tiling once per shape: time one update per candidate ---
    if (!tuned) {
      BC(cudaMemsetAsync(counters, 0, 64, st));
      BC(cudaMemsetAsync(status, 0, 64, st));
      BC(launch_pack_points(points, total, d, DP, (float)scale, Xs, status, st));
      BC(launch_batched_seed_init(sc, B, Xs, DP, o.rng_seed, y, it, conv, state, st));
      float best_ms = 1e30f;
      std::pair<int, int> best = cfg;
      cudaEvent_t e0, e1;
      BC(cudaEventCreate(&e0));
      BC(cudaEventCreate(&e1));
      const int* cands = d <= 7 ? kMinChunksLow : kMinChunksWide;
      for (int tm : kTwMults)
        for (int ci = 0; ci < 3; ++ci) {
          const int mc = cands[ci];
          const BLayout Lc = make_blayout(total, B, d, sms, tm, mc);
          BC(launch_batched_compact(sc, B, state, it, conv, active, 1, max_iter, R, DA, Lc.tl,
                                    task_off, part_off, list_off, totals, counters, no_cond,
                                    status, st));
          BC(cudaEventRecord(e0, st));
          BC(launch_batched_step(Xs, d, DP, y, active, sc, B, kPlanActive, task_off, part_off,
                                 totals, part, Lc.TW, status, st));
          BC(cudaEventRecord(e1, st));
          BC(cudaEventSynchronize(e1));
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (ms < best_ms) {
            best_ms = ms;
            best = {tm, mc};
          }
        }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      // the trial compactions counted evaluations: the real run starts afresh
      BC(cudaMemcpyAsync(sc, hsc.data(), (size_t)B * sizeof(SetCtl), cudaMemcpyHostToDevice, st));
      cfg = best;
      Lo = make_blayout(total, B, d, sms, cfg.first, cfg.second);
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tuned[key] = cfg;
    }
    const Tiling tl = Lo.tl;

    // --- the graph of the whole call (built once per key) ---
    BGraphKey gk;
    memset(&gk, 0, sizeof(gk));
    gk.points = points;
    gk.modes = out_modes;
    gk.n_modes = out_n_modes;
    gk.labels = out_labels;
    gk.margins = out_margins;
    gk.ws = ws;
    gk.total = total;
    gk.B = B;
    gk.d = d;
    gk.max_iter = max_iter;
    gk.max_modes = max_modes;
    gk.max_n = max_n;
    gk.dev = dev;
    gk.tw_mult = cfg.first;
    gk.min_chunk = cfg.second;
    gk.h = h;
    gk.tol = tol;
    memcpy(gk.opts, &o, sizeof(fms_options));
    BGraphCache& gc = bgraph_cache();
    cudaGraphExec_t exec = nullptr;
    for (int i = 0; i < gc.used; ++i)
      if (memcmp(&gc.key[i], &gk, sizeof(gk)) == 0) exec = gc.exec[i];
    if (!exec) {
      cudaStream_t cs0 = bcapture_stream(dev, 0), cs1 = bcapture_stream(dev, 1),
                   cs2 = bcapture_stream(dev, 2);
      cudaGraph_t g = nullptr;
      cudaError_t e = (cs0 && cs1 && cs2) ? cudaGraphCreate(&g, 0) : cudaErrorNotSupported;
      cudaGraphConditionalHandle h_round = 0, h_upd = 0, h_ref = 0;
      bool capturing = false;
      if (e == cudaSuccess)
        e = cudaGraphConditionalHandleCreate(&h_round, g, 1, cudaGraphCondAssignDefault);
      if (e == cudaSuccess)
        e = cudaGraphConditionalHandleCreate(&h_ref, g, 0, cudaGraphCondAssignDefault);
      if (e == cudaSuccess)
        e = cudaStreamBeginCaptureToGraph(cs0, g, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal);
      capturing = e == cudaSuccess;
      // packing and the first seeds
      if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, 64, cs0);
      if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, 64, cs0);
      if (e == cudaSuccess)
        e = launch_pack_points(points, total, d, DP, (float)scale, Xs, status, cs0);
      if (e == cudaSuccess)
        e = launch_batched_seed_init(sc, B, Xs, DP, o.rng_seed, y, it, conv, state, cs0);
      // seed rounds: WHILE any set doubles its seed count
      cudaGraph_t round_body = nullptr;
      if (e == cudaSuccess) e = begin_while(cs0, h_round, cs1, &round_body);
      if (e == cudaSuccess) {
        cudaError_t e2 =
            cudaGraphConditionalHandleCreate(&h_upd, round_body, 0, cudaGraphCondAssignDefault);
        if (e2 == cudaSuccess)
          e2 = launch_batched_compact(sc, B, state, it, conv, active, 1, max_iter, R, DA, tl,
                                      task_off, part_off, list_off, totals, counters,
                                      BatchCond{h_upd, 1}, status, cs1);
        // updates of the round: WHILE any set has active seeds
        cudaGraph_t upd_body = nullptr;
        if (e2 == cudaSuccess) e2 = begin_while(cs1, h_upd, cs2, &upd_body);
        if (e2 == cudaSuccess) {
          cudaError_t e3 = launch_batched_step(Xs, d, DP, y, active, sc, B, kPlanActive, task_off,
                                               part_off, totals, part, Lo.TW, status, cs2);
          if (e3 == cudaSuccess)
            e3 = launch_batched_update(part, active, sc, B, list_off, part_off, totals, y, it,
                                       conv, state, d, DP, DA, tol2_s, max_iter, grid_upd, cs2);
          if (e3 == cudaSuccess)
            e3 = launch_batched_compact(sc, B, state, it, conv, active, 0, max_iter, R, DA, tl,
                                        task_off, part_off, list_off, totals, counters,
                                        BatchCond{h_upd, 1}, status, cs2);
          e2 = end_body(cs2, e3);
        }
        // prune: kept seeds, their densities, the per-set prune, seed-count decision
        if (e2 == cudaSuccess)
          e2 = launch_batched_kept(sc, B, state, conv, o.gamma >= 1.f ? 1 : 0, kept, R, DA, tl,
                                   task_off, part_off, list_off, totals, counters, cs1);
        if (e2 == cudaSuccess)
          e2 = launch_batched_step(Xs, d, DP, y, kept, sc, B, kPlanKept, task_off, part_off,
                                   totals, part, Lo.TW, status, cs1);
        if (e2 == cudaSuccess)
          e2 = launch_batched_score(part, sc, B, list_off, part_off, totals, DA, score, grid_upd,
                                    cs1);
        if (e2 == cudaSuccess)
          e2 = launch_batched_prune_f(sc, B, kept, score, y, DP, d, (float)r2_s, acc1, plist,
                                      max_n, cs1);
        if (e2 == cudaSuccess)
          e2 = launch_batched_advance(sc, B, o.L, o.all_seeds ? 0 : 1, o.gamma, counters,
                                      BatchCond{h_round, 1}, status, cs1);
        if (e2 == cudaSuccess)
          e2 = launch_batched_seed_init(sc, B, Xs, DP, o.rng_seed, y, it, conv, state, cs1);
        e = end_body(cs1, e2);
      }
      // refinement (FP64 positions) and the density at the refined modes
      if (e == cudaSuccess)
        e = launch_batched_refine_setup(sc, B, y, kept, acc1, DP, ym, yf, ract, mdone, 1, R, tl,
                                        cs0);
      if (!o.skip_refine) {
        const double rtol_s = 1e-5 * (double)h * scale;
        if (e == cudaSuccess)
          e = launch_plan(sc, B, kPlanModes, R, DA, task_off, part_off, list_off, totals,
                          BatchCond{h_ref, 1}, status, cs0);
        cudaGraph_t ref_body = nullptr;
        if (e == cudaSuccess) e = begin_while(cs0, h_ref, cs1, &ref_body);
        if (e == cudaSuccess) {
          cudaError_t e2 = launch_batched_step(Xs, d, DP, yf, ract, sc, B, kPlanModes, task_off,
                                               part_off, totals, part, Lo.TW, status, cs1);
          if (e2 == cudaSuccess)
            e2 = launch_batched_refine_update(part, ract, sc, B, list_off, part_off, totals, ym,
                                              yf, mdone, mscore, d, DP, DA, rtol_s * rtol_s, 0,
                                              grid_upd, cs1);
          if (e2 == cudaSuccess)
            e2 = launch_batched_refine_compact(sc, B, mdone, ract, kRefineMax, R, DA, tl,
                                               task_off, part_off, list_off, totals, counters,
                                               BatchCond{h_ref, 1}, status, cs1);
          e = end_body(cs1, e2);
        }
        if (e == cudaSuccess)
          e = launch_batched_refine_setup(sc, B, y, kept, acc1, DP, ym, yf, ract, mdone, 0, R, tl,
                                          cs0);
      }
      // (unrefined: the accepted seeds are the modes)
      if (e == cudaSuccess)
        e = launch_plan(sc, B, kPlanModes, R, DA, task_off, part_off, list_off, totals, no_cond,
                        status, cs0);
      if (e == cudaSuccess)
        e = launch_batched_step(Xs, d, DP, yf, ract, sc, B, kPlanModes, task_off, part_off,
                                totals, part, Lo.TW, status, cs0);
      if (e == cudaSuccess)
        e = launch_batched_refine_update(part, ract, sc, B, list_off, part_off, totals, ym, yf,
                                         mdone, mscore, d, DP, DA, 0.0, 1, grid_upd, cs0);
      // second prune, canonical order, labels
      if (e == cudaSuccess)
        e = launch_batched_prune_d(sc, B, mscore, ym, DP, d, r2_s, acc2, plist, max_n, cs0);
      if (e == cudaSuccess)
        e = launch_batched_canonical(sc, B, ym, mscore, acc2, d, DP, 1.0 / scale, out_modes,
                                     max_modes, modes_full, out_n_modes, cs0);
      if (e == cudaSuccess)
        e = launch_batched_label(points, pt_off, B, d, sc, modes_full, out_labels, out_margins,
                                 total, cs0);
      if (capturing) {
        cudaGraph_t gout = g;
        const cudaError_t e3 = cudaStreamEndCapture(cs0, &gout);
        if (e == cudaSuccess) e = e3;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        if (exec) cudaGraphExecDestroy(exec);
        cudaGetLastError();
        rc = FMS_ERR_CUDA;
        goto done;
      }
      const int slot = gc.next;
      if (slot < gc.used && gc.exec[slot]) cudaGraphExecDestroy(gc.exec[slot]);
      gc.key[slot] = gk;
      gc.exec[slot] = exec;
      gc.next = (gc.next + 1) % BGraphCache::kEntries;
      if (gc.used < BGraphCache::kEntries) ++gc.used;
    }
    BC(cudaGraphLaunch(exec, st));
    // the one synchronisation of the call: control blocks, status, loop counts
    BC(cudaMemcpyAsync(hsc.data(), sc, (size_t)B * sizeof(SetCtl), cudaMemcpyDeviceToHost, st));
    BC(cudaMemcpyAsync(&hstatus, status, 4, cudaMemcpyDeviceToHost, st));
    BC(cudaMemcpyAsync(hcnt, counters, 16, cudaMemcpyDeviceToHost, st));
    BC(cudaStreamSynchronize(st));
    if (hstatus & kStNonFinite) rc = FMS_ERR_NONFINITE;
    else if (hstatus & kStTimeout) rc = FMS_ERR_TIMEOUT;
    int64_t ev = 0;
    int maxMr = 0, iters = 0, conv_n = 0, kept_n = 0, seeds = 0, modes = 0;
    for (int b = 0; b < B; ++b) {
      ev += hsc[b].evals;
      maxMr = hsc[b].Mr > maxMr ? hsc[b].Mr : maxMr;
      iters = hsc[b].steps > iters ? hsc[b].steps : iters;
      conv_n += hsc[b].n_conv;
      kept_n += hsc[b].K;
      seeds += hsc[b].N;
      modes += hsc[b].Mr;
    }
    if (rc == FMS_OK && maxMr > max_modes) rc = FMS_ERR_CAPACITY;
    if (stats) {
      const int rounds = hcnt[kCtrRounds], updates = hcnt[kCtrUpdates],
                refines = hcnt[kCtrRefine];
      // kernels: pack + seed init; per round compact, kept, step, score, prune,
      // advance, seed init; per update step, update, compact; refinement setup,
      // plan and per refinement update step, update, compact; the density
      // pass (setup, plan, step, update); second prune, order, labels
      stats->iterations = iters;
      stats->rounds = rounds;
      stats->n_seeds_final = seeds;
      stats->n_converged = conv_n;
      stats->n_kept = kept_n;
      stats->n_discarded = seeds - kept_n;
      stats->n_modes = modes;
      stats->refine_iterations = refines;
      stats->kernel_launches = 2 + 7 * rounds + 3 * updates +
                               (o.skip_refine ? 0 : 2 + 3 * refines) + 4 + 3;
      stats->evals = ev;
      stats->workspace_bytes = need;
      stats->graph = 1;
    }
  }
done:
  if (owns) {
    cudaFreeAsync(ws, st);
    cudaStreamSynchronize(st);
  }
  return rc;
#undef BC
}

}  // extern "C"
