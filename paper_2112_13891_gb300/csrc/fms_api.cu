// C ABI entry points (include/fms.h) and the host-side control of one
// clustering call.  Every arithmetic step runs in the kernels of k_*.cu; the
// host only carves the workspace, launches, and reads the small control
// blocks the device writes (one synchronisation per batch of updates).
#include <math.h>
#include <string.h>

#include <vector>

#include "../../include/fms.h"
#include "fms_internal.cuh"

using namespace fms;

namespace {

constexpr int kUpdatesPerBatch = 8;   // updates issued between host checks
constexpr int kRefineMaxIter = 50;    // refinement cap (updates per mode)
constexpr int kHistCap = 65536;       // convergence histogram entries (cluster rounds)
constexpr double kRefineTolFactor = 1e-5;

struct Dev {
  int sms = 0;
};

// SM count of the current device (queried once per device)
Dev device_info() {
  constexpr int kMaxDevices = 64;
  static int sms_cache[kMaxDevices] = {0};
  Dev d;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return d;
  if (dev >= 0 && dev < kMaxDevices && sms_cache[dev] > 0) {
    d.sms = sms_cache[dev];
    return d;
  }
  if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) d.sms = 0;
  if (dev >= 0 && dev < kMaxDevices && d.sms > 0) sms_cache[dev] = d.sms;
  return d;
}

// Workspace carving.  All sizes in bytes, every region 256-byte aligned.
struct Layout {
  size_t off_Xs, off_y, off_seed_idx, off_it, off_conv, off_state, off_active, off_kept,
      off_alive, off_acc1, off_acc2, off_score, off_ym, off_mdone, off_mscore, off_modes_full,
      off_part, off_part64, off_ctl, off_mctl, off_status, off_slog, off_yf, off_ract, off_rctl,
      off_hist, off_S, off_img, off_wlast, off_grid, total;
  int DP, DA, R, grid_ctas;
  int64_t Ncap;
  Tiling tl;
  int tc_ctas;   // > 0: seed updates start on the tensor-core step (grid size)
};

constexpr int kSlogCap = 4096;

// Control region of a clustering call: IterCtl, MergeCtl, the refinement's
// IterCtl and the status word at fixed offsets, so that one device -> host
// copy into pinned memory reads all of them.
constexpr size_t kCtlMergeOff = 256, kCtlRefineOff = 512, kCtlStatusOff = 768;
constexpr size_t kCtlBlockBytes = 1024;
static_assert(sizeof(IterCtl) <= kCtlMergeOff && sizeof(MergeCtl) <= 256 &&
                  sizeof(IterCtl) <= 256,
              "control region");

// Pinned staging of the control region (one per host thread, kept for the
// life of the thread): pageable destinations would make every readback a
// staged, host-blocking copy.
unsigned char* pinned_ctl() {
  thread_local unsigned char* buf = nullptr;
  if (!buf && cudaMallocHost(&buf, kCtlBlockBytes) != cudaSuccess) buf = nullptr;
  return buf;
}

constexpr size_t kCtlRoundOff = 896;   // RoundCtl of the device-driven rounds
static_assert(kCtlRoundOff + sizeof(RoundCtl) <= kCtlBlockBytes, "control region");

// ---------------------------------------------------------------------------
// CUDA-graph form of fms_cluster.  When every round fits the cluster kernels,
// the whole call (packing, Seed Selection, the rounds with their prunes and
// seed-count decisions, refinement, labels) is one graph: a conditional WHILE
// node repeats the round body while round_advance asks for another round, and
// an IF node runs the post-round work; the host synchronises once, to read
// the control region.  A graph bakes in its pointers and scalars, so it is
// kept per (arguments, options, device) and built the second time the same
// call is seen (a one-off call takes the host-driven path at no build cost).
// ---------------------------------------------------------------------------
struct GraphKey {
  const void* points;
  const void* points_copy;
  const void* modes;
  const void* labels;
  const void* margins;
  const void* ws;
  size_t ws_bytes;
  int64_t n;
  int32_t d, max_iter, max_modes, dev;
  float h, tol;
  unsigned char opts[sizeof(fms_options)];
};

struct GraphEntry {
  GraphKey key;
  cudaGraphExec_t exec = nullptr;
  int kernels_pre = 0, kernels_round = 0, kernels_post = 0;
  bool failed = false;
};

struct GraphCache {
  static constexpr int kEntries = 4, kSeen = 8;
  GraphEntry entries[kEntries];
  int used = 0, next = 0;
  GraphKey seen[kSeen];
  int n_seen = 0, next_seen = 0;
  // builds stop when they outrun the reuse (a working set larger than the
  // cache would rebuild on every call)
  int64_t builds = 0, hits = 0;
  bool disabled = false;   // set while fms_cluster_frames runs its frames
  ~GraphCache() {
    for (int i = 0; i < used; ++i)
      if (entries[i].exec) cudaGraphExecDestroy(entries[i].exec);
  }
};

bool same_key(const GraphKey& a, const GraphKey& b) { return memcmp(&a, &b, sizeof(GraphKey)) == 0; }

GraphCache& graph_cache() {
  thread_local GraphCache c;
  return c;
}

// Private capture streams (per device and purpose), kept for the thread's life.
cudaStream_t capture_stream(int dev, int which) {
  constexpr int kMaxDevices = 64;
  thread_local cudaStream_t s[kMaxDevices][2] = {};
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  if (!s[dev][which] &&
      cudaStreamCreateWithFlags(&s[dev][which], cudaStreamNonBlocking) != cudaSuccess)
    s[dev][which] = nullptr;
  return s[dev][which];
}

// During capture on `cs`: add a conditional node after the captured work and
// return its body graph; further capture on `cs` depends on the node.
cudaError_t add_conditional(cudaStream_t cs, cudaGraphConditionalHandle h,
                            cudaGraphConditionalNodeType type, cudaGraph_t* body) {
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
  np.conditional.type = type;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, cg, deps, nullptr, nd, &np);
  if (e != cudaSuccess) return e;
  *body = np.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1,
                                             cudaStreamSetCaptureDependencies);
}

// Whether a call's seed updates start on the tensor-core step.
bool use_tensor_step(int d, int32_t precision) {
  if (precision == FMS_PRECISION_TENSOR) return d >= 8 && d <= kTcMaxDim;
  if (precision == FMS_PRECISION_AUTO) return d >= 9 && d <= kTcMaxDim;
  return false;
}

Layout make_layout(int64_t n, int d, int64_t Ncap, int sms, bool tensor) {
  Layout L{};
  L.DP = padded_dim(d);
  L.DA = step_accumulators(d);
  L.R = step_seeds_per_warp(d);
  L.tl.target_warps = (sms > 0 ? sms : 1) * step_resident_warps_per_sm(d);
  L.grid_ctas = (L.tl.target_warps + 7) / 8;
  L.tl.min_chunk = step_min_chunk(d);
  L.Ncap = Ncap;
  const int64_t TW8 = 8LL * L.tl.target_warps;
  const int64_t Gmax = (Ncap + L.R - 1) / L.R;
  size_t part_floats = (size_t)(TW8 + Gmax + 1) * L.R * L.DA;
  L.tc_ctas = tensor ? tc_grid(d) : 0;
  if (tensor) {
    // tensor-core chunking: C <= max(4, 4 grid / G + 1) chunks of s <= 2 * 128 G seeds
    const size_t tc_floats =
        ((size_t)8 * L.tc_ctas * kTcTile + (size_t)4 * Ncap + kTcTile) * L.DA;
    if (tc_floats > part_floats) part_floats = tc_floats;
  }
  const size_t part64_doubles = 1;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += align256(bytes > 0 ? bytes : 1);
    return at;
  };
  L.off_Xs = take((size_t)n * L.DP * 4);
  L.off_y = take((size_t)Ncap * L.DP * 4);
  L.off_seed_idx = take((size_t)Ncap * 4);
  L.off_it = take((size_t)Ncap * 4);
  L.off_conv = take((size_t)Ncap * 4);
  L.off_state = take((size_t)Ncap * 4);
  L.off_active = take((size_t)Ncap * 4);
  L.off_kept = take((size_t)Ncap * 4);
  L.off_alive = take((size_t)Ncap * 4);
  L.off_acc1 = take((size_t)Ncap * 4);
  L.off_acc2 = take((size_t)Ncap * 4);
  L.off_score = take((size_t)Ncap * 4);
  L.off_ym = take((size_t)Ncap * L.DP * 8);
  L.off_mdone = take((size_t)Ncap * 4);
  L.off_mscore = take((size_t)Ncap * 8);
  L.off_modes_full = take((size_t)Ncap * d * 4);
  L.off_part = take(part_floats * 4);
  L.off_part64 = take(part64_doubles * 8);
  // control blocks and the status word in one region, read back with one copy
  L.off_ctl = take(kCtlBlockBytes);
  L.off_mctl = L.off_ctl + kCtlMergeOff;
  L.off_rctl = L.off_ctl + kCtlRefineOff;
  L.off_status = L.off_ctl + kCtlStatusOff;
  L.off_slog = take((size_t)kSlogCap * 2 * 4);   // ms_step log, coarse step log
  L.off_yf = take((size_t)Ncap * L.DP * 4);
  L.off_ract = take((size_t)Ncap * 4);
  L.off_hist = take((size_t)(kHistCap + 2) * 4);
  L.off_S = take(64);
  L.off_img = take(tensor ? tc_image_bytes(n, d) : 0);
  L.off_wlast = take((size_t)Ncap * 4);   // sum w of each seed's latest cluster-round update
  L.off_grid = take(d <= 7 ? grid_scratch_bytes(d) : 0);   // grid rounds: barrier + accumulators
  L.total = o;
  return L;
}

// Grid-round launch plan (occupancy and shared-memory checks), cached per
// host thread for the last few (device, n, d, max_iter class) seen.
GridPlan cached_grid_plan(int64_t n, int d, int sms, int max_iter) {
  struct Entry {
    int dev;
    int64_t n;
    int d, sms, hist_ok;
    GridPlan p;
  };
  thread_local Entry cache[8];
  thread_local int used = 0, next = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GridPlan{};
  const int hist_ok = max_iter < kGridHist ? 1 : 0;
  for (int i = 0; i < used; ++i)
    if (cache[i].dev == dev && cache[i].n == n && cache[i].d == d && cache[i].sms == sms &&
        cache[i].hist_ok == hist_ok)
      return cache[i].p;
  Entry e{dev, n, d, sms, hist_ok, grid_round_plan(n, d, sms, max_iter)};
  cache[next] = e;
  next = (next + 1) % 8;
  if (used < 8) ++used;
  return e.p;
}

void fill_defaults(const fms_options* in, fms_options* o) {
  fms_options_default(o);
  if (!in) return;
  o->all_seeds = in->all_seeds;
  if (in->n_initial > 0) o->n_initial = in->n_initial;
  if (in->L > 0.0f) o->L = in->L;
  if (in->gamma > 0.0f) o->gamma = in->gamma;
  if (in->merge_radius > 0.0f) o->merge_radius = in->merge_radius;
  o->skip_refine = in->skip_refine;
  o->rng_seed = in->rng_seed;
  o->seed_indices = in->seed_indices;
  o->n_seed_indices = in->n_seed_indices;
  o->profile = in->profile;
  o->precision = in->precision;
  o->kernel = in->kernel;
  o->metric = in->metric;
  for (int i = 0; i < 3; ++i) o->reserved[i] = in->reserved[i];
}

int64_t seed_capacity(int64_t n, const fms_options& o) {
  if (o.seed_indices) return o.n_seed_indices;
  return n;
}

#define FMS_CUDA(call)                          \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) {                    \
      rc = FMS_ERR_CUDA;                        \
      goto done;                                \
    }                                           \
  } while (0)

// FMS_LAUNCH: a kernel launch (counted for fms_stats.kernel_launches)
#define FMS_LAUNCH(call)                        \
  do {                                          \
    ++n_launches;                               \
    FMS_CUDA(call);                             \
  } while (0)

template <typename T>
T* at(void* base, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}

}  // namespace

extern "C" {

const char* fms_strerror(fms_status s) {
  switch (s) {
    case FMS_OK: return "ok";
    case FMS_ERR_INVALID_ARG: return "invalid argument";
    case FMS_ERR_NONFINITE: return "non-finite point coordinate";
    case FMS_ERR_CAPACITY: return "more modes than max_modes";
    case FMS_ERR_TIMEOUT: return "a bounded device wait timed out";
    case FMS_ERR_CUDA: return "CUDA runtime error";
    case FMS_ERR_WORKSPACE: return "workspace too small or misaligned";
    case FMS_ERR_UNSUPPORTED: return "unsupported dimension or mode";
  }
  return "unknown status";
}

void fms_options_default(fms_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->n_initial = 128;
  o->L = 8.0f;
  o->gamma = 0.95f;
  o->merge_radius = 0.0f;
}

size_t fms_workspace_size(int64_t n, int32_t d, const fms_options* opt) {
  if (n < 1 || n > INT32_MAX || d < 1 || d > FMS_MAX_DIM) return 0;
  fms_options o;
  fill_defaults(opt, &o);
  const int64_t Ncap = seed_capacity(n, o);
  if (Ncap < 1) return 0;
  return make_layout(n, d, Ncap, device_info().sms,
                     o.kernel == FMS_KERNEL_GAUSSIAN && o.metric != FMS_METRIC_COSINE &&
                         use_tensor_step(d, o.precision))
      .total;
}

// Device-to-host copies of the results that fms_cluster_host queues on the
// stream before the call's last readback, so they complete under its one
// synchronisation (copying again is harmless if the graph hands back).
struct HostCopies {
  int count;
  void* dst[3];
  const void* src[3];
  size_t bytes[3];
  // non-null: the points are read from host memory; the packing kernel also
  // copies them here and the label kernel reads this copy
  float* points_copy;
};

static fms_status cluster_impl(const float* points, int64_t n, int32_t d, float h, float tol,
                               int32_t max_iter, const fms_options* opt_in, float* out_modes,
                               int32_t max_modes, int32_t* out_n_modes, int32_t* out_labels,
                               float* out_margins, void* workspace, size_t workspace_bytes,
                               fms_stats* stats, void* stream_, const HostCopies* hc);

fms_status fms_cluster(const float* points, int64_t n, int32_t d, float h, float tol,
                       int32_t max_iter, const fms_options* opt_in, float* out_modes,
                       int32_t max_modes, int32_t* out_n_modes, int32_t* out_labels,
                       float* out_margins, void* workspace, size_t workspace_bytes,
                       fms_stats* stats, void* stream_) {
  return cluster_impl(points, n, d, h, tol, max_iter, opt_in, out_modes, max_modes, out_n_modes,
                      out_labels, out_margins, workspace, workspace_bytes, stats, stream_,
                      nullptr);
}

static fms_status cluster_impl(const float* points, int64_t n, int32_t d, float h, float tol,
                               int32_t max_iter, const fms_options* opt_in, float* out_modes,
                               int32_t max_modes, int32_t* out_n_modes, int32_t* out_labels,
                               float* out_margins, void* workspace, size_t workspace_bytes,
                               fms_stats* stats, void* stream_, const HostCopies* hc) {
  fms_status rc = FMS_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream_);
  // points in host memory: the packing kernel also copies them to pcopy, and
  // the label kernel reads that copy
  float* pcopy = hc ? hc->points_copy : nullptr;
  const float* lpoints = pcopy ? pcopy : points;
  fms_options o;
  fill_defaults(opt_in, &o);
  if (stats) memset(stats, 0, sizeof(*stats));
  if (!points || !out_labels || !out_n_modes || n < 1 || n > INT32_MAX || d < 1 ||
      d > FMS_MAX_DIM || !(h > 0.0f) || !isfinite(h) || !(tol >= 0.0f) || !isfinite(tol) ||
      max_iter < 1 || max_modes < 0 || (max_modes > 0 && !out_modes) ||
      !(o.gamma > 0.0f && o.gamma <= 1.0f) || !(o.L > 0.0f) || !isfinite(o.merge_radius) ||
      o.merge_radius < 0.0f || (o.seed_indices && o.n_seed_indices < 1))
    return FMS_ERR_INVALID_ARG;
  for (int i = 0; i < 3; ++i)
    if (o.reserved[i] != 0) return FMS_ERR_INVALID_ARG;
  if (o.precision < FMS_PRECISION_AUTO || o.precision > FMS_PRECISION_TENSOR)
    return FMS_ERR_INVALID_ARG;
  if (o.kernel != FMS_KERNEL_GAUSSIAN && o.kernel != FMS_KERNEL_FLAT) return FMS_ERR_INVALID_ARG;
  if (o.metric != FMS_METRIC_EUCLIDEAN && o.metric != FMS_METRIC_COSINE) return FMS_ERR_INVALID_ARG;
  const bool cosine = o.metric == FMS_METRIC_COSINE;
  const int kf = o.kernel == FMS_KERNEL_FLAT ? kKernelFlat : kKernelGaussian;
  if (tol == 0.0f) tol = 1e-3f * h;
  if (o.all_seeds) o.gamma = 1.0f;

  const Dev dv = device_info();
  if (dv.sms <= 0) return FMS_ERR_CUDA;
  const int64_t Ncap = seed_capacity(n, o);
  const bool tensor = kf == kKernelGaussian && !cosine && use_tensor_step(d, o.precision);
  const Layout Lo = make_layout(n, d, Ncap, dv.sms, tensor);
  const int DP = Lo.DP, DA = Lo.DA, R = Lo.R;
  bool owns_ws = false;
  void* ws = workspace;
  std::vector<cudaEvent_t> evs;
  std::vector<int> ev_slot;
  std::vector<cudaEvent_t> round_evs;      // pairs around cluster round launches
  std::vector<cudaEvent_t> tc_evs;         // pairs around tensor-core step launches
  std::vector<int> tc_slot;
  cudaEvent_t phase_ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  double phase_acc[4] = {0, 0, 0, 0};
  IterCtl hctl{}, hrctl{};
  MergeCtl hm{};
  uint32_t hstatus = 0;
  int32_t N = 0, rounds = 0, Mfinal = 0, K_last = 0;
  int n_launches = 0;

  if (ws) {
    if (workspace_bytes < Lo.total || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0)
      return FMS_ERR_WORKSPACE;
  } else {
    if (cudaMallocAsync(&ws, Lo.total, st) != cudaSuccess) return FMS_ERR_CUDA;
    owns_ws = true;
  }
  {
    float* Xs = at<float>(ws, Lo.off_Xs);
    float* y = at<float>(ws, Lo.off_y);
    int32_t* seed_idx = at<int32_t>(ws, Lo.off_seed_idx);
    int32_t* it = at<int32_t>(ws, Lo.off_it);
    int32_t* conv = at<int32_t>(ws, Lo.off_conv);
    int32_t* state = at<int32_t>(ws, Lo.off_state);
    int32_t* active = at<int32_t>(ws, Lo.off_active);
    int32_t* kept = at<int32_t>(ws, Lo.off_kept);
    int32_t* alive = at<int32_t>(ws, Lo.off_alive);
    int32_t* acc1 = at<int32_t>(ws, Lo.off_acc1);
    int32_t* acc2 = at<int32_t>(ws, Lo.off_acc2);
    float* score = at<float>(ws, Lo.off_score);
    double* ym = at<double>(ws, Lo.off_ym);
    int32_t* mdone = at<int32_t>(ws, Lo.off_mdone);
    double* mscore = at<double>(ws, Lo.off_mscore);
    float* modes_full = at<float>(ws, Lo.off_modes_full);
    float* part = at<float>(ws, Lo.off_part);
    IterCtl* ctl = at<IterCtl>(ws, Lo.off_ctl);
    MergeCtl* mctl = at<MergeCtl>(ws, Lo.off_mctl);
    uint32_t* status = at<uint32_t>(ws, Lo.off_status);
    int32_t* slog = at<int32_t>(ws, Lo.off_slog);
    float* yf = at<float>(ws, Lo.off_yf);
    int32_t* ract = at<int32_t>(ws, Lo.off_ract);
    IterCtl* rctl = at<IterCtl>(ws, Lo.off_rctl);
    int32_t* hist = at<int32_t>(ws, Lo.off_hist);
    int32_t* S_dev = at<int32_t>(ws, Lo.off_S);
    unsigned char* img = at<unsigned char>(ws, Lo.off_img);
    float* wlast = at<float>(ws, Lo.off_wlast);
    unsigned char* hbuf = pinned_ctl();
    // read the control region (pinned staging when available), then sync
    auto readback = [&]() -> cudaError_t {
      cudaError_t e;
      if (hbuf) {
        e = cudaMemcpyAsync(hbuf, ctl, kCtlBlockBytes, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        memcpy(&hctl, hbuf, sizeof(IterCtl));
        memcpy(&hm, hbuf + kCtlMergeOff, sizeof(MergeCtl));
        memcpy(&hrctl, hbuf + kCtlRefineOff, sizeof(IterCtl));
        memcpy(&hstatus, hbuf + kCtlStatusOff, sizeof(uint32_t));
        return cudaSuccess;
      }
      e = cudaMemcpyAsync(&hctl, ctl, sizeof(IterCtl), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&hm, mctl, sizeof(MergeCtl), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&hrctl, rctl, sizeof(IterCtl), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&hstatus, status, 4, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      return e;
    };
    // the caller's host copies of the results (fms_cluster_host), queued
    // before the readback that ends the call
    auto host_copies = [&]() -> cudaError_t {
      for (int i = 0; hc && i < hc->count; ++i) {
        if (hc->bytes[i] == 0) continue;
        const cudaError_t e = cudaMemcpyAsync(hc->dst[i], hc->src[i], hc->bytes[i],
                                              cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return e;
      }
      return cudaSuccess;
    };
    int32_t* tclog = slog + kSlogCap;
    Tiling tl_iter = Lo.tl;   // the seed-update loop (tensor-core chunking when on)
    tl_iter.tc_ctas = Lo.tc_ctas;
    const int32_t init_state = tensor ? kCoarse : kRunning;
    const int qmax = d <= 7 ? round_max_clusters(d) : 0;
    // persistent grid rounds (one CTA per SM) for d <= 7 when they fit
    const GridPlan gp = d <= 7 ? cached_grid_plan(n, d, dv.sms, max_iter) : GridPlan{};
    void* grid_scratch = at<void>(ws, Lo.off_grid);

    const double scale = sqrt(1.4426950408889634 / (2.0 * (double)h * (double)h));
    // cosine metric: the packed points lie on the sphere of radius scale, and
    // every update is projected back onto it
    const float sphere_r = cosine ? (float)scale : 0.0f;
    const double sphere_rd = cosine ? scale : 0.0;
    const double tol_s = (double)tol * scale;
    const float tol2_s = (float)(tol_s * tol_s);
    const float coarse_tol2_s = (float)(100.0 * tol_s * tol_s);   // (10 tol)^2
    const double r_merge = o.merge_radius > 0.0f ? (double)o.merge_radius : (double)h;
    const double r2_s = (r_merge * scale) * (r_merge * scale);
    const bool allow_doubling = !o.all_seeds && !o.seed_indices;
    // one block per seed (many chunks) or one warp per seed: enough blocks for
    // either, at most 8 per SM
    auto update_grid = [&](int64_t m) -> int {
      int64_t g = m;
      if (g > (int64_t)dv.sms * 8) g = (int64_t)dv.sms * 8;
      return g < 1 ? 1 : (int)g;
    };
    int n_slog = 0, n_tclog = 0;

    auto step_launch = [&](const float* pos, const int32_t* list, const int32_t* s_ptr,
                           const int32_t* C_ptr, const int32_t* Lc_ptr,
                           const int32_t* p_lo = nullptr) -> cudaError_t {
      int32_t* lg = nullptr;
      if (o.profile && n_slog < kSlogCap) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
          return cudaErrorUnknown;
        cudaEventRecord(a, st);
        lg = slog + n_slog;
        cudaError_t e = launch_ms_step(Xs, n, d, DP, pos, list, s_ptr, C_ptr, Lc_ptr, part,
                                       Lo.tl.target_warps, st, lg, p_lo, kf, status);
        cudaEventRecord(b, st);
        evs.push_back(a);
        evs.push_back(b);
        ev_slot.push_back(n_slog++);
        return e;
      }
      return launch_ms_step(Xs, n, d, DP, pos, list, s_ptr, C_ptr, Lc_ptr, part,
                            Lo.tl.target_warps, st, nullptr, p_lo, kf, status);
    };
    // the coarse step for active positions [0, ctl->s_tc)
    auto tc_launch = [&]() -> cudaError_t {
      int32_t* lg = nullptr;
      cudaEvent_t a = nullptr, b = nullptr;
      if (o.profile && n_tclog < kSlogCap) {
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
          return cudaErrorUnknown;
        cudaEventRecord(a, st);
        lg = tclog + n_tclog;
      }
      cudaError_t e = launch_ms_step_tc(img, n, d, DP, DA, y, active, &ctl->s, &ctl->s_tc,
                                        &ctl->C, &ctl->Lc, part, status, st, lg);
      if (lg) {
        cudaEventRecord(b, st);
        tc_evs.push_back(a);
        tc_evs.push_back(b);
        tc_slot.push_back(n_tclog++);
      }
      return e;
    };

    // --- Seed Selection (Alg. 2): initial seed count ---
    int32_t N0;
    if (o.all_seeds) N0 = (int32_t)n;
    else if (o.seed_indices) N0 = o.n_seed_indices;
    else N0 = (int32_t)(o.n_initial < n ? o.n_initial : n);
    RoundCtl* rctl_round = at<RoundCtl>(ws, Lo.off_ctl + kCtlRoundOff);
    const int cap_seeds = gp.ok ? gp.seeds : qmax * kSeedsPerCluster;
    const int cap_modes = qmax * kModesPerCluster;
    // one grid round over the RUNNING seeds of [0, N) (N and target from rcp
    // when non-null)
    auto grid_launch = [&](const RoundCtl* rcp, int N_, int target_, cudaStream_t s_) {
      GridRoundArgs ga{};
      ga.Xs = Xs;
      ga.n = (int)n;
      ga.y = y;
      ga.it = it;
      ga.conv = conv;
      ga.state = state;
      ga.wlast = wlast;
      ga.hist = hist;
      ga.rc = rcp;
      ga.N_arg = N_;
      ga.target_arg = target_;
      ga.max_iter = max_iter;
      ga.tol2_s = tol2_s;
      ga.sphere_r = sphere_r;
      ga.evals = reinterpret_cast<unsigned long long*>(&ctl->evals);
      ga.status = status;
      return launch_ms_grid_round(gp, d, kf, ga, grid_scratch, s_);
    };
    const int keep_exhausted = o.gamma >= 1.0f ? 1 : 0;
    const double rtol_s = kRefineTolFactor * (double)h * scale;

    // --- the CUDA-graph form (see GraphKey) ---
    // resume: 0 host path from the start, 1 host rounds from the graph's state,
    // 2 host refinement and labels, 3 the graph did everything
    int resume = 0;
    const bool graph_ok = !graph_cache().disabled && !o.profile && !owns_ws && hbuf &&
                          qmax > 0 && !tensor &&
                          !o.all_seeds && !keep_exhausted && !o.seed_indices &&
                          !o.skip_refine && max_iter <= kHistCap && N0 <= cap_seeds;
    if (graph_ok) {
      GraphKey key;
      memset(&key, 0, sizeof(key));
      key.points = points;
      key.points_copy = hc ? hc->points_copy : nullptr;
      key.modes = out_modes;
      key.labels = out_labels;
      key.margins = out_margins;
      key.ws = ws;
      key.ws_bytes = workspace_bytes;
      key.n = n;
      key.d = d;
      key.max_iter = max_iter;
      key.max_modes = max_modes;
      cudaGetDevice(&key.dev);
      key.h = h;
      key.tol = tol;
      memcpy(key.opts, &o, sizeof(fms_options));
      GraphCache& gc = graph_cache();
      GraphEntry* ge = nullptr;
      for (int i = 0; i < gc.used; ++i)
        if (same_key(gc.entries[i].key, key)) ge = &gc.entries[i];
      bool seen = false;
      for (int i = 0; i < gc.n_seen; ++i)
        if (same_key(gc.seen[i], key)) seen = true;
      if (!ge && !seen) {
        gc.seen[gc.next_seen] = key;
        gc.next_seen = (gc.next_seen + 1) % GraphCache::kSeen;
        if (gc.n_seen < GraphCache::kSeen) ++gc.n_seen;
      } else if (!ge && gc.builds < 8 + 2 * gc.hits) {
        ++gc.builds;
        // build: the same sequence of launches as the host path, captured on
        // private streams, with the round's N and target read from RoundCtl
        GraphEntry* slot = &gc.entries[gc.next];
        if (gc.used == GraphCache::kEntries && slot->exec) cudaGraphExecDestroy(slot->exec);
        gc.next = (gc.next + 1) % GraphCache::kEntries;
        if (gc.used < GraphCache::kEntries) ++gc.used;
        *slot = GraphEntry();
        slot->key = key;
        cudaStream_t cs = capture_stream(key.dev, 0), cs2 = capture_stream(key.dev, 1);
        cudaGraph_t g = nullptr;
        bool capturing = false;
        cudaError_t e = (cs && cs2) ? cudaGraphCreate(&g, 0) : cudaErrorNotSupported;
        cudaGraphConditionalHandle h_loop = 0, h_post = 0;
        if (e == cudaSuccess)
          e = cudaGraphConditionalHandleCreate(&h_loop, g, 1, cudaGraphCondAssignDefault);
        if (e == cudaSuccess)
          e = cudaGraphConditionalHandleCreate(&h_post, g, 0, cudaGraphCondAssignDefault);
        if (e == cudaSuccess)
          e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal);
        capturing = e == cudaSuccess;
        // before the rounds
        if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, kCtlBlockBytes, cs);
        if (e == cudaSuccess) e = cudaMemsetAsync(hist, 0, (size_t)(kHistCap + 2) * 4, cs);
        if (e == cudaSuccess)
          e = launch_pack_points(points, n, d, DP, (float)scale, Xs, status, cs, cosine ? 1 : 0,
                                 pcopy);
        if (e == cudaSuccess)
          e = launch_seed_init(Xs, n, DP, o.rng_seed, nullptr, 0, 0, N0, seed_idx, y, it, conv,
                               state, status, cs, init_state);
        if (e == cudaSuccess) e = launch_round_begin(rctl_round, N0, o.gamma, cs);
        slot->kernels_pre = 3;
        // the rounds
        cudaGraph_t body = nullptr;
        if (e == cudaSuccess) e = add_conditional(cs, h_loop, cudaGraphCondTypeWhile, &body);
        if (e == cudaSuccess)
          e = cudaStreamBeginCaptureToGraph(cs2, body, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          cudaError_t e2 = cudaSuccess;
          if (gp.ok) {
            e2 = grid_launch(rctl_round, 0, 0, cs2);
          } else {
            e2 = launch_round_list(state, 0, active, S_dev, cs2, rctl_round);
            if (e2 == cudaSuccess)
              e2 = launch_ms_round(Xs, n, d, y, it, conv, state, active, S_dev, qmax, hist, 0,
                                   max_iter, tol2_s,
                                   reinterpret_cast<unsigned long long*>(&ctl->evals), wlast,
                                   cs2, kf, rctl_round, sphere_r);
          }
          if (e2 == cudaSuccess)
            e2 = launch_round_finish(hist, 0, max_iter, state, conv, 0, keep_exhausted, kept,
                                     mctl, ctl, n, R, Lo.tl, cs2, rctl_round, wlast, score);
          if (e2 == cudaSuccess)
            e2 = launch_greedy_merge_f(kept, &mctl->K, score, y, DP, d, (float)r2_s, alive, acc1,
                                       &mctl->M, cap_seeds, cs2, status);
          if (e2 == cudaSuccess)
            e2 = launch_round_advance(rctl_round, mctl, n, o.L, allow_doubling ? 1 : 0, o.gamma,
                                      cap_seeds, cap_modes, o.rng_seed, Xs, DP, seed_idx, y, it,
                                      conv, state, init_state, h_loop, h_post, cs2);
          cudaGraph_t gb = body;
          const cudaError_t e3 = cudaStreamEndCapture(cs2, &gb);
          e = e2 != cudaSuccess ? e2 : e3;
        }
        slot->kernels_round = gp.ok ? 4 : 5;
        // after the rounds: refinement, second prune, order, labels
        cudaGraph_t post = nullptr;
        if (e == cudaSuccess) e = add_conditional(cs, h_post, cudaGraphCondTypeIf, &post);
        if (e == cudaSuccess)
          e = cudaStreamBeginCaptureToGraph(cs2, post, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          cudaError_t e2 =
              gp.ok ? launch_ms_grid_refine(
                          gp, Xs, n, d, y, kept, acc1, &mctl->M, ym, yf, mscore, rtol_s * rtol_s,
                          kRefineMaxIter, &rctl->steps,
                          reinterpret_cast<unsigned long long*>(&rctl->evals), status,
                          grid_scratch, cs2, kf, sphere_rd)
                    : launch_ms_refine(
                          Xs, n, d, y, kept, acc1, &mctl->M, qmax, ym, yf, mscore, rtol_s * rtol_s,
                          kRefineMaxIter, &rctl->steps,
                          reinterpret_cast<unsigned long long*>(&rctl->evals), cs2, kf, sphere_rd);
          if (e2 == cudaSuccess)
            e2 = launch_greedy_merge_d(&mctl->M, mscore, ym, DP, d, r2_s, alive, acc2, &mctl->Mr,
                                       cap_modes, cs2);
          if (e2 == cudaSuccess)
            e2 = launch_canonical_order(ym, mscore, acc2, &mctl->Mr, d, DP, 1.0 / scale,
                                        out_modes, max_modes, modes_full, nullptr, cap_modes,
                                        cs2);
          if (e2 == cudaSuccess)
            e2 = launch_label(lpoints, n, d, modes_full, &mctl->Mr, 0, out_labels, out_margins,
                              cs2, cosine ? 1 : 0);
          cudaGraph_t gp = post;
          const cudaError_t e3 = cudaStreamEndCapture(cs2, &gp);
          e = e2 != cudaSuccess ? e2 : e3;
        }
        slot->kernels_post = 4;
        if (capturing) {
          cudaGraph_t gout = g;
          const cudaError_t e3 = cudaStreamEndCapture(cs, &gout);
          if (e == cudaSuccess) e = e3;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&slot->exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
          if (slot->exec) cudaGraphExecDestroy(slot->exec);
          slot->exec = nullptr;
          slot->failed = true;
          cudaGetLastError();   // clear the error the failed build left
        }
        ge = slot;
      }
      if (ge && ge->exec) {
        ++gc.hits;
        FMS_CUDA(cudaGraphLaunch(ge->exec, st));
        FMS_CUDA(host_copies());
        FMS_CUDA(readback());
        RoundCtl rcv;
        memcpy(&rcv, hbuf + kCtlRoundOff, sizeof(RoundCtl));
        rounds = rcv.rounds;
        N = rcv.N;
        K_last = rcv.K_last;
        n_launches = ge->kernels_pre + ge->kernels_round * rcv.rounds +
                     (rcv.leave == 0 ? ge->kernels_post : 0);
        if (hstatus & (kStNonFinite | kStBadArg)) goto device_error;
        if (hstatus & kStTimeout) {
          rc = FMS_ERR_TIMEOUT;
          goto done;
        }
        resume = rcv.leave == 0 ? 3 : (rcv.leave == 1 ? 1 : 2);
      }
    }
    if (resume == 0) {
      FMS_CUDA(cudaMemsetAsync(ctl, 0, kCtlBlockBytes, st));   // ctl, mctl, rctl, status, round
      FMS_CUDA(cudaMemsetAsync(hist, 0, (size_t)(kHistCap + 2) * 4, st));
    }
    if (o.profile)
      for (int i = 0; i < 5; ++i)
        if (cudaEventCreate(&phase_ev[i]) != cudaSuccess) {
          rc = FMS_ERR_CUDA;
          goto done;
        }
    auto mark = [&](int i) {
      if (o.profile) cudaEventRecord(phase_ev[i], st);
    };
    // phase accounting: [0] rounds, [1] prunes + doubling, [2] refine + order, [3] labels
    auto phase_add = [&](int slot, int a, int b) {
      if (!o.profile) return;
      float t = 0.f;
      cudaEventSynchronize(phase_ev[b]);
      if (cudaEventElapsedTime(&t, phase_ev[a], phase_ev[b]) == cudaSuccess) phase_acc[slot] += t;
    };
    if (resume == 0) {
      mark(0);
      FMS_LAUNCH(launch_pack_points(points, n, d, DP, (float)scale, Xs, status, st,
                                    cosine ? 1 : 0, pcopy));
      if (tensor) FMS_LAUNCH(launch_tc_pack(Xs, n, d, DP, img, st));
      N = N0;
      FMS_LAUNCH(launch_seed_init(Xs, n, DP, o.rng_seed, o.seed_indices, 0, 0, N, seed_idx, y,
                                  it, conv, state, status, st, init_state));
    }

    for (; resume <= 1;) {
      ++rounds;
      int target = (int)ceil((double)o.gamma * (double)N);
      if (target < 1) target = 1;
      if (target > N) target = N;
      // --- mean-shift iterations under Early Stopping (Sec. II-C) ---
      const bool use_grid = gp.ok && N <= gp.seeds;
      const bool use_clusters =
          use_grid || (qmax > 0 && N <= qmax * kSeedsPerCluster && max_iter <= kHistCap);
      if (use_clusters) {
        // persistent round (grid of one CTA per SM, or thread-block clusters
        // when the grid plan does not fit): no host round trips
        cudaEvent_t ra = nullptr, rb = nullptr;
        if (!use_grid) FMS_LAUNCH(launch_round_list(state, N, active, S_dev, st));
        if (o.profile) {
          cudaEventCreate(&ra);
          cudaEventCreate(&rb);
          cudaEventRecord(ra, st);
          round_evs.push_back(ra);
          round_evs.push_back(rb);
        }
        if (use_grid) {
          FMS_LAUNCH(grid_launch(nullptr, N, target, st));
        } else {
          int clusters = (N + 7) / 8;
          if (clusters > qmax) clusters = qmax;
          FMS_LAUNCH(launch_ms_round(Xs, n, d, y, it, conv, state, active, S_dev, clusters, hist,
                                     target, max_iter, tol2_s,
                                     reinterpret_cast<unsigned long long*>(&ctl->evals), wlast,
                                     st, kf, nullptr, sphere_r));
        }
        if (o.profile) cudaEventRecord(rb, st);
        // the prune's densities: sum w of each kept seed's last update (ms_round);
        // with gamma = 1 kept seeds need not have converged, so a density pass
        // at their positions instead
        FMS_LAUNCH(launch_round_finish(hist, target, max_iter, state, conv, N, keep_exhausted,
                                       kept, mctl, ctl, n, R, Lo.tl, st, nullptr,
                                       keep_exhausted ? nullptr : wlast, score));
        mark(1);
        if (keep_exhausted) {
          FMS_LAUNCH(step_launch(y, kept, &mctl->K, &mctl->C, &mctl->Lc));
          FMS_LAUNCH(launch_score_reduce(part, mctl, DA, score, N, st));
        }
      } else {
        FMS_LAUNCH(launch_iter_begin(ctl, state, it, conv, active, n, R, tl_iter, N, target,
                                     max_iter, st));
        for (;;) {
          for (int b = 0; b < kUpdatesPerBatch; ++b) {
            if (tensor) {
              FMS_LAUNCH(tc_launch());
              FMS_LAUNCH(step_launch(y, active, &ctl->s, &ctl->C, &ctl->Lc, &ctl->s_tc));
            } else {
              FMS_LAUNCH(step_launch(y, active, &ctl->s, &ctl->C, &ctl->Lc));
            }
            FMS_LAUNCH(launch_update(part, active, ctl, y, it, conv, state, d, DP, DA, tol2_s,
                                     max_iter, n, R, tl_iter, N, target, st, update_grid(N),
                                     coarse_tol2_s, sphere_r, wlast));
          }
          FMS_CUDA(readback());
          if (hstatus & (kStNonFinite | kStBadArg)) goto device_error;
          if (hstatus & kStTimeout) {
            rc = FMS_ERR_TIMEOUT;
            goto done;
          }
          if (hctl.done) break;
        }
        // --- prune candidates (the prune of Alg. 2) and their densities: with
        // gamma < 1 every candidate converged, and its density is sum w of its
        // last update (one step <= tol before it); kept seeds that did not
        // converge (gamma = 1) get a density pass at their positions ---
        if (keep_exhausted) {
          FMS_LAUNCH(launch_kept_list(ctl, state, conv, 1, kept, mctl, n, R, Lo.tl, st));
          mark(1);
          FMS_LAUNCH(step_launch(y, kept, &mctl->K, &mctl->C, &mctl->Lc));
          FMS_LAUNCH(launch_score_reduce(part, mctl, DA, score, N, st));
        } else {
          FMS_LAUNCH(launch_kept_list(ctl, state, conv, 0, kept, mctl, n, R, Lo.tl, st, wlast,
                                      score));
          mark(1);
        }
      }
      FMS_LAUNCH(launch_greedy_merge_f(kept, &mctl->K, score, y, DP, d, (float)r2_s, alive, acc1,
                                       &mctl->M, N, st, status));
      // --- seed-count control (Sec. II-D) ---
      FMS_LAUNCH(launch_doubling_decision(mctl, N, n, o.L, allow_doubling ? 1 : 0, st));
      mark(2);
      FMS_CUDA(readback());
      phase_add(0, 0, 1);
      phase_add(1, 1, 2);
      K_last = hm.K;
      if (hm.next_N > N) {
        mark(0);
        FMS_LAUNCH(launch_seed_init(Xs, n, DP, o.rng_seed, nullptr, N, N, hm.next_N - N, seed_idx,
                                  y, it, conv, state, status, st, init_state));
        N = hm.next_N;
        continue;
      }
      break;
    }

    std::vector<int32_t> hslog(n_slog), htclog(n_tclog);
    if (resume <= 2) {
    mark(2);
    // --- refinement and second prune ---
    if (!o.skip_refine && hm.M > 0 && qmax > 0 && hm.M <= qmax * kModesPerCluster) {
      // cluster-persistent refinement (all updates, and each mode's density, in one launch)
      const double rtol_s = kRefineTolFactor * (double)h * scale;
      const int clusters = hm.M < qmax ? hm.M : qmax;
      if (gp.ok && hm.M <= grid_refine_capacity())
        FMS_LAUNCH(launch_ms_grid_refine(gp, Xs, n, d, y, kept, acc1, &mctl->M, ym, yf, mscore,
                                         rtol_s * rtol_s, kRefineMaxIter, &rctl->steps,
                                         reinterpret_cast<unsigned long long*>(&rctl->evals),
                                         status, grid_scratch, st, kf, sphere_rd));
      else
        FMS_LAUNCH(launch_ms_refine(Xs, n, d, y, kept, acc1, &mctl->M, clusters, ym, yf, mscore,
                                    rtol_s * rtol_s, kRefineMaxIter, &rctl->steps,
                                    reinterpret_cast<unsigned long long*>(&rctl->evals), st, kf,
                                    sphere_rd));
      FMS_LAUNCH(launch_greedy_merge_d(&mctl->M, mscore, ym, DP, d, r2_s, alive, acc2, &mctl->Mr,
                                       hm.M, st));
      FMS_LAUNCH(launch_canonical_order(ym, mscore, acc2, &mctl->Mr, d, DP, 1.0 / scale,
                                        out_modes, max_modes, modes_full, nullptr, hm.M, st));
    } else if (!o.skip_refine && hm.M > 0) {
      // refinement with the ms_step kernel (many modes, or d > 7)
      const double rtol_s = kRefineTolFactor * (double)h * scale;
      FMS_LAUNCH(launch_refine_setup(y, kept, acc1, &mctl->M, DP, ym, yf, ract, mdone, rctl, 1, n,
                                     R, Lo.tl, hm.M, st));
      for (int batch = 0; batch * kUpdatesPerBatch < kRefineMaxIter; ++batch) {
        for (int i = 0; i < kUpdatesPerBatch && batch * kUpdatesPerBatch + i < kRefineMaxIter; ++i) {
          FMS_LAUNCH(step_launch(yf, ract, &rctl->s, &rctl->C, &rctl->Lc));
          FMS_LAUNCH(launch_refine_update(part, ract, rctl, ym, yf, mdone, mscore, d, DP, DA,
                                          rtol_s * rtol_s, kRefineMaxIter, n, R, Lo.tl, hm.M, st,
                                          sphere_rd));
        }
        FMS_CUDA(readback());
        if (hrctl.done) break;
      }
      // the second prune's densities: sum w (FP64 over chunks) of each mode's
      // last refinement update, recorded by refine_update (as in ms_refine)
      FMS_LAUNCH(launch_greedy_merge_d(&mctl->M, mscore, ym, DP, d, r2_s, alive, acc2, &mctl->Mr,
                                       hm.M, st));
      FMS_LAUNCH(launch_canonical_order(ym, mscore, acc2, &mctl->Mr, d, DP, 1.0 / scale,
                                        out_modes, max_modes, modes_full, nullptr, hm.M, st));
    } else {
      FMS_LAUNCH(launch_unrefined_modes(y, kept, acc1, score, mctl, DP, ym, mscore, hm.M, st));
      FMS_CUDA(cudaMemcpyAsync(&mctl->Mr, &mctl->M, 4, cudaMemcpyDeviceToDevice, st));
      FMS_LAUNCH(launch_canonical_order(ym, mscore, nullptr, &mctl->Mr, d, DP, 1.0 / scale,
                                      out_modes, max_modes, modes_full, nullptr, hm.M, st));
    }
    // --- labels (the labelling of Alg. 2) ---
    mark(3);
    FMS_LAUNCH(launch_label(lpoints, n, d, modes_full, &mctl->Mr, 0, out_labels, out_margins, st,
                            cosine ? 1 : 0));
    mark(4);
    hslog.assign(n_slog, 0);
    htclog.assign(n_tclog, 0);
    if (n_slog > 0)
      FMS_CUDA(cudaMemcpyAsync(hslog.data(), slog, (size_t)n_slog * 4, cudaMemcpyDeviceToHost, st));
    if (n_tclog > 0)
      FMS_CUDA(cudaMemcpyAsync(htclog.data(), tclog, (size_t)n_tclog * 4, cudaMemcpyDeviceToHost,
                               st));
    FMS_CUDA(host_copies());
    FMS_CUDA(readback());
    }
    Mfinal = hm.Mr;
    *out_n_modes = Mfinal;
    if (hstatus & kStNonFinite) goto device_error;
    if (hstatus & kStBadArg) goto device_error;
    if (hstatus & kStTimeout) {
      rc = FMS_ERR_TIMEOUT;
      goto done;
    }
    if (Mfinal > max_modes) rc = FMS_ERR_CAPACITY;
    if (stats) {
      stats->iterations = hctl.steps;
      stats->rounds = rounds;
      stats->n_seeds_final = N;
      stats->n_converged = hctl.n_converged;
      stats->n_kept = K_last;
      stats->n_discarded = N - K_last;
      stats->n_modes = Mfinal;
      stats->refine_iterations = hrctl.steps;
      stats->t_star_last = hm.t_star;
      stats->kernel_launches = n_launches;
      stats->evals = hctl.evals;
      stats->score_evals = hm.evals + hrctl.evals;
      stats->workspace_bytes = Lo.total;
      stats->graph = resume != 0 ? 1 : 0;
      if (o.profile) {
        phase_add(2, 2, 3);
        phase_add(3, 3, 4);
        for (int i = 0; i < 4; ++i) stats->phase_ms[i] = phase_acc[i];
        double rms = 0.0;
        for (size_t i = 0; i + 1 < round_evs.size(); i += 2) {
          float t = 0.f;
          if (cudaEventElapsedTime(&t, round_evs[i], round_evs[i + 1]) == cudaSuccess) rms += t;
        }
        stats->round_kernel_ms = rms;
        stats->round_launches = (int32_t)(round_evs.size() / 2);
        stats->round_evals = hctl.evals;
        double ms = 0.0;
        int launches = 0;
        int64_t ev = 0;
        for (size_t i = 0; i < ev_slot.size(); ++i) {
          const int s_i = hslog[ev_slot[i]];
          if (s_i <= 0) continue;
          float t = 0.0f;
          cudaEventElapsedTime(&t, evs[2 * i], evs[2 * i + 1]);
          ms += t;
          ++launches;
          ev += (int64_t)s_i * n;
        }
        stats->step_kernel_ms = ms;
        stats->step_launches = launches;
        stats->step_evals = ev;
        double tms = 0.0;
        int tl_n = 0;
        int64_t tev = 0;
        for (size_t i = 0; i < tc_slot.size(); ++i) {
          const int s_i = htclog[tc_slot[i]];
          if (s_i <= 0) continue;
          float t = 0.0f;
          cudaEventElapsedTime(&t, tc_evs[2 * i], tc_evs[2 * i + 1]);
          tms += t;
          ++tl_n;
          tev += (int64_t)s_i * n;
        }
        stats->coarse_kernel_ms = tms;
        stats->coarse_launches = tl_n;
        stats->coarse_evals = tev;
      }
    }
    goto done;
  }
device_error:
  if (hstatus & kStNonFinite) rc = FMS_ERR_NONFINITE;
  else rc = FMS_ERR_INVALID_ARG;
done:
  for (cudaEvent_t e : evs) cudaEventDestroy(e);
  for (cudaEvent_t e : round_evs) cudaEventDestroy(e);
  for (cudaEvent_t e : tc_evs) cudaEventDestroy(e);
  for (cudaEvent_t e : phase_ev)
    if (e) cudaEventDestroy(e);
  if (owns_ws) {
    cudaFreeAsync(ws, st);
    if (rc == FMS_OK || rc == FMS_ERR_CAPACITY) {
      if (cudaStreamSynchronize(st) != cudaSuccess) rc = FMS_ERR_CUDA;
    }
  }
  return rc;
}

// fms_cluster_host: the clustering workspace, then the device copies of the
// points, labels, margins and modes (256-byte aligned regions).
struct HostLayout {
  size_t cluster, off_points, off_labels, off_margins, off_modes, total;
};

static HostLayout host_layout(int64_t n, int32_t d, int32_t max_modes, const fms_options* opt) {
  HostLayout L{};
  L.cluster = fms_workspace_size(n, d, opt);
  if (L.cluster == 0) return L;
  size_t o = align256(L.cluster);
  L.off_points = o;
  o += align256((size_t)n * d * 4);
  L.off_labels = o;
  o += align256((size_t)n * 4);
  L.off_margins = o;
  o += align256((size_t)n * 4);
  L.off_modes = o;
  o += align256((size_t)(max_modes > 0 ? max_modes : 1) * d * 4);
  L.total = o;
  return L;
}

size_t fms_cluster_host_workspace_size(int64_t n, int32_t d, int32_t max_modes,
                                       const fms_options* opt) {
  if (max_modes < 0) return 0;
  const HostLayout L = host_layout(n, d, max_modes, opt);
  return L.cluster == 0 ? 0 : L.total;
}

fms_status fms_cluster_host(const float* points, int64_t n, int32_t d, float h, float tol,
                            int32_t max_iter, const fms_options* opt, float* out_modes,
                            int32_t max_modes, int32_t* out_n_modes, int32_t* out_labels,
                            float* out_margins, void* workspace, size_t workspace_bytes,
                            fms_stats* stats, void* stream_) {
  if (stats) memset(stats, 0, sizeof(*stats));
  if (!points || !out_labels || !out_n_modes || n < 1 || n > INT32_MAX || d < 1 ||
      d > FMS_MAX_DIM || max_modes < 0 || (max_modes > 0 && !out_modes))
    return FMS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream_);
  const HostLayout L = host_layout(n, d, max_modes, opt);
  if (L.cluster == 0) return FMS_ERR_INVALID_ARG;
  void* ws = workspace;
  bool owns = false;
  if (ws) {
    if (workspace_bytes < L.total || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0)
      return FMS_ERR_WORKSPACE;
  } else {
    if (cudaMallocAsync(&ws, L.total, st) != cudaSuccess) return FMS_ERR_CUDA;
    owns = true;
  }
  // Page-locked host buffers are addressable by the kernels (over the CPU-GPU
  // link): the packing and label kernels then read the points and write the
  // labels and margins there directly instead of through staging copies.
  auto mapped = [](const void* p) -> void* {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
  };
  const float* mpoints = static_cast<const float*>(mapped(points));
  int32_t* mlabels = static_cast<int32_t*>(mapped(out_labels));
  float* mmargins = out_margins ? static_cast<float*>(mapped(out_margins)) : nullptr;
  float* dpoints = at<float>(ws, L.off_points);
  int32_t* dlabels = mlabels ? mlabels : at<int32_t>(ws, L.off_labels);
  float* dmargins = out_margins ? (mmargins ? mmargins : at<float>(ws, L.off_margins)) : nullptr;
  float* dmodes = at<float>(ws, L.off_modes);
  fms_status rc = FMS_OK;
  if (!mpoints && cudaMemcpyAsync(dpoints, points, (size_t)n * d * 4, cudaMemcpyHostToDevice,
                                  st) != cudaSuccess) {
    rc = FMS_ERR_CUDA;
  } else {
    HostCopies hc{};
    hc.points_copy = mpoints ? dpoints : nullptr;
    if (!mlabels) {
      hc.dst[hc.count] = out_labels;
      hc.src[hc.count] = dlabels;
      hc.bytes[hc.count++] = (size_t)n * 4;
    }
    if (out_margins && !mmargins) {
      hc.dst[hc.count] = out_margins;
      hc.src[hc.count] = dmargins;
      hc.bytes[hc.count++] = (size_t)n * 4;
    }
    if (max_modes > 0) {
      hc.dst[hc.count] = out_modes;
      hc.src[hc.count] = dmodes;
      hc.bytes[hc.count++] = (size_t)max_modes * d * 4;
    }
    rc = cluster_impl(mpoints ? mpoints : dpoints, n, d, h, tol, max_iter, opt,
                      max_modes > 0 ? dmodes : nullptr,
                      max_modes, out_n_modes, dlabels, dmargins, ws, L.cluster, stats, stream_,
                      &hc);
  }
  if (owns) {
    cudaFreeAsync(ws, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && (rc == FMS_OK || rc == FMS_ERR_CAPACITY))
      rc = FMS_ERR_CUDA;
  }
  return rc;
}

extern "C++" {
namespace fms {
// k_step_tc.cu: the bounded-wait self-test kernel
cudaError_t launch_wait_selftest(uint32_t* status, long spins, int variant, cudaStream_t st);
}  // namespace fms
}

fms_status fms_selftest_bounded_wait(int32_t variant, int64_t spins, uint32_t* out_status,
                                     void* stream_) {
  if (variant < 0 || variant > 2 || spins < 1 || !out_status) return FMS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream_);
  uint32_t* dstatus = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&dstatus), 4, st) != cudaSuccess)
    return FMS_ERR_CUDA;
  fms_status rc = FMS_OK;
  if (cudaMemsetAsync(dstatus, 0, 4, st) != cudaSuccess ||
      fms::launch_wait_selftest(dstatus, (long)spins, variant, st) != cudaSuccess ||
      cudaMemcpyAsync(out_status, dstatus, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    rc = FMS_ERR_CUDA;
  cudaFreeAsync(dstatus, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) rc = FMS_ERR_CUDA;
  if (rc == FMS_OK && (*out_status & kStTimeout)) rc = FMS_ERR_TIMEOUT;
  return rc;
}

fms_status fms_cluster_frames(const float* frames, int32_t F, int64_t n, int32_t d, float h,
                              float tol, int32_t max_iter, const fms_options* opt_in, float H,
                              float* out_modes, int32_t max_modes, int32_t* out_n_modes,
                              int32_t* out_labels, float* out_margins, int32_t* out_seed_counts,
                              void* workspace, size_t workspace_bytes, fms_stats* stats,
                              void* stream_) {
  fms_options o;
  fill_defaults(opt_in, &o);
  if (stats) memset(stats, 0, sizeof(*stats));
  if (!frames || F < 1 || !out_n_modes || !out_labels || n < 1 || n > INT32_MAX || d < 1 ||
      d > FMS_MAX_DIM || o.all_seeds || o.seed_indices || max_modes < 0 ||
      (max_modes > 0 && !out_modes))
    return FMS_ERR_INVALID_ARG;
  if (!(H > 0.0f)) H = 32.0f;
  cudaStream_t st = static_cast<cudaStream_t>(stream_);
  const size_t need = fms_workspace_size(n, d, &o);
  if (need == 0) return FMS_ERR_INVALID_ARG;
  void* ws = workspace;
  bool owns = false;
  if (ws) {
    if (workspace_bytes < need) return FMS_ERR_WORKSPACE;
  } else {
    if (cudaMallocAsync(&ws, need, st) != cudaSuccess) return FMS_ERR_CUDA;
    owns = true;
    workspace_bytes = need;
  }
  fms_status rc = FMS_OK;
  int64_t N = o.n_initial;
  // frames have their own pointers, so the per-call graph cache would only
  // churn: the frames run on the host-driven path
  struct NoGraph {
    bool prev;
    NoGraph() : prev(graph_cache().disabled) { graph_cache().disabled = true; }
    ~NoGraph() { graph_cache().disabled = prev; }
  } no_graph;
  for (int32_t f = 0; f < F; ++f) {
    fms_options of = o;
    of.n_initial = (int32_t)(N < n ? N : n);
    if (out_seed_counts) out_seed_counts[f] = of.n_initial;
    fms_stats sf;
    const fms_status r = fms_cluster(
        frames + (size_t)f * (size_t)n * d, n, d, h, tol, max_iter, &of,
        out_modes ? out_modes + (size_t)f * max_modes * d : nullptr, max_modes, out_n_modes + f,
        out_labels + (size_t)f * n, out_margins ? out_margins + (size_t)f * n : nullptr, ws,
        workspace_bytes, &sf, stream_);
    if (r != FMS_OK && r != FMS_ERR_CAPACITY) {
      rc = r;
      break;
    }
    if (r == FMS_ERR_CAPACITY) rc = FMS_ERR_CAPACITY;
    if (stats) {
      const fms_stats acc = *stats;
      *stats = sf;
      stats->iterations += acc.iterations;
      stats->rounds += acc.rounds;
      stats->kernel_launches += acc.kernel_launches;
      stats->evals += acc.evals;
      stats->score_evals += acc.score_evals;
    }
    // Sec. II-D: N > H*M -> the next frame starts with N - M seeds
    const int64_t Nf = sf.n_seeds_final, M = *(out_n_modes + f);
    N = (double)Nf > (double)H * (double)M ? Nf - M : Nf;
    if (N < 1) N = 1;
  }
  if (owns) {
    cudaFreeAsync(ws, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == FMS_OK) rc = FMS_ERR_CUDA;
  }
  return rc;
}

fms_status fms_select_seeds(int64_t n, uint64_t rng_seed, int64_t start, int64_t count,
                            int32_t* out_indices, void* stream) {
  if (n < 1 || n > INT32_MAX || start < 0 || count < 0 || start + count > n ||
      (count > 0 && !out_indices))
    return FMS_ERR_INVALID_ARG;
  if (launch_select_seeds(n, rng_seed, start, count, out_indices,
                          static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return FMS_ERR_CUDA;
  return FMS_OK;
}


size_t fms_step_workspace_size(int64_t n, int32_t d, int64_t m) {
  if (n < 1 || n > INT32_MAX || d < 1 || d > FMS_MAX_DIM || m < 1 || m > INT32_MAX) return 0;
  return step_layout(n, d, m, device_info().sms).total;
}

fms_status fms_mean_shift_step(const float* points, int64_t n, int32_t d, float h,
                               const float* seeds, int64_t m, float* out_seeds, float* out_wsum,
                               void* workspace, size_t workspace_bytes, void* stream_) {
  if (!points || !seeds || !out_seeds || n < 1 || n > INT32_MAX || d < 1 || d > FMS_MAX_DIM ||
      m < 1 || m > INT32_MAX || !(h > 0.0f) || !isfinite(h))
    return FMS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream_);
  const Dev dv = device_info();
  if (dv.sms <= 0) return FMS_ERR_CUDA;
  const StepLayout L = step_layout(n, d, m, dv.sms);
  fms_status rc = FMS_OK;
  bool owns = false;
  void* ws = workspace;
  uint32_t hstatus = 0;
  if (ws) {
    if (workspace_bytes < L.total || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0)
      return FMS_ERR_WORKSPACE;
  } else {
    if (cudaMallocAsync(&ws, L.total, st) != cudaSuccess) return FMS_ERR_CUDA;
    owns = true;
  }
  {
    const double scale = sqrt(1.4426950408889634 / (2.0 * (double)h * (double)h));
    float* Xs = at<float>(ws, L.off_Xs);
    float* Ys = at<float>(ws, L.off_Ys);
    int32_t* active = at<int32_t>(ws, L.off_active);
    float* part = at<float>(ws, L.off_part);
    IterCtl* ctl = at<IterCtl>(ws, L.off_ctl);
    uint32_t* status = at<uint32_t>(ws, L.off_status);
    FMS_CUDA(cudaMemsetAsync(status, 0, 64, st));
    FMS_CUDA(launch_pack_points(points, n, d, L.DP, (float)scale, Xs, status, st));
    FMS_CUDA(launch_pack_points(seeds, m, d, L.DP, (float)scale, Ys, status, st));
    FMS_CUDA(launch_step_setup(active, (int32_t)m, ctl, L.C, L.Lc, st));
    FMS_CUDA(launch_ms_step(Xs, n, d, L.DP, Ys, active, &ctl->s, &ctl->C, &ctl->Lc, part,
                            L.grid_ctas * 8, st, nullptr, nullptr, kKernelGaussian, status));
    FMS_CUDA(launch_step_finish(part, ctl, seeds, d, L.DA, 1.0 / scale, out_seeds, out_wsum,
                                (int)m, st));
    if (owns) {
      FMS_CUDA(cudaMemcpyAsync(&hstatus, status, 4, cudaMemcpyDeviceToHost, st));
      FMS_CUDA(cudaStreamSynchronize(st));
      if (hstatus & kStNonFinite) rc = FMS_ERR_NONFINITE;
      else if (hstatus & kStTimeout) rc = FMS_ERR_TIMEOUT;
    }
  }
done:
  if (owns) cudaFreeAsync(ws, st);
  return rc;
}

namespace {
struct CoarseLayout {
  size_t off_Xs, off_img, off_Ys, off_active, off_part, off_ctl, off_status, total;
  int DP, DA, C, Lc, grid;
};

CoarseLayout coarse_layout(int64_t n, int d, int64_t m) {
  CoarseLayout L{};
  L.DP = padded_dim(d);
  L.DA = L.DP + 4;
  L.grid = tc_grid(d);
  tc_choose_chunks(n, (int32_t)m, L.grid, &L.C, &L.Lc);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at_ = o;
    o += align256(bytes > 0 ? bytes : 1);
    return at_;
  };
  L.off_Xs = take((size_t)n * L.DP * 4);
  L.off_img = take(tc_image_bytes(n, d));
  L.off_Ys = take((size_t)m * L.DP * 4);
  L.off_active = take((size_t)m * 4);
  L.off_part = take((size_t)L.C * (size_t)m * L.DA * 4);
  L.off_ctl = take(sizeof(IterCtl));
  L.off_status = take(64);
  L.total = o;
  return L;
}
}  // namespace

size_t fms_coarse_step_workspace_size(int64_t n, int32_t d, int64_t m) {
  if (n < 1 || n > INT32_MAX || d < 1 || d > kTcMaxDim || m < 1 || m > INT32_MAX) return 0;
  return coarse_layout(n, d, m).total;
}

fms_status fms_mean_shift_step_coarse(const float* points, int64_t n, int32_t d, float h,
                                      const float* seeds, int64_t m, float* out_seeds,
                                      float* out_wsum, void* workspace, size_t workspace_bytes,
                                      void* stream_) {
  if (!points || !seeds || !out_seeds || n < 1 || n > INT32_MAX || d < 1 || d > FMS_MAX_DIM ||
      m < 1 || m > INT32_MAX || !(h > 0.0f) || !isfinite(h))
    return FMS_ERR_INVALID_ARG;
  if (d > kTcMaxDim) return FMS_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream_);
  if (device_info().sms <= 0) return FMS_ERR_CUDA;
  const CoarseLayout L = coarse_layout(n, d, m);
  fms_status rc = FMS_OK;
  bool owns = false;
  void* ws = workspace;
  uint32_t hstatus = 0;
  if (ws) {
    if (workspace_bytes < L.total || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0)
      return FMS_ERR_WORKSPACE;
  } else {
    if (cudaMallocAsync(&ws, L.total, st) != cudaSuccess) return FMS_ERR_CUDA;
    owns = true;
  }
  {
    const double scale = sqrt(1.4426950408889634 / (2.0 * (double)h * (double)h));
    float* Xs = at<float>(ws, L.off_Xs);
    unsigned char* img = at<unsigned char>(ws, L.off_img);
    float* Ys = at<float>(ws, L.off_Ys);
    int32_t* active = at<int32_t>(ws, L.off_active);
    float* part = at<float>(ws, L.off_part);
    IterCtl* ctl = at<IterCtl>(ws, L.off_ctl);
    uint32_t* status = at<uint32_t>(ws, L.off_status);
    FMS_CUDA(cudaMemsetAsync(status, 0, 64, st));
    FMS_CUDA(launch_pack_points(points, n, d, L.DP, (float)scale, Xs, status, st));
    FMS_CUDA(launch_tc_pack(Xs, n, d, L.DP, img, st));
    FMS_CUDA(launch_pack_points(seeds, m, d, L.DP, (float)scale, Ys, status, st));
    FMS_CUDA(launch_step_setup(active, (int32_t)m, ctl, L.C, L.Lc, st));
    FMS_CUDA(launch_ms_step_tc(img, n, d, L.DP, L.DA, Ys, active, &ctl->s, &ctl->s, &ctl->C,
                               &ctl->Lc, part, status, st));
    FMS_CUDA(launch_step_finish(part, ctl, seeds, d, L.DA, 1.0 / scale, out_seeds, out_wsum,
                                (int)m, st));
    if (owns) {
      FMS_CUDA(cudaMemcpyAsync(&hstatus, status, 4, cudaMemcpyDeviceToHost, st));
      FMS_CUDA(cudaStreamSynchronize(st));
      if (hstatus & kStNonFinite) rc = FMS_ERR_NONFINITE;
      else if (hstatus & kStTimeout) rc = FMS_ERR_TIMEOUT;
      else if (hstatus & kStBadArg) rc = FMS_ERR_INVALID_ARG;
    }
  }
done:
  if (owns) cudaFreeAsync(ws, st);
  return rc;
}

fms_status fms_label_points(const float* points, int64_t n, int32_t d, const float* modes,
                            int32_t M, int32_t* labels, float* margins, void* stream) {
  if (!points || !modes || !labels || n < 1 || d < 1 || d > FMS_MAX_DIM || M < 1)
    return FMS_ERR_INVALID_ARG;
  if (launch_label(points, n, d, modes, nullptr, M, labels, margins,
                   static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return FMS_ERR_CUDA;
  return FMS_OK;
}

}  // extern "C"
