// ms_step: partial sums of one Gaussian mean-shift update for the active seeds.
//
// For every active seed y and every point x_j (Sec. II-B, Alg. 2 line 6: all
// points, no window search) the update needs
//   W = sum_j w_j,   S = sum_j w_j (x_j - y),   w_j = exp(-||y - x_j||^2 / (2h^2)),
// after which m(y) = y + S / W (Eq. 6 with the Gaussian profile).  Points are
// stored pre-scaled by s = sqrt(log2(e)/(2h^2)), so w_j = exp2(-||ys - xs_j||^2)
// is one MUFU.EX2 of a sum of squared exact differences.
//
// Work decomposition: a warp task is (seed group of R seeds, chunk of Lc
// points).  Tasks are spread over a fixed grid of persistent warps.  The R
// seeds of a task live in registers; the 32 lanes walk the chunk's points with
// stride 32, so every point load feeds R evaluations.  At the end of the chunk
// the R x DA per-lane accumulators (R * DA = 32) are reduced across the warp by
// a butterfly reduce-scatter that leaves accumulator v in lane v, and the warp
// writes its 32 partial sums with one coalesced store.  The summation order of
// a seed does not depend on which slot of the task it occupies, so a seed's
// trajectory is the same whatever other seeds are active.
#include "fms_internal.cuh"

namespace fms {

// Butterfly reduce-scatter over a warp: on return lane l holds the warp-wide
// sum of v[l].  31 shuffles for 32 values; the pairing tree is the same for
// every value index.
__device__ __forceinline__ float reduce_scatter32(float (&v)[32], int lane) {
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

// A point as loaded by one lane: DP = 4 -> one float4, DP = 8 -> two.
template <int DP>
struct Pt;
template <>
struct Pt<4> {
  float4 a;
};
template <>
struct Pt<8> {
  float4 a, b;
};

// Load point j, or a point so far away that its weight is exactly 0 (and
// w * (x - y) = 0) when j is past the end of the chunk.  Coordinates of 1e18
// give squared distances of ~1e36 (finite), so exp2 underflows to 0.
template <int DP>
__device__ __forceinline__ Pt<DP> load_pt(const float* __restrict__ Xs, int j, int j1) {
  Pt<DP> p;
  const float4 far = make_float4(1e18f, 1e18f, 1e18f, 1e18f);
  if constexpr (DP == 4) {
    p.a = j < j1 ? __ldg(reinterpret_cast<const float4*>(Xs) + j) : far;
  } else {
    p.a = j < j1 ? __ldg(reinterpret_cast<const float4*>(Xs) + 2 * j) : far;
    p.b = j < j1 ? __ldg(reinterpret_cast<const float4*>(Xs) + 2 * j + 1) : far;
  }
  return p;
}

template <int D, int DP>
__device__ __forceinline__ void coords(const Pt<DP>& p, float (&x)[D]) {
  const float t[8] = {p.a.x, p.a.y, p.a.z, p.a.w,
                      DP == 8 ? reinterpret_cast<const Pt<8>&>(p).b.x : 0.f,
                      DP == 8 ? reinterpret_cast<const Pt<8>&>(p).b.y : 0.f,
                      DP == 8 ? reinterpret_cast<const Pt<8>&>(p).b.z : 0.f,
                      DP == 8 ? reinterpret_cast<const Pt<8>&>(p).b.w : 0.f};
#pragma unroll
  for (int k = 0; k < D; ++k) x[k] = t[k];
}

// R seeds in registers against one point: exact differences, one exp2 each.
template <int D, int R, int DA>
__device__ __forceinline__ void eval_point(const float (&x)[D], const float (&ys)[R][D],
                                           float (&acc)[R][DA]) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    float dx[D];
#pragma unroll
    for (int k = 0; k < D; ++k) dx[k] = x[k] - ys[r][k];
    float t = -dx[0] * dx[0];
#pragma unroll
    for (int k = 1; k < D; ++k) t = fmaf(-dx[k], dx[k], t);
    const float w = ex2_ftz(t);
    acc[r][0] += w;
#pragma unroll
    for (int k = 0; k < D; ++k) acc[r][1 + k] = fmaf(w, dx[k], acc[r][1 + k]);
  }
}

// Low-dimensional path: D <= 7, DA accumulators per seed (sum w, d sums, pad),
// R = 32 / DA seeds per warp task.  Each lane keeps a ring of four points in
// flight (the loads for points i+4..i+7 are issued before points i..i+3 are
// evaluated), which hides the L1/L2 latency of the point stream.
template <int D, int DP, int DA>
__global__ void __launch_bounds__(256) ms_step_lowd(const float* __restrict__ Xs, int64_t n,
                                                    const float* __restrict__ y,
                                                    const int32_t* __restrict__ active,
                                                    const int32_t* __restrict__ s_ptr,
                                                    const int32_t* __restrict__ C_ptr,
                                                    const int32_t* __restrict__ Lc_ptr,
                                                    float* __restrict__ part,
                                                    int32_t* __restrict__ s_log) {
  constexpr int R = 32 / DA;
  static_assert(R * DA == 32 && D + 1 <= DA, "accumulator layout");
  const int s = *s_ptr;
  if (s_log && blockIdx.x == 0 && threadIdx.x == 0) *s_log = s;
  if (s <= 0) return;
  const int C = *C_ptr;
  const int Lc = *Lc_ptr;
  const int G = (s + R - 1) / R;
  const int64_t T = (int64_t)G * C;
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t task = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); task < T;
       task += nw) {
    const int g = (int)(task % G);
    const int c = (int)(task / G);
    float ys[R][D];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      int p = g * R + r;
      p = p < s ? p : s - 1;
      const int64_t slot = __ldg(active + p);
#pragma unroll
      for (int k = 0; k < D; ++k) ys[r][k] = __ldg(y + slot * DP + k);
    }
    float acc[R][DA];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int k = 0; k < DA; ++k) acc[r][k] = 0.0f;

    const int j0 = c * Lc;
    const int j1 = (int)(j0 + Lc < n ? j0 + Lc : n);
    int j = j0 + lane;
    Pt<DP> b0 = load_pt<DP>(Xs, j, j1), b1 = load_pt<DP>(Xs, j + 32, j1);
    Pt<DP> b2 = load_pt<DP>(Xs, j + 64, j1), b3 = load_pt<DP>(Xs, j + 96, j1);
    for (; j < j1; j += 128) {
      const Pt<DP> p0 = b0, p1 = b1, p2 = b2, p3 = b3;
      b0 = load_pt<DP>(Xs, j + 128, j1);
      b1 = load_pt<DP>(Xs, j + 160, j1);
      b2 = load_pt<DP>(Xs, j + 192, j1);
      b3 = load_pt<DP>(Xs, j + 224, j1);
      float x[D];
      coords<D, DP>(p0, x);
      eval_point<D, R, DA>(x, ys, acc);
      coords<D, DP>(p1, x);
      eval_point<D, R, DA>(x, ys, acc);
      coords<D, DP>(p2, x);
      eval_point<D, R, DA>(x, ys, acc);
      coords<D, DP>(p3, x);
      eval_point<D, R, DA>(x, ys, acc);
    }
    float v[32];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int k = 0; k < DA; ++k) v[r * DA + k] = acc[r][k];
    const float tot = reduce_scatter32(v, lane);
    const int p = g * R + lane / DA;
    if (p < s) part[((int64_t)c * s + p) * DA + (lane % DA)] = tot;
  }
}

// Generic FP32 path for 8 <= d <= 64: lanes own seeds (RG per lane), points
// are read with warp-uniform (broadcast) loads, so no cross-lane reduction is
// needed.  DPAD is the padded dimension (pad coordinates are zero on both
// sides and contribute nothing); DA = DPAD + 4 accumulators per seed in part.
template <int DPAD, int RG>
__global__ void __launch_bounds__(128) ms_step_wide(const float* __restrict__ Xs, int64_t n,
                                                    int DP, const float* __restrict__ y,
                                                    const int32_t* __restrict__ active,
                                                    const int32_t* __restrict__ s_ptr,
                                                    const int32_t* __restrict__ C_ptr,
                                                    const int32_t* __restrict__ Lc_ptr,
                                                    float* __restrict__ part,
                                                    int32_t* __restrict__ s_log) {
  constexpr int DA = DPAD + 4;
  constexpr int SPW = 32 * RG;  // seeds per warp task
  const int s = *s_ptr;
  if (s_log && blockIdx.x == 0 && threadIdx.x == 0) *s_log = s;
  if (s <= 0) return;
  const int C = *C_ptr;
  const int Lc = *Lc_ptr;
  const int G = (s + SPW - 1) / SPW;
  const int64_t T = (int64_t)G * C;
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t task = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); task < T;
       task += nw) {
    const int g = (int)(task % G);
    const int c = (int)(task / G);
    float ys[RG][DPAD];
    float acc[RG][DPAD + 1];
#pragma unroll
    for (int r = 0; r < RG; ++r) {
      int p = g * SPW + r * 32 + lane;
      p = p < s ? p : s - 1;
      const int64_t slot = __ldg(active + p);
#pragma unroll
      for (int k = 0; k < DPAD; ++k) ys[r][k] = k < DP ? __ldg(y + slot * DP + k) : 0.0f;
#pragma unroll
      for (int k = 0; k <= DPAD; ++k) acc[r][k] = 0.0f;
    }
    const int64_t j0 = (int64_t)c * Lc;
    const int64_t j1 = j0 + Lc < n ? j0 + Lc : n;
    for (int64_t j = j0; j < j1; ++j) {
      float x[DPAD];
      const float4* xp = reinterpret_cast<const float4*>(Xs + j * DP);
#pragma unroll
      for (int q = 0; q < DPAD / 4; ++q) {
        float4 v = (4 * q < DP) ? __ldg(xp + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        x[4 * q] = v.x;
        x[4 * q + 1] = v.y;
        x[4 * q + 2] = v.z;
        x[4 * q + 3] = v.w;
      }
#pragma unroll
      for (int r = 0; r < RG; ++r) {
        float dx[DPAD];
#pragma unroll
        for (int k = 0; k < DPAD; ++k) dx[k] = x[k] - ys[r][k];
        float t = -dx[0] * dx[0];
#pragma unroll
        for (int k = 1; k < DPAD; ++k) t = fmaf(-dx[k], dx[k], t);
        const float w = ex2_ftz(t);
        acc[r][0] += w;
#pragma unroll
        for (int k = 0; k < DPAD; ++k) acc[r][1 + k] = fmaf(w, dx[k], acc[r][1 + k]);
      }
    }
#pragma unroll
    for (int r = 0; r < RG; ++r) {
      const int p = g * SPW + r * 32 + lane;
      if (p < s) {
        float* o = part + ((int64_t)c * s + p) * DA;
#pragma unroll
        for (int k = 0; k <= DPAD; ++k) o[k] = acc[r][k];
      }
    }
  }
}

int step_seeds_per_warp(int d) {
  if (d <= 1) return 16;
  if (d <= 3) return 8;
  if (d <= 7) return 4;
  if (d <= 8) return 32 * 4;
  if (d <= 16) return 32 * 2;
  return 32;
}

int step_accumulators(int d) {
  if (d <= 1) return 2;
  if (d <= 3) return 4;
  if (d <= 7) return 8;
  if (d <= 8) return 12;
  if (d <= 16) return 20;
  if (d <= 32) return 36;
  return 68;
}


// Resident warps per SM of the ms_step kernel used for dimension d (queried
// once per dimension from the occupancy calculator).
int step_resident_warps_per_sm(int d) {
  static int cache[FMS_MAX_DIM_PAD + 1] = {0};
  if (d < 1 || d > FMS_MAX_DIM_PAD) return 8;
  if (cache[d]) return cache[d];
  int blocks = 0, threads = 256;
  cudaError_t e = cudaSuccess;
  switch (d) {
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ms_step_lowd<1, 4, 2>, 256, 0); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ms_step_lowd<2, 4, 4>, 256, 0); break;
    case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ms_step_lowd<3, 4, 4>, 256, 0); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ms_step_lowd<4, 4, 8>, 256, 0); break;
    case 5: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ms_step_lowd<5, 8, 8>, 256, 0); break;
    case 6: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ms_step_lowd<6, 8, 8>, 256, 0); break;
    case 7: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ms_step_lowd<7, 8, 8>, 256, 0); break;
    default:
      threads = 128;
      if (d <= 8) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ms_step_wide<8, 4>, 128, 0);
      else if (d <= 16) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ms_step_wide<16, 2>, 128, 0);
      else if (d <= 32) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ms_step_wide<32, 1>, 128, 0);
      else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ms_step_wide<64, 1>, 128, 0);
      break;
  }
  if (e != cudaSuccess || blocks < 1) blocks = 1;
  cache[d] = blocks * threads / 32;
  return cache[d];
}

cudaError_t launch_ms_step(const float* Xs, int64_t n, int d, int DP, const float* y,
                           const int32_t* active, const int32_t* s_ptr, const int32_t* C_ptr,
                           const int32_t* Lc_ptr, float* part, int target_warps, cudaStream_t st,
                           int32_t* s_log) {
  const dim3 g((target_warps + 7) / 8);
  const int grid_ctas = (int)g.x;
  switch (d) {
    case 1: ms_step_lowd<1, 4, 2><<<g, 256, 0, st>>>(Xs, n, y, active, s_ptr, C_ptr, Lc_ptr, part, s_log); break;
    case 2: ms_step_lowd<2, 4, 4><<<g, 256, 0, st>>>(Xs, n, y, active, s_ptr, C_ptr, Lc_ptr, part, s_log); break;
    case 3: ms_step_lowd<3, 4, 4><<<g, 256, 0, st>>>(Xs, n, y, active, s_ptr, C_ptr, Lc_ptr, part, s_log); break;
    case 4: ms_step_lowd<4, 4, 8><<<g, 256, 0, st>>>(Xs, n, y, active, s_ptr, C_ptr, Lc_ptr, part, s_log); break;
    case 5: ms_step_lowd<5, 8, 8><<<g, 256, 0, st>>>(Xs, n, y, active, s_ptr, C_ptr, Lc_ptr, part, s_log); break;
    case 6: ms_step_lowd<6, 8, 8><<<g, 256, 0, st>>>(Xs, n, y, active, s_ptr, C_ptr, Lc_ptr, part, s_log); break;
    case 7: ms_step_lowd<7, 8, 8><<<g, 256, 0, st>>>(Xs, n, y, active, s_ptr, C_ptr, Lc_ptr, part, s_log); break;
    default:
      if (d <= 8)
        ms_step_wide<8, 4><<<grid_ctas * 2, 128, 0, st>>>(Xs, n, DP, y, active, s_ptr, C_ptr, Lc_ptr, part, s_log);
      else if (d <= 16)
        ms_step_wide<16, 2><<<grid_ctas * 2, 128, 0, st>>>(Xs, n, DP, y, active, s_ptr, C_ptr, Lc_ptr, part, s_log);
      else if (d <= 32)
        ms_step_wide<32, 1><<<grid_ctas * 2, 128, 0, st>>>(Xs, n, DP, y, active, s_ptr, C_ptr, Lc_ptr, part, s_log);
      else
        ms_step_wide<64, 1><<<grid_ctas * 2, 128, 0, st>>>(Xs, n, DP, y, active, s_ptr, C_ptr, Lc_ptr, part, s_log);
      break;
  }
  return cudaGetLastError();
}

}  // namespace fms
