// ms_step: partial sums of one Gaussian mean-shift update for the active seeds.
//
// For every active seed y and every point x_j (Sec. II-B, the update of Alg. 2: all
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
#include "fms_step_body.cuh"

namespace fms {

// Low-dimensional path: D <= 7, DA accumulators per seed (sum w, d sums, pad),
// R = 32 / DA seeds per warp task.  Each lane keeps a ring of four points in
// flight (the loads for points i+4..i+7 are issued before points i..i+3 are
// evaluated), which hides the L1/L2 latency of the point stream.
template <int D, int DP, int DA, int KF>
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
    const int j0 = c * Lc;
    const int j1 = (int)(j0 + Lc < n ? j0 + Lc : n);
    lowd_task<D, DP, DA, KF>(Xs, j0, j1, y, active, s, g, c, part, lane);
  }
}

// Generic FP32 path for d > 8: lanes own seeds (RG per lane), every warp
// stages its chunk's points into shared memory 32 rows at a time with bulk
// copies (a two-tile ring per warp) and reads them with broadcast loads, so no
// cross-lane reduction is needed.  DPAD is the padded dimension (pad
// coordinates are zero on both sides and contribute nothing); DA = DPAD + 4
// accumulators per seed in part.
template <int DPAD, int RG, int KF>
__global__ void __launch_bounds__(128, DPAD <= 16 ? 6 : (DPAD <= 32 ? 3 : 2)) ms_step_wide(const float* __restrict__ Xs, int64_t n,
                                                    int DP, const float* __restrict__ y,
                                                    const int32_t* __restrict__ active,
                                                    const int32_t* __restrict__ s_ptr,
                                                    const int32_t* __restrict__ C_ptr,
                                                    const int32_t* __restrict__ Lc_ptr,
                                                    float* __restrict__ part,
                                                    int32_t* __restrict__ s_log,
                                                    const int32_t* __restrict__ p_lo_ptr,
                                                    uint32_t* __restrict__ status) {
  extern __shared__ __align__(16) float wide_tiles[];
  __shared__ __align__(8) uint64_t wide_bars[4][2];
  constexpr int DA = DPAD + 4;
  constexpr int SPW = 32 * RG;  // seeds per warp task
  const int s = *s_ptr;
  const int p_lo = p_lo_ptr ? *p_lo_ptr : 0;
  if (s_log && blockIdx.x == 0 && threadIdx.x == 0) *s_log = s - p_lo;
  if (s - p_lo <= 0) return;
  const int C = *C_ptr;
  const int Lc = *Lc_ptr;
  const int G = (s - p_lo + SPW - 1) / SPW;
  const int64_t T = (int64_t)G * C;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t* bars = wide_bars[warp];
  float* tiles = wide_tiles + warp * 2 * kWideTile * DPAD;
  tc::ring_init(bars, lane);
  uint32_t use0 = 0u, use1 = 0u;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t task = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; task < T; task += nw) {
    const int g = (int)(task % G);
    const int c = (int)(task / G);
    const int j0 = c * Lc;
    const int j1 = (int)(j0 + Lc < n ? j0 + Lc : n);
    if (!wide_task<DPAD, RG, KF>(Xs, j0, j1, y, active, s, g, c, part, lane, p_lo, tiles, bars,
                                 use0, use1, status))
      break;
  }
}

// d = 8: the quad kernel (8 seed slots x 4 point lanes per warp).  At d = 32
// (one seed per slot) its four distinct point rows per load cost more L1
// wavefronts per evaluation than the arithmetic can cover (measured: 73 vs 170
// Geval/s with 65,536 seeds); at 9 <= d <= 16 the staged wide kernel measured
// 8.1 against 10.7 ms for one update of 65,536 x 65,536, so quad tasks serve
// d = 8 only.
template <int DPAD, int RG, int KF>
__global__ void __launch_bounds__(128) ms_step_quad(const float* __restrict__ Xs, int64_t n,
                                                    int DP, const float* __restrict__ y,
                                                    const int32_t* __restrict__ active,
                                                    const int32_t* __restrict__ s_ptr,
                                                    const int32_t* __restrict__ C_ptr,
                                                    const int32_t* __restrict__ Lc_ptr,
                                                    float* __restrict__ part,
                                                    int32_t* __restrict__ s_log,
                                                    const int32_t* __restrict__ p_lo_ptr) {
  constexpr int SPT = 8 * RG;  // seeds per warp task
  const int s = *s_ptr;
  const int p_lo = p_lo_ptr ? *p_lo_ptr : 0;
  if (s_log && blockIdx.x == 0 && threadIdx.x == 0) *s_log = s - p_lo;
  if (s - p_lo <= 0) return;
  const int C = *C_ptr;
  const int Lc = *Lc_ptr;
  const int G = (s - p_lo + SPT - 1) / SPT;
  const int64_t T = (int64_t)G * C;
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t task = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); task < T;
       task += nw) {
    const int g = (int)(task % G);
    const int c = (int)(task / G);
    const int j0 = c * Lc;
    const int j1 = (int)(j0 + Lc < n ? j0 + Lc : n);
    quad_task<DPAD, RG, KF>(Xs, DP, j0, j1, y, active, s, g, c, part, lane, p_lo);
  }
}

int step_seeds_per_warp(int d) {
  if (d <= 1) return 16;
  if (d <= 3) return 8;
  if (d <= 7) return 4;
  if (d <= 8) return 8 * 4;    // quad kernel: 8 slots x RG seeds
  return 32;                   // wide kernel: 32 lanes x 1 seed
}

int batched_seeds_per_warp(int d) {
  if (d <= 7) return step_seeds_per_warp(d);
  if (d <= 8) return 32 * 4;   // wide tasks: 32 lanes x RG seeds
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
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ms_step_lowd<1, 4, 2, 0>, 256, 0); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ms_step_lowd<2, 4, 4, 0>, 256, 0); break;
    case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ms_step_lowd<3, 4, 4, 0>, 256, 0); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ms_step_lowd<4, 4, 8, 0>, 256, 0); break;
    case 5: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ms_step_lowd<5, 8, 8, 0>, 256, 0); break;
    case 6: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ms_step_lowd<6, 8, 8, 0>, 256, 0); break;
    case 7: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ms_step_lowd<7, 8, 8, 0>, 256, 0); break;
    default:
      threads = 128;
      if (d <= 8) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ms_step_quad<8, 4, 0>, 128, 0);
      else if (d <= 16) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ms_step_wide<16, 1, 0>, 128, wide_smem_bytes<16>());
      else if (d <= 32) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ms_step_wide<32, 1, 0>, 128, wide_smem_bytes<32>());
      else {
        e = cudaFuncSetAttribute(ms_step_wide<64, 1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, wide_smem_bytes<64>());
        if (e == cudaSuccess)
          e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ms_step_wide<64, 1, 0>, 128, wide_smem_bytes<64>());
      }
      break;
  }
  if (e != cudaSuccess || blocks < 1) blocks = 1;
  cache[d] = blocks * threads / 32;
  return cache[d];
}

template <int KF>
static cudaError_t launch_ms_step_t(const float* Xs, int64_t n, int d, int DP, const float* y,
                                   const int32_t* active, const int32_t* s_ptr,
                                   const int32_t* C_ptr, const int32_t* Lc_ptr, float* part,
                                   int target_warps, cudaStream_t st, int32_t* s_log,
                                   const int32_t* p_lo_ptr, uint32_t* status) {
  const dim3 g((target_warps + 7) / 8);
  const int grid_ctas = (int)g.x;
  // the quad and wide kernels read rows of exactly their compiled width
  if (d > 7 && DP != padded_dim(d)) return cudaErrorInvalidValue;
  switch (d) {
    case 1: ms_step_lowd<1, 4, 2, KF><<<g, 256, 0, st>>>(Xs, n, y, active, s_ptr, C_ptr, Lc_ptr, part, s_log); break;
    case 2: ms_step_lowd<2, 4, 4, KF><<<g, 256, 0, st>>>(Xs, n, y, active, s_ptr, C_ptr, Lc_ptr, part, s_log); break;
    case 3: ms_step_lowd<3, 4, 4, KF><<<g, 256, 0, st>>>(Xs, n, y, active, s_ptr, C_ptr, Lc_ptr, part, s_log); break;
    case 4: ms_step_lowd<4, 4, 8, KF><<<g, 256, 0, st>>>(Xs, n, y, active, s_ptr, C_ptr, Lc_ptr, part, s_log); break;
    case 5: ms_step_lowd<5, 8, 8, KF><<<g, 256, 0, st>>>(Xs, n, y, active, s_ptr, C_ptr, Lc_ptr, part, s_log); break;
    case 6: ms_step_lowd<6, 8, 8, KF><<<g, 256, 0, st>>>(Xs, n, y, active, s_ptr, C_ptr, Lc_ptr, part, s_log); break;
    case 7: ms_step_lowd<7, 8, 8, KF><<<g, 256, 0, st>>>(Xs, n, y, active, s_ptr, C_ptr, Lc_ptr, part, s_log); break;
    default:
      if (d <= 8)
        ms_step_quad<8, 4, KF><<<grid_ctas * 2, 128, 0, st>>>(Xs, n, DP, y, active, s_ptr, C_ptr, Lc_ptr, part, s_log, p_lo_ptr);
      else if (d <= 16)
        ms_step_wide<16, 1, KF><<<grid_ctas * 2, 128, wide_smem_bytes<16>(), st>>>(Xs, n, DP, y, active, s_ptr, C_ptr, Lc_ptr, part, s_log, p_lo_ptr, status);
      else if (d <= 32)
        ms_step_wide<32, 1, KF><<<grid_ctas * 2, 128, wide_smem_bytes<32>(), st>>>(Xs, n, DP, y, active, s_ptr, C_ptr, Lc_ptr, part, s_log, p_lo_ptr, status);
      else {
        static bool attr = false;
        if (!attr) {
          const cudaError_t e = cudaFuncSetAttribute(ms_step_wide<64, 1, KF>, cudaFuncAttributeMaxDynamicSharedMemorySize, wide_smem_bytes<64>());
          if (e != cudaSuccess) return e;
          attr = true;
        }
        ms_step_wide<64, 1, KF><<<grid_ctas * 2, 128, wide_smem_bytes<64>(), st>>>(Xs, n, DP, y, active, s_ptr, C_ptr, Lc_ptr, part, s_log, p_lo_ptr, status);
      }
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_ms_step(const float* Xs, int64_t n, int d, int DP, const float* y,
                           const int32_t* active, const int32_t* s_ptr, const int32_t* C_ptr,
                           const int32_t* Lc_ptr, float* part, int target_warps, cudaStream_t st,
                           int32_t* s_log, const int32_t* p_lo_ptr, int kf, uint32_t* status) {
  if (d > 8 && !status) return cudaErrorInvalidValue;   // the staged kernel reports timeouts
  if (kf == kKernelFlat)
    return launch_ms_step_t<kKernelFlat>(Xs, n, d, DP, y, active, s_ptr, C_ptr, Lc_ptr, part,
                                         target_warps, st, s_log, p_lo_ptr, status);
  return launch_ms_step_t<kKernelGaussian>(Xs, n, d, DP, y, active, s_ptr, C_ptr, Lc_ptr, part,
                                           target_warps, st, s_log, p_lo_ptr, status);
}

}  // namespace fms
