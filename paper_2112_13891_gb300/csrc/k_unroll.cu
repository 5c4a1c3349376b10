// Differentiable unrolled mean-shift steps: T Gaussian updates of every seed
// (for B independent sets at once) and their adjoint.
//
// Forward (Eq. 6 with the Gaussian weight), for each set and seed i:
//   W_i = sum_j w_ij,  y_i <- mu_i = sum_j w_ij x_j / W_i,
//   w_ij = exp(-||y_i - x_j||^2 / (2h^2)) = exp2(-c ||y_i - x_j||^2), c = log2(e)/(2h^2).
// Adjoint of one update, with p_ij = w_ij / W_i, g_i = dL/dmu_i and
// a_ij = g_i . (x_j - mu_i) (derived by differentiating log w_ij):
//   dL/dy_i  = (1/h^2) sum_j p_ij a_ij (x_j - mu_i)
//   dL/dx_j += p_ij [g_i - a_ij (x_j - y_i) / h^2]
//   dL/dh   += (1/h^3) sum_ij p_ij ||y_i - x_j||^2 a_ij
// The weights are recomputed tile by tile: nothing of size m x n is stored.
// Positions Y_t are checkpointed every k updates; the backward recomputes one
// segment of k updates from its checkpoint, then walks it in reverse.
//
// Kernels (FP32, or FP64 for checking gradients; exact differences,
// fixed-order reductions; rows padded to DPAD = 4, 8, 16 or 32 values, the
// padding known at compile time):
//   fwd_partial   lanes own R seeds, points streamed with warp-uniform loads
//                 (the next point's row loaded while this one is evaluated),
//                 partial (W, S = sum w (x - y)) per point chunk
//   fwd_finish    y' = y + S/W, W_t kept for the backward; a seed whose W
//                 underflows (every point farther than ~13 h) is listed for
//   fwd_rescue    which recomputes it with the weights taken relative to its
//                 nearest point, w = exp2(-c (D2 - D2min)) (the shift cancels
//                 in w / W), and records the shift c D2min for the backward
//   seed_data     one row per seed [y | g | 1/W, shift, g . (y - mu)] for
//                 the adjoint passes (no division or scattered load per pair)
//   bwd_seed      lanes own seeds: partial sum_j p a (x - y), sum_j p a and
//                 sum_j p a ||y - x||^2 per point chunk
//   bwd_point     lanes own R points, seeds streamed: partial
//                 sum_i p_ij [g_i - a_ij (x_j - y_i) / h^2] per seed chunk
// Both adjoint passes take a_ij = g_i . (x_j - y_i) + g_i . (y_i - mu_i): every
// term is a difference of nearby positions (no cancellation of coordinates).
//   finish kernels sum the chunk partials in chunk order.
#include "fms_internal.cuh"
#include "fms_tc.cuh"

namespace fms {

template <int DPAD>
__device__ __forceinline__ void load_row(const float* __restrict__ p, float (&v)[DPAD]) {
#pragma unroll
  for (int q = 0; q < DPAD / 4; ++q) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p) + q);
    v[4 * q] = t.x;
    v[4 * q + 1] = t.y;
    v[4 * q + 2] = t.z;
    v[4 * q + 3] = t.w;
  }
}

template <int DPAD>
__device__ __forceinline__ void load_row(const double* __restrict__ p, double (&v)[DPAD]) {
#pragma unroll
  for (int q = 0; q < DPAD / 2; ++q) {
    const double2 t = __ldg(reinterpret_cast<const double2*>(p) + q);
    v[2 * q] = t.x;
    v[2 * q + 1] = t.y;
  }
}

// a row already in shared memory (staged by the ring): plain vector loads
template <int DPAD>
__device__ __forceinline__ void smem_row(const float* p, float (&v)[DPAD]) {
#pragma unroll
  for (int q = 0; q < DPAD / 4; ++q) {
    const float4 t = reinterpret_cast<const float4*>(p)[q];
    v[4 * q] = t.x;
    v[4 * q + 1] = t.y;
    v[4 * q + 2] = t.z;
    v[4 * q + 3] = t.w;
  }
}
template <int DPAD>
__device__ __forceinline__ void smem_row(const double* p, double (&v)[DPAD]) {
#pragma unroll
  for (int q = 0; q < DPAD / 2; ++q) {
    const double2 t = reinterpret_cast<const double2*>(p)[q];
    v[2 * q] = t.x;
    v[2 * q + 1] = t.y;
  }
}

// Per-warp staging rings of the three pair kernels (tc::ring_rows): the
// forward and seed-major passes stream point rows (DPAD values), the
// point-major pass streams seed rows (2 DPAD + 4 values); 4 warps per CTA.
template <typename T, int ROW>
constexpr int unroll_ring_smem() {
  return 4 * 2 * tc::kRingRows * ROW * (int)sizeof(T);
}

// the element type's exp2, fma and min (FP32: the MUFU exp2 with flush to zero)
__device__ __forceinline__ float uex2(float x) { return ex2_ftz(x); }
__device__ __forceinline__ double uex2(double x) { return exp2(x); }
__device__ __forceinline__ float ufma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double ufma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float umin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double umin(double a, double b) { return fmin(a, b); }

// Below this W the unshifted weights lose precision (FP32 terms under 2^-126
// flush to zero) and the seed is recomputed with a shift.
template <typename T>
__device__ __forceinline__ T unroll_min_w() {
  return sizeof(T) == 4 ? (T)1e-20f : (T)1e-280;
}

// seeds (forward, seed-major adjoint) or points (point-major adjoint) per lane
template <typename T, int DPAD>
constexpr int unroll_fwd_r() {
  return sizeof(T) != 4 ? 1 : (DPAD <= 4 ? 4 : (DPAD <= 8 ? 2 : 1));
}
template <typename T, int DPAD>
constexpr int unroll_point_r() {
  return sizeof(T) != 4 ? 1 : (DPAD <= 16 ? 2 : 1);
}

// ---- forward partials: grid-stride over (set, seed group of 32 R, point chunk)
template <typename T, int DPAD, int R>
__global__ void __launch_bounds__(128)
    unroll_fwd_partial(const T* __restrict__ X, const T* __restrict__ Y, UGeom g,
                       T c, T* __restrict__ part, uint32_t* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char ring_smem[];
  __shared__ __align__(8) uint64_t ring_bars[4][2];
  constexpr int SPW = 32 * R;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* tiles = reinterpret_cast<T*>(ring_smem) + warp * 2 * tc::kRingRows * DPAD;
  tc::ring_init(ring_bars[warp], lane);
  uint32_t use0 = 0u, use1 = 0u;
  const int Gs = (g.m + SPW - 1) / SPW;
  const int64_t NT = (int64_t)g.B * Gs * g.Cp;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t task = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); task < NT;
       task += nw) {
    const int ch = (int)(task % g.Cp);
    const int64_t rest = task / g.Cp;
    const int gs = (int)(rest % Gs);
    const int b = (int)(rest / Gs);
    const T* Xb = X + (int64_t)b * g.n * DPAD;
    T y[R][DPAD], S[R][DPAD], W[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = min(gs * SPW + r * 32 + lane, g.m - 1);
      load_row<DPAD>(Y + ((int64_t)b * g.m + i) * DPAD, y[r]);
      W[r] = T(0);
#pragma unroll
      for (int k = 0; k < DPAD; ++k) S[r][k] = T(0);
    }
    const int j0 = ch * g.Lp, j1 = min(g.n, j0 + g.Lp);
    const bool ok = tc::ring_rows<DPAD>(Xb, j0, j1, tiles, ring_bars[warp], use0, use1, lane,
                                        status, [&](const T* row) {
      T x[DPAD];
      smem_row<DPAD>(row, x);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        T dx[DPAD], D2 = T(0);
#pragma unroll
        for (int k = 0; k < DPAD; ++k) {
          dx[k] = x[k] - y[r][k];
          D2 = ufma(dx[k], dx[k], D2);
        }
        const T w = uex2(-c * D2);
        W[r] += w;
#pragma unroll
        for (int k = 0; k < DPAD; ++k) S[r][k] = ufma(w, dx[k], S[r][k]);
      }
    });
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = gs * SPW + r * 32 + lane;
      if (!ok) W[r] = T(NAN);   // a wait gave up: the seed's update comes out NaN
      if (i < g.m) {
        T* o = part + (((int64_t)b * g.Cp + ch) * g.m + i) * (DPAD + 1);
        o[0] = W[r];
#pragma unroll
        for (int k = 0; k < DPAD; ++k)
          if (k < g.d) o[1 + k] = S[r][k];
      }
    }
    if (!ok) break;
  }
}

// y_next = y + S/W (sums over chunks in chunk order), W kept for the backward.
// Seeds with W < unroll_min_w<T>() (or not finite) go to the rescue list instead.
template <typename T>
__global__ void unroll_fwd_finish(const T* __restrict__ part, const T* __restrict__ Y,
                                  UGeom g, T* __restrict__ Ynext, T* __restrict__ Wout,
                                  T* __restrict__ Sh, int32_t* __restrict__ rlist,
                                  int32_t* __restrict__ rcount) {
  const int64_t total = (int64_t)g.B * g.m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / g.m), i = (int)(e % g.m);
    T W = T(0);
    for (int ch = 0; ch < g.Cp; ++ch) W += part[(((int64_t)b * g.Cp + ch) * g.m + i) * (g.DP + 1)];
    if (!(W >= unroll_min_w<T>()) || !isfinite(W)) {
      rlist[atomicAdd(rcount, 1)] = (int32_t)e;
      continue;
    }
    if (Wout) Wout[e] = W;
    if (Sh) Sh[e] = T(0);
    for (int k = 0; k < g.DP; ++k) {
      T v = T(0);
      if (k < g.d) {
        T S = T(0);
        for (int ch = 0; ch < g.Cp; ++ch)
          S += part[(((int64_t)b * g.Cp + ch) * g.m + i) * (g.DP + 1) + 1 + k];
        v = Y[e * g.DP + k] + S / W;
      }
      Ynext[e * g.DP + k] = v;
    }
  }
}

// Recomputes the listed seeds (one warp each, points over lanes): pass 1 the
// nearest squared distance D2min, pass 2 the weights exp2(-c (D2 - D2min)),
// their sums (fixed xor tree over lanes) and y' = y + S/W; the shift c D2min
// goes to Sh for the backward.  One block; it clears the list count at the end.
template <typename T, int DPAD>
__global__ void __launch_bounds__(1024)
    unroll_fwd_rescue(const T* __restrict__ X, const T* __restrict__ Y, UGeom g, T c,
                      const int32_t* __restrict__ rlist, int32_t* rcount,
                      T* __restrict__ Ynext, T* __restrict__ Wout,
                      T* __restrict__ Sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cnt = *(volatile int32_t*)rcount;
  for (int q = warp; q < cnt; q += (int)(blockDim.x >> 5)) {
    const int64_t e = rlist[q];
    const int b = (int)(e / g.m);
    const T* Xb = X + (int64_t)b * g.n * DPAD;
    T y[DPAD];
    load_row<DPAD>(Y + e * DPAD, y);
    T dmin = T(INFINITY);
    for (int j = lane; j < g.n; j += 32) {
      T x[DPAD];
      load_row<DPAD>(Xb + (int64_t)j * DPAD, x);
      T D2 = T(0);
#pragma unroll
      for (int k = 0; k < DPAD; ++k) {
        const T e = x[k] - y[k];
        D2 = ufma(e, e, D2);
      }
      dmin = umin(dmin, D2);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) dmin = umin(dmin, __shfl_xor_sync(kFull, dmin, o));
    const T sh = c * dmin;
    T W = T(0), S[DPAD];
#pragma unroll
    for (int k = 0; k < DPAD; ++k) S[k] = T(0);
    for (int j = lane; j < g.n; j += 32) {
      T x[DPAD];
      load_row<DPAD>(Xb + (int64_t)j * DPAD, x);
      T dx[DPAD], D2 = T(0);
#pragma unroll
      for (int k = 0; k < DPAD; ++k) {
        dx[k] = x[k] - y[k];
        D2 = ufma(dx[k], dx[k], D2);
      }
      const T w = uex2(ufma(-c, D2, sh));
      W += w;
#pragma unroll
      for (int k = 0; k < DPAD; ++k) S[k] = ufma(w, dx[k], S[k]);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      W += __shfl_xor_sync(kFull, W, o);
#pragma unroll
      for (int k = 0; k < DPAD; ++k) S[k] += __shfl_xor_sync(kFull, S[k], o);
    }
    if (lane == 0) {
      if (Wout) Wout[e] = W;
      if (Sh) Sh[e] = sh;
#pragma unroll
      for (int k = 0; k < DPAD; ++k)
        if (k < g.DP) Ynext[e * g.DP + k] = k < g.d ? y[k] + S[k] / W : T(0);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *rcount = 0;
}

// ---- adjoint inputs per seed: SD row = [y | g | 1/W, shift, g . (y - mu), 0]
template <typename T, int DPAD>
__global__ void unroll_seed_data(const T* __restrict__ Y, const T* __restrict__ MU,
                                 const T* __restrict__ G, const T* __restrict__ Wt,
                                 const T* __restrict__ Sh, UGeom g, T* __restrict__ SD) {
  constexpr int SDW = 2 * DPAD + 4;
  const int64_t total = (int64_t)g.B * g.m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    T* o = SD + e * SDW;
    T gm = T(0);
#pragma unroll
    for (int k = 0; k < DPAD; ++k) {
      const T gk = G[e * DPAD + k];
      o[k] = Y[e * DPAD + k];
      o[DPAD + k] = gk;
      gm = ufma(gk, Y[e * DPAD + k] - MU[e * DPAD + k], gm);
    }
    o[2 * DPAD] = T(1) / Wt[e];
    o[2 * DPAD + 1] = Sh[e];
    o[2 * DPAD + 2] = gm;
    o[2 * DPAD + 3] = T(0);
  }
}

// ---- backward, seed-major: partial sums over point chunks of
//   DY_i = sum_j p_ij a_ij (x_j - mu_i) = sum_j p a (x_j - y_i) + (y_i - mu_i) sum_j p a,
//   DH_i = sum_j p_ij a_ij ||y_i - x_j||^2 = sum_j p a (||y_i - x_j||^2 - s_i).
// The last form holds for any s_i because sum_j p_ij a_ij = g_i . sum_j p_ij
// (x_j - mu_i) = 0; s_i = the seed's weight shift in squared-distance units
// (0 unless the seed was rescued).  For a seed far from every point (D2 of
// hundreds) the FP32 rounding of D2 perturbs its weights by ~1e-5, which
// leaves sum p a at ~1e-5 instead of 0; subtracting s_i keeps that residual
// from being multiplied by D2.
template <typename T, int DPAD>
__global__ void __launch_bounds__(128)
    unroll_bwd_seed(const T* __restrict__ X, const T* __restrict__ MU,
                    const T* __restrict__ SD, UGeom g, T c, T* __restrict__ part,
                    uint32_t* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char ring_smem[];
  __shared__ __align__(8) uint64_t ring_bars[4][2];
  constexpr int SDW = 2 * DPAD + 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* tiles = reinterpret_cast<T*>(ring_smem) + warp * 2 * tc::kRingRows * DPAD;
  tc::ring_init(ring_bars[warp], lane);
  uint32_t use0 = 0u, use1 = 0u;
  const int Gs = (g.m + 31) / 32;
  const int64_t NT = (int64_t)g.B * Gs * g.Cp;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t task = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); task < NT;
       task += nw) {
    const int ch = (int)(task % g.Cp);
    const int64_t rest = task / g.Cp;
    const int gs = (int)(rest % Gs);
    const int b = (int)(rest / Gs);
    const int i = min(gs * 32 + lane, g.m - 1);
    const int64_t row = (int64_t)b * g.m + i;
    const T* Xb = X + (int64_t)b * g.n * DPAD;
    const T* sd = SD + row * SDW;
    T y[DPAD], gg[DPAD], DY[DPAD], DH = T(0), SA = T(0);
    load_row<DPAD>(sd, y);
    load_row<DPAD>(sd + DPAD, gg);
    T tail[4];
    load_row<4>(sd + 2 * DPAD, tail);
    const T invW = tail[0], sh = tail[1], gd = tail[2];
    const T s0 = sh / c;
#pragma unroll
    for (int k = 0; k < DPAD; ++k) DY[k] = T(0);
    const int j0 = ch * g.Lp, j1 = min(g.n, j0 + g.Lp);
    const bool ok = tc::ring_rows<DPAD>(Xb, j0, j1, tiles, ring_bars[warp], use0, use1, lane,
                                        status, [&](const T* row) {
      T x[DPAD];
      smem_row<DPAD>(row, x);
      T dx[DPAD], D2 = T(0), a = gd;
#pragma unroll
      for (int k = 0; k < DPAD; ++k) {
        dx[k] = x[k] - y[k];
        D2 = ufma(dx[k], dx[k], D2);
        a = ufma(gg[k], dx[k], a);
      }
      const T pa = uex2(ufma(-c, D2, sh)) * invW * a;
      DH = ufma(pa, D2 - s0, DH);
      SA += pa;
#pragma unroll
      for (int k = 0; k < DPAD; ++k) DY[k] = ufma(pa, dx[k], DY[k]);
    });
    if (!ok) DH = T(NAN);   // a wait gave up: the gradient comes out NaN
    if (gs * 32 + lane < g.m) {
      T mu[DPAD];
      load_row<DPAD>(MU + row * DPAD, mu);
      T* o = part + (((int64_t)b * g.Cp + ch) * g.m + i) * (DPAD + 1);
      o[0] = DH;
#pragma unroll
      for (int k = 0; k < DPAD; ++k)
        if (k < g.d) o[1 + k] = ok ? ufma(y[k] - mu[k], SA, DY[k]) : T(NAN);
    }
    if (!ok) break;
  }
}

// G_prev = DY / h^2 (the gradient w.r.t. the positions before this update);
// dh_part[b*m + i] = DH_i / h^3.
template <typename T>
__global__ void unroll_bwd_seed_finish(const T* __restrict__ part, UGeom g, T inv_h2,
                                       T inv_h3, T* __restrict__ Gprev,
                                       T* __restrict__ dh_part) {
  const int64_t total = (int64_t)g.B * g.m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / g.m), i = (int)(e % g.m);
    T DH = T(0);
    for (int ch = 0; ch < g.Cp; ++ch) DH += part[(((int64_t)b * g.Cp + ch) * g.m + i) * (g.DP + 1)];
    dh_part[e] = DH * inv_h3;
    for (int k = 0; k < g.DP; ++k) {
      T v = T(0);
      if (k < g.d) {
        for (int ch = 0; ch < g.Cp; ++ch)
          v += part[(((int64_t)b * g.Cp + ch) * g.m + i) * (g.DP + 1) + 1 + k];
        v *= inv_h2;
      }
      Gprev[e * g.DP + k] = v;
    }
  }
}

// ---- backward, point-major: partial over seed chunks of
//   DX_j = sum_i p_ij g_i - (1/h^2) sum_i p_ij a_ij (x_j - y_i).
// Lanes own R points; the seed rows (SD) are read with warp-uniform loads.
template <typename T, int DPAD, int R>
__global__ void __launch_bounds__(128)
    unroll_bwd_point(const T* __restrict__ X, const T* __restrict__ SD, UGeom g, T c,
                     T inv_h2, T* __restrict__ part, uint32_t* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char ring_smem[];
  __shared__ __align__(8) uint64_t ring_bars[4][2];
  constexpr int SDW = 2 * DPAD + 4;
  constexpr int PPW = 32 * R;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* tiles = reinterpret_cast<T*>(ring_smem) + warp * 2 * tc::kRingRows * SDW;
  tc::ring_init(ring_bars[warp], lane);
  uint32_t use0 = 0u, use1 = 0u;
  const int Gp = (g.n + PPW - 1) / PPW;
  const int64_t NT = (int64_t)g.B * Gp * g.Cs;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t task = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); task < NT;
       task += nw) {
    const int ch = (int)(task % g.Cs);
    const int64_t rest = task / g.Cs;
    const int gp = (int)(rest % Gp);
    const int b = (int)(rest / Gp);
    T x[R][DPAD], DX[R][DPAD];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int j = min(gp * PPW + r * 32 + lane, g.n - 1);
      load_row<DPAD>(X + ((int64_t)b * g.n + j) * DPAD, x[r]);
#pragma unroll
      for (int k = 0; k < DPAD; ++k) DX[r][k] = T(0);
    }
    const int i0 = ch * g.Ls, i1 = min(g.m, i0 + g.Ls);
    const T* sdb = SD + (int64_t)b * g.m * SDW;
    const bool ok = tc::ring_rows<SDW>(sdb, i0, i1, tiles, ring_bars[warp], use0, use1, lane,
                                       status, [&](const T* sd) {
      T y[DPAD], gg[DPAD];
      smem_row<DPAD>(sd, y);
      smem_row<DPAD>(sd + DPAD, gg);
      T tail[4];
      smem_row<4>(sd + 2 * DPAD, tail);
      const T invW = tail[0], sh = tail[1], gd = tail[2];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        T dx[DPAD], D2 = T(0), a = gd;
#pragma unroll
        for (int k = 0; k < DPAD; ++k) {
          dx[k] = x[r][k] - y[k];
          D2 = ufma(dx[k], dx[k], D2);
          a = ufma(gg[k], dx[k], a);
        }
        const T p = uex2(ufma(-c, D2, sh)) * invW;
        const T q = p * a * inv_h2;
#pragma unroll
        for (int k = 0; k < DPAD; ++k) DX[r][k] = ufma(p, gg[k], ufma(-q, dx[k], DX[r][k]));
      }
    });
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int j = gp * PPW + r * 32 + lane;
      if (!ok)
#pragma unroll
        for (int k = 0; k < DPAD; ++k) DX[r][k] = T(NAN);   // a wait gave up
      if (j < g.n) {
        T* o = part + (((int64_t)b * g.Cs + ch) * g.n + j) * DPAD;
#pragma unroll
        for (int k = 0; k < DPAD; ++k) o[k] = k < g.d ? DX[r][k] : T(0);
      }
    }
    if (!ok) break;
  }
}

// dX += sum over seed chunks (chunk order).
template <typename T>
__global__ void unroll_bwd_point_finish(const T* __restrict__ part, UGeom g,
                                        T* __restrict__ dX) {
  const int64_t total = (int64_t)g.B * g.n * g.DP;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t bj = e / g.DP;
    const int k = (int)(e % g.DP);
    const int b = (int)(bj / g.n), j = (int)(bj % g.n);
    T v = T(0);
    for (int ch = 0; ch < g.Cs; ++ch) v += part[(((int64_t)b * g.Cs + ch) * g.n + j) * g.DP + k];
    dX[e] += v;
  }
}

// dh[b] += sum_i dh_part[b, i] in FP64, seeds in order (one block per set).
template <typename T>
__global__ void unroll_dh_reduce(const T* __restrict__ dh_part, UGeom g,
                                 double* __restrict__ dh) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < g.m; i += blockDim.x) s += (double)dh_part[(int64_t)b * g.m + i];
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    dh[b] += t;
  }
}

// Row repacking between the caller's [rows x d] and the padded [rows x DP].
template <typename T>
__global__ void unroll_pack(const T* __restrict__ src, int64_t rows, int d, int DP,
                            T* __restrict__ dst) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * DP;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / DP;
    const int k = (int)(e % DP);
    dst[e] = k < d ? src[r * d + k] : T(0);
  }
}

template <typename T>
__global__ void unroll_unpack(const T* __restrict__ src, int64_t rows, int d, int DP,
                              T* __restrict__ dst) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * d;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / d;
    const int k = (int)(e % d);
    dst[e] = src[r * DP + k];
  }
}

static int blocks_for(int64_t work, int per = 256) {
  int64_t b = (work + per - 1) / per;
  if (b < 1) b = 1;
  if (b > 8192) b = 8192;
  return (int)b;
}

// dynamic shared memory above the default 48 KB needs the kernel's attribute
// (set once per kernel)
template <typename K>
static cudaError_t ring_attr(K kernel, int bytes, bool& done) {
  if (done || bytes <= 48 * 1024) return cudaSuccess;
  const cudaError_t e =
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done = true;
  return e;
}

template <typename T, int DPAD>
static cudaError_t fwd_step_t(const T* X, const T* Y, const UGeom& g, T c, T* part, T* Ynext,
                              T* Wout, T* Sh, int32_t* rlist, int32_t* rcount, int grid,
                              uint32_t* status, cudaStream_t st) {
  constexpr int sm = unroll_ring_smem<T, DPAD>();
  static bool attr = false;
  const cudaError_t ea = ring_attr(unroll_fwd_partial<T, DPAD, unroll_fwd_r<T, DPAD>()>, sm, attr);
  if (ea != cudaSuccess) return ea;
  unroll_fwd_partial<T, DPAD, unroll_fwd_r<T, DPAD>()><<<grid, 128, sm, st>>>(X, Y, g, c, part,
                                                                               status);
  unroll_fwd_finish<T><<<blocks_for((int64_t)g.B * g.m), 256, 0, st>>>(part, Y, g, Ynext, Wout,
                                                                       Sh, rlist, rcount);
  unroll_fwd_rescue<T, DPAD><<<1, 1024, 0, st>>>(X, Y, g, c, rlist, rcount, Ynext, Wout, Sh);
  return cudaGetLastError();
}

template <typename T>
cudaError_t unroll_fwd_step(const T* X, const T* Y, const UGeom& g, T c, T* part, T* Ynext,
                            T* Wout, T* Sh, int32_t* rlist, int32_t* rcount, int grid,
                            uint32_t* status, cudaStream_t st) {
  switch (g.DP) {
    case 4: return fwd_step_t<T, 4>(X, Y, g, c, part, Ynext, Wout, Sh, rlist, rcount, grid, status, st);
    case 8: return fwd_step_t<T, 8>(X, Y, g, c, part, Ynext, Wout, Sh, rlist, rcount, grid, status, st);
    case 16: return fwd_step_t<T, 16>(X, Y, g, c, part, Ynext, Wout, Sh, rlist, rcount, grid, status, st);
    case 32: return fwd_step_t<T, 32>(X, Y, g, c, part, Ynext, Wout, Sh, rlist, rcount, grid, status, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T, int DPAD>
static cudaError_t bwd_step_t(const T* X, const T* Y, const T* MU, const T* G, const T* Wt,
                              const T* Sh, const UGeom& g, T c, T inv_h2, T inv_h3, T* part_s,
                              T* part_p, T* SD, T* dh_part, T* Gprev, T* dX, double* dh, int grid,
                              uint32_t* status, cudaStream_t st) {
  constexpr int sm_p = unroll_ring_smem<T, 2 * DPAD + 4>(), sm_s = unroll_ring_smem<T, DPAD>();
  static bool attr_p = false, attr_s = false;
  cudaError_t ea = ring_attr(unroll_bwd_point<T, DPAD, unroll_point_r<T, DPAD>()>, sm_p, attr_p);
  if (ea == cudaSuccess) ea = ring_attr(unroll_bwd_seed<T, DPAD>, sm_s, attr_s);
  if (ea != cudaSuccess) return ea;
  unroll_seed_data<T, DPAD><<<blocks_for((int64_t)g.B * g.m), 256, 0, st>>>(Y, MU, G, Wt, Sh, g,
                                                                           SD);
  unroll_bwd_point<T, DPAD, unroll_point_r<T, DPAD>()><<<grid, 128, sm_p, st>>>(
      X, SD, g, c, inv_h2, part_p, status);
  unroll_bwd_seed<T, DPAD><<<grid, 128, sm_s, st>>>(X, MU, SD, g, c, part_s, status);
  unroll_bwd_point_finish<T><<<blocks_for((int64_t)g.B * g.n * g.DP), 256, 0, st>>>(part_p, g, dX);
  unroll_bwd_seed_finish<T><<<blocks_for((int64_t)g.B * g.m), 256, 0, st>>>(part_s, g, inv_h2,
                                                                            inv_h3, Gprev,
                                                                            dh_part);
  unroll_dh_reduce<T><<<g.B, 256, 0, st>>>(dh_part, g, dh);
  return cudaGetLastError();
}

template <typename T>
cudaError_t unroll_bwd_step(const T* X, const T* Y, const T* MU, const T* G, const T* Wt,
                            const T* Sh, const UGeom& g, T c, T inv_h2, T inv_h3, T* part_s,
                            T* part_p, T* SD, T* dh_part, T* Gprev, T* dX, double* dh, int grid,
                            uint32_t* status, cudaStream_t st) {
  switch (g.DP) {
    case 4: return bwd_step_t<T, 4>(X, Y, MU, G, Wt, Sh, g, c, inv_h2, inv_h3, part_s, part_p, SD, dh_part, Gprev, dX, dh, grid, status, st);
    case 8: return bwd_step_t<T, 8>(X, Y, MU, G, Wt, Sh, g, c, inv_h2, inv_h3, part_s, part_p, SD, dh_part, Gprev, dX, dh, grid, status, st);
    case 16: return bwd_step_t<T, 16>(X, Y, MU, G, Wt, Sh, g, c, inv_h2, inv_h3, part_s, part_p, SD, dh_part, Gprev, dX, dh, grid, status, st);
    case 32: return bwd_step_t<T, 32>(X, Y, MU, G, Wt, Sh, g, c, inv_h2, inv_h3, part_s, part_p, SD, dh_part, Gprev, dX, dh, grid, status, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t unroll_pack_rows(const T* src, int64_t rows, int d, int DP, T* dst, cudaStream_t st) {
  unroll_pack<T><<<blocks_for(rows * DP), 256, 0, st>>>(src, rows, d, DP, dst);
  return cudaGetLastError();
}

template <typename T>
cudaError_t unroll_unpack_rows(const T* src, int64_t rows, int d, int DP, T* dst,
                               cudaStream_t st) {
  unroll_unpack<T><<<blocks_for(rows * d), 256, 0, st>>>(src, rows, d, DP, dst);
  return cudaGetLastError();
}

#define FMS_UNROLL_INST(T)                                                                      \
  template cudaError_t unroll_fwd_step<T>(const T*, const T*, const UGeom&, T, T*, T*, T*, T*,  \
                                          int32_t*, int32_t*, int, uint32_t*, cudaStream_t);   \
  template cudaError_t unroll_bwd_step<T>(const T*, const T*, const T*, const T*, const T*,     \
                                          const T*, const UGeom&, T, T, T, T*, T*, T*, T*, T*, \
                                          T*, double*, int, uint32_t*, cudaStream_t);          \
  template cudaError_t unroll_pack_rows<T>(const T*, int64_t, int, int, T*, cudaStream_t);      \
  template cudaError_t unroll_unpack_rows<T>(const T*, int64_t, int, int, T*, cudaStream_t);
FMS_UNROLL_INST(float)
FMS_UNROLL_INST(double)
#undef FMS_UNROLL_INST

}  // namespace fms
