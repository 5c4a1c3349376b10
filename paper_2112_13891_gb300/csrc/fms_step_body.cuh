// Per-task bodies of the ms_step kernels, shared by the single-set kernels
// (k_step.cu) and the batched kernels (k_batched.cu).
#pragma once

#include "fms_internal.cuh"
#include "fms_tc.cuh"

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

// R seeds in registers against one point: exact differences, one weight each.
template <int D, int R, int DA, int KF = kKernelGaussian>
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
    const float w = kweight<KF>(t);
    acc[r][0] += w;
#pragma unroll
    for (int k = 0; k < D; ++k) acc[r][1 + k] = fmaf(w, dx[k], acc[r][1 + k]);
  }
}

// One low-d warp task: R seeds (active positions g*R.., clamped to s-1) of a
// set against the points [j0, j1) of that set; writes 32 partials to
// part_task (index (c * s + p) * DA + k relative to the set's partial block).
template <int D, int DP, int DA, int KF = kKernelGaussian>
__device__ __forceinline__ void lowd_task(const float* __restrict__ Xs, int j0, int j1,
                                          const float* __restrict__ y,
                                          const int32_t* __restrict__ active, int s, int g, int c,
                                          float* __restrict__ part, int lane) {
  constexpr int R = 32 / DA;
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
    eval_point<D, R, DA, KF>(x, ys, acc);
    coords<D, DP>(p1, x);
    eval_point<D, R, DA, KF>(x, ys, acc);
    coords<D, DP>(p2, x);
    eval_point<D, R, DA, KF>(x, ys, acc);
    coords<D, DP>(p3, x);
    eval_point<D, R, DA, KF>(x, ys, acc);
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

// One wide warp task: lanes own seeds (RG per lane, 32*RG seeds per task),
// points [j0, j1) staged into shared memory 32 rows at a time by bulk copies
// (TMA) into a two-tile ring of the warp's own (tiles: 2 x 32 x DPAD floats,
// bars: two mbarriers of count 1, use0 / use1: completed phases of each,
// carried across the warp's tasks), read back with broadcast loads; DA = DPAD + 4.
// Group g covers active positions p_lo + g*32*RG ... (positions below p_lo
// belong to the tensor-core step).  Every wait is bounded: one that gives up
// sets kStTimeout in *status, waits once more for the warp's copies in flight
// and makes the task return false (the caller stops).
constexpr int kWideTile = tc::kRingRows;   // rows per staged tile (tc::ring_init sets up the ring)

// dynamic shared memory of a 128-thread CTA of wide tasks: 4 warps x 2 tiles
template <int DPAD>
constexpr int wide_smem_bytes() {
  return 4 * 2 * kWideTile * DPAD * 4;
}

template <int DPAD, int RG, int KF = kKernelGaussian>
__device__ __forceinline__ bool wide_task(const float* __restrict__ Xs, int j0, int j1,
                                          const float* __restrict__ y,
                                          const int32_t* __restrict__ active, int s, int g, int c,
                                          float* __restrict__ part, int lane, int p_lo,
                                          float* tiles, uint64_t* bars, uint32_t& use0,
                                          uint32_t& use1, uint32_t* status) {
  constexpr int DA = DPAD + 4;
  constexpr int SPW = 32 * RG;
  float ys[RG][DPAD];
  float acc[RG][DPAD + 1];
#pragma unroll
  for (int r = 0; r < RG; ++r) {
    int p = p_lo + g * SPW + r * 32 + lane;
    p = p < s ? p : s - 1;
    const int64_t slot = __ldg(active + p);
#pragma unroll
    for (int k = 0; k < DPAD; ++k) ys[r][k] = __ldg(y + slot * DPAD + k);
#pragma unroll
    for (int k = 0; k <= DPAD; ++k) acc[r][k] = 0.0f;
  }
  const bool ok = tc::ring_rows<DPAD>(Xs, j0, j1, tiles, bars, use0, use1, lane, status,
                                      [&](const float* row) {
    float x[DPAD];
    const float4* xp = reinterpret_cast<const float4*>(row);
#pragma unroll
    for (int u = 0; u < DPAD / 4; ++u) {
      const float4 v = xp[u];
      x[4 * u] = v.x;
      x[4 * u + 1] = v.y;
      x[4 * u + 2] = v.z;
      x[4 * u + 3] = v.w;
    }
#pragma unroll
    for (int r = 0; r < RG; ++r) {
      float dx[DPAD];
#pragma unroll
      for (int k = 0; k < DPAD; ++k) dx[k] = x[k] - ys[r][k];
      float tt = -dx[0] * dx[0];
#pragma unroll
      for (int k = 1; k < DPAD; ++k) tt = fmaf(-dx[k], dx[k], tt);
      const float w = kweight<KF>(tt);
      acc[r][0] += w;
#pragma unroll
      for (int k = 0; k < DPAD; ++k) acc[r][1 + k] = fmaf(w, dx[k], acc[r][1 + k]);
    }
  });
  if (!ok) return false;
#pragma unroll
  for (int r = 0; r < RG; ++r) {
    const int p = p_lo + g * SPW + r * 32 + lane;
    if (p < s) {
      float* o = part + ((int64_t)c * s + p) * DA;
#pragma unroll
      for (int k = 0; k <= DPAD; ++k) o[k] = acc[r][k];
    }
  }
  return true;
}

// One quad warp task (8 <= d <= 16): the warp's lanes are 8 seed slots x 4
// point lanes (lane = 4 * slot + point lane); a slot holds RG seeds (8 * RG
// seeds per task), point lane q walks the chunk's points j0 + q, j0 + q + 4,
// ... in increasing order, and the four point lanes of a slot are combined by
// a fixed two-level xor tree.  Each point load feeds 8 * RG evaluations, and a
// task needs only 8 * RG seeds, so chunks stay long when few seeds are active
// (partials are C x s x DA floats).  The partial of a seed depends only on
// the chunk, not on the seed's slot or on the other seeds.
template <int DPAD, int RG, int KF = kKernelGaussian>
__device__ __forceinline__ void quad_task(const float* __restrict__ Xs, int DP, int j0, int j1,
                                          const float* __restrict__ y,
                                          const int32_t* __restrict__ active, int s, int g, int c,
                                          float* __restrict__ part, int lane, int p_lo = 0) {
  constexpr int DA = DPAD + 4;
  constexpr int SPT = 8 * RG;
  const int slot_l = lane >> 2, q = lane & 3;
  float ys[RG][DPAD];
  float acc[RG][DPAD + 1];
#pragma unroll
  for (int r = 0; r < RG; ++r) {
    int p = p_lo + g * SPT + r * 8 + slot_l;
    p = p < s ? p : s - 1;
    const int64_t slot = __ldg(active + p);
#pragma unroll
    for (int k = 0; k < DPAD; ++k) ys[r][k] = __ldg(y + slot * DPAD + k);
#pragma unroll
    for (int k = 0; k <= DPAD; ++k) acc[r][k] = 0.0f;
  }
  auto load_point = [&](int j, float (&x)[DPAD]) {
    const float4* xp = reinterpret_cast<const float4*>(Xs + (int64_t)j * DPAD);
#pragma unroll
    for (int u = 0; u < DPAD / 4; ++u) {
      const float4 v = __ldg(xp + u);
      x[4 * u] = v.x;
      x[4 * u + 1] = v.y;
      x[4 * u + 2] = v.z;
      x[4 * u + 3] = v.w;
    }
  };
  auto eval = [&](const float (&x)[DPAD]) {
#pragma unroll
    for (int r = 0; r < RG; ++r) {
      float dx[DPAD];
#pragma unroll
      for (int k = 0; k < DPAD; ++k) dx[k] = x[k] - ys[r][k];
      float t = -dx[0] * dx[0];
#pragma unroll
      for (int k = 1; k < DPAD; ++k) t = fmaf(-dx[k], dx[k], t);
      const float w = kweight<KF>(t);
      acc[r][0] += w;
#pragma unroll
      for (int k = 0; k < DPAD; ++k) acc[r][1 + k] = fmaf(w, dx[k], acc[r][1 + k]);
    }
  };
  // two points per step, both loads issued before either is evaluated
  int j = j0 + q;
  for (; j + 4 < j1; j += 8) {
    float xa[DPAD], xb[DPAD];
    load_point(j, xa);
    load_point(j + 4, xb);
    eval(xa);
    eval(xb);
  }
  if (j < j1) {
    float xa[DPAD];
    load_point(j, xa);
    eval(xa);
  }
#pragma unroll
  for (int r = 0; r < RG; ++r) {
#pragma unroll
    for (int k = 0; k <= DPAD; ++k) {
      float v = acc[r][k];
      v += __shfl_xor_sync(kFull, v, 1);
      v += __shfl_xor_sync(kFull, v, 2);
      acc[r][k] = v;
    }
    const int p = p_lo + g * SPT + r * 8 + slot_l;
    if (p < s) {
      float* o = part + ((int64_t)c * s + p) * DA;
#pragma unroll
      for (int k = 0; k <= DPAD; ++k)
        if ((k & 3) == q) o[k] = acc[r][k];
    }
  }
}

}  // namespace fms
