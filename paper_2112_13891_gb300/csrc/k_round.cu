// ms_round: one Seed-Selection round of Gaussian mean-shift updates, run by
// thread-block clusters that own disjoint seed subsets and iterate them with
// no grid-wide synchronisation.
//
// Decomposition.  A cluster of kClusterCtas CTAs (one per SM, 16 warps each)
// owns up to kSeedsPerCluster seeds.  CTA rank r of the cluster owns a fixed
// slice of the points, split again into a fixed sub-slice per warp.  In each
// update every warp evaluates all active seeds of its cluster (groups of R
// seeds in registers) against its sub-slice; the warp partials are summed in
// warp order, then the CTA partials are summed in rank order through
// distributed shared memory (partials double-buffered by update parity, so one
// cluster barrier per update suffices).  Every CTA computes the same update
// from the same sums, so the seed state stays replicated in shared memory;
// rank 0 writes it back to global memory.  A pass over the points serves a
// block of R seeds, or a full block plus a last block of at most R/2.  A seed's summation order depends only on n and the
// slice layout, never on which other seeds are active, so results do not
// depend on timing.
//
// Early Stopping (Sec. II-C) without a barrier across clusters.  Converging
// seeds add 1 to hist[c] (c = the update at which they converged).  With
// count(r) = sum_{c<=r} hist[c] over all seeds of all rounds, the stop update
// of a fresh run is t* = min{r : count(r) >= ceil(gamma*N)} and a seed is kept
// iff it converged at c <= t*.  A seed that has made k updates without
// converging may stop as soon as count(k) >= target: then t* <= k < c, so it
// cannot be kept whatever happens elsewhere.  count only grows, so a stale
// read only delays a stop; no seed is ever stopped wrongly and the kept set is
// exactly that of the synchronous rule.  Stopped seeds stay RUNNING with their
// update count (a later round may resume them).  Rank 0 takes the count test
// during the update's point pass, with the counts read at the start of the
// update, and every rank applies its decisions in the same update, after the
// cluster barrier.
#include <cooperative_groups.h>

#include "fms_internal.cuh"

namespace cg = cooperative_groups;

namespace fms {

constexpr int kRoundWarps = 16;

__device__ __forceinline__ float rs32(float (&v)[32], int lane) {
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

template <int DP>
struct RPt;
template <>
struct RPt<4> {
  float4 a;
};
template <>
struct RPt<8> {
  float4 a, b;
};

template <int DP>
__device__ __forceinline__ RPt<DP> rload(const float* __restrict__ Xs, int j, int j1) {
  RPt<DP> p;
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
__device__ __forceinline__ void rcoords(const RPt<DP>& p, float (&x)[D]) {
  float t[8];
  t[0] = p.a.x;
  t[1] = p.a.y;
  t[2] = p.a.z;
  t[3] = p.a.w;
  if constexpr (DP == 8) {
    t[4] = reinterpret_cast<const RPt<8>&>(p).b.x;
    t[5] = reinterpret_cast<const RPt<8>&>(p).b.y;
    t[6] = reinterpret_cast<const RPt<8>&>(p).b.z;
    t[7] = reinterpret_cast<const RPt<8>&>(p).b.w;
  }
#pragma unroll
  for (int k = 0; k < D; ++k) x[k] = t[k];
}

template <int D, int R, int DA, int KF>
__device__ __forceinline__ void reval(const float (&x)[D], const float (&ys)[R][D],
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

// RR seeds in registers, evaluated two at a time with packed f32x2 arithmetic
// (one FADD2/FMUL2/FFMA2 serves a pair of seeds against the same point).  For
// a pair, nd = y - x = -(x - y) exactly (an FFMA with -1), the squared
// distance, the weight and sum w are bit-identical to the scalar
// exact-difference evaluation of reval, and the pair accumulates sum w (y - x)
// = -sum w (x - y) exactly at every step (round-to-nearest is sign-symmetric),
// so every seed's sums are the same bits as reval's.  An odd last seed takes
// the scalar path.
template <int D, int RR, int KF>
struct SeedPack {
  static constexpr int NP = RR / 2;
  static constexpr int NPA = NP > 0 ? NP : 1;
  float2 yp[NPA][D];
  float2 Wp[NPA];
  float2 Sp[NPA][D];   // sum w (y - x) of the pair
  float y1[D], W1, S1[D];

  __device__ __forceinline__ void load(const float (&ys)[RR][D]) {
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      Wp[p] = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        yp[p][k] = make_float2(ys[2 * p][k], ys[2 * p + 1][k]);
        Sp[p][k] = make_float2(0.f, 0.f);
      }
    }
    W1 = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      y1[k] = (RR & 1) ? ys[RR - 1][k] : 0.f;
      S1[k] = 0.f;
    }
  }

  __device__ __forceinline__ void eval(const float (&x)[D]) {
    float2 xx[D];
#pragma unroll
    for (int k = 0; k < D; ++k) xx[k] = make_float2(x[k], x[k]);
    const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      float2 nd[D];
#pragma unroll
      for (int k = 0; k < D; ++k) nd[k] = __ffma2_rn(xx[k], m1, yp[p][k]);
      float2 dd = __fmul2_rn(nd[0], nd[0]);
#pragma unroll
      for (int k = 1; k < D; ++k) dd = __ffma2_rn(nd[k], nd[k], dd);
      const float2 w = make_float2(kweight<KF>(-dd.x), kweight<KF>(-dd.y));
      Wp[p] = __fadd2_rn(Wp[p], w);
#pragma unroll
      for (int k = 0; k < D; ++k) Sp[p][k] = __ffma2_rn(w, nd[k], Sp[p][k]);
    }
    if constexpr ((RR & 1) != 0) {
      float dx[D];
#pragma unroll
      for (int k = 0; k < D; ++k) dx[k] = x[k] - y1[k];
      float t = -dx[0] * dx[0];
#pragma unroll
      for (int k = 1; k < D; ++k) t = fmaf(-dx[k], dx[k], t);
      const float w = kweight<KF>(t);
      W1 += w;
#pragma unroll
      for (int k = 0; k < D; ++k) S1[k] = fmaf(w, dx[k], S1[k]);
    }
  }

  // accumulators of seed r: acc[r][0] = sum w, acc[r][1 + k] = sum w (x - y)_k
  template <int DA>
  __device__ __forceinline__ void store(float (&acc)[RR][DA]) const {
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      acc[2 * p][0] = Wp[p].x;
      acc[2 * p + 1][0] = Wp[p].y;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        acc[2 * p][1 + k] = -Sp[p][k].x;
        acc[2 * p + 1][1 + k] = -Sp[p][k].y;
      }
#pragma unroll
      for (int k = D + 1; k < DA; ++k) acc[2 * p][k] = acc[2 * p + 1][k] = 0.f;
    }
    if constexpr ((RR & 1) != 0) {
      acc[RR - 1][0] = W1;
#pragma unroll
      for (int k = 0; k < D; ++k) acc[RR - 1][1 + k] = S1[k];
#pragma unroll
      for (int k = D + 1; k < DA; ++k) acc[RR - 1][k] = 0.f;
    }
  }
};

// Partial sums of RR seeds (active positions a0..a0+RR-1, clamped to A-1)
// over the points [w0, w1) handled by this warp: lane l returns accumulator
// l % DA of seed l / DA (zero for seed slots beyond RR).  The arithmetic of a
// seed does not depend on RR.
template <int D, int DP, int DA, int RR, int KF>
__device__ __forceinline__ float group_partial(const float* __restrict__ Xs, int w0, int w1,
                                               int lane, const int* alist, int a0, int A,
                                               const float (*sy)[D]) {
  float ys[RR][D];
#pragma unroll
  for (int r = 0; r < RR; ++r) {
    const int i = alist[min(a0 + r, A - 1)];
#pragma unroll
    for (int k = 0; k < D; ++k) ys[r][k] = sy[i][k];
  }
  SeedPack<D, RR, KF> sp;
  sp.load(ys);
  // NB point loads per lane in flight: with few seeds a point costs few
  // instructions, so more loads must be in flight to cover the L2 latency.
  // The lane's points are evaluated in increasing order whatever NB is (and
  // points past w1 are far away, weight exactly 0), so a seed's sums have
  // the same bits in every pass shape.
  constexpr int NB = DP == 4 ? (RR <= 2 ? 12 : (RR <= 4 ? 6 : 4)) : (RR <= 1 ? 8 : 4);
  int j = w0 + lane;
  RPt<DP> b[NB];
#pragma unroll
  for (int u = 0; u < NB; ++u) b[u] = rload<DP>(Xs, j + 32 * u, w1);
  for (; j < w1; j += 32 * NB) {
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const RPt<DP> p = b[u];
      b[u] = rload<DP>(Xs, j + 32 * (NB + u), w1);
      float x[D];
      rcoords<D, DP>(p, x);
      sp.eval(x);
    }
  }
  float acc[RR][DA];
  sp.store(acc);
  float v[32];
#pragma unroll
  for (int e = 0; e < 32; ++e) v[e] = 0.0f;
#pragma unroll
  for (int r = 0; r < RR; ++r)
#pragma unroll
    for (int k = 0; k < DA; ++k) v[r * DA + k] = acc[r][k];
  return rs32(v, lane);
}

// One point pass for a full block of RA = 32 / DA seeds (active positions
// a0 ..) and a partial block of RB seeds (positions a0 + RA ..): the point
// loads are shared by both blocks.  Returns the block results in res[0]
// (lane l: accumulator l % DA of seed l / DA) and res[1].  A seed's arithmetic
// is the same as in group_partial.
template <int D, int DP, int DA, int RA, int RB, int KF>
__device__ __forceinline__ void group_pair(const float* __restrict__ Xs, int w0, int w1, int lane,
                                           const int* alist, int a0, int A, const float (*sy)[D],
                                           float (&res)[2]) {
  constexpr int RR = RA + RB;
  float ys[RR][D];
#pragma unroll
  for (int r = 0; r < RR; ++r) {
    const int i = alist[min(a0 + r, A - 1)];
#pragma unroll
    for (int k = 0; k < D; ++k) ys[r][k] = sy[i][k];
  }
  SeedPack<D, RR, KF> sp;
  sp.load(ys);
  int j = w0 + lane;
  RPt<DP> b0 = rload<DP>(Xs, j, w1), b1 = rload<DP>(Xs, j + 32, w1);
  RPt<DP> b2 = rload<DP>(Xs, j + 64, w1), b3 = rload<DP>(Xs, j + 96, w1);
  for (; j < w1; j += 128) {
    const RPt<DP> p0 = b0, p1 = b1, p2 = b2, p3 = b3;
    b0 = rload<DP>(Xs, j + 128, w1);
    b1 = rload<DP>(Xs, j + 160, w1);
    b2 = rload<DP>(Xs, j + 192, w1);
    b3 = rload<DP>(Xs, j + 224, w1);
    float x[D];
    rcoords<D, DP>(p0, x);
    sp.eval(x);
    rcoords<D, DP>(p1, x);
    sp.eval(x);
    rcoords<D, DP>(p2, x);
    sp.eval(x);
    rcoords<D, DP>(p3, x);
    sp.eval(x);
  }
  float acc[RR][DA];
  sp.store(acc);
  float v[32];
#pragma unroll
  for (int r = 0; r < RA; ++r)
#pragma unroll
    for (int k = 0; k < DA; ++k) v[r * DA + k] = acc[r][k];
  res[0] = rs32(v, lane);
#pragma unroll
  for (int e = 0; e < 32; ++e) v[e] = 0.0f;
#pragma unroll
  for (int r = 0; r < RB; ++r)
#pragma unroll
    for (int k = 0; k < DA; ++k) v[r * DA + k] = acc[RA + r][k];
  res[1] = rs32(v, lane);
}

template <int D, int DP, int DA, int KF>
__global__ void __launch_bounds__(kRoundWarps * 32, 1)
    ms_round_kernel(const float* __restrict__ Xs, int n, float* __restrict__ y,
                    int32_t* __restrict__ it, int32_t* __restrict__ conv,
                    int32_t* __restrict__ state, const int32_t* __restrict__ list,
                    const int32_t* __restrict__ S_ptr, int32_t* hist, int target_arg,
                    int max_iter, float tol2_s, unsigned long long* evals,
                    const RoundCtl* __restrict__ rc, float* __restrict__ wlast, float sphere_r) {
  const int target = rc ? rc->target : target_arg;
  constexpr int R = 32 / DA;
  constexpr int SMAX = kSeedsPerCluster;
  constexpr int GMAX = (SMAX + R - 1) / R;
  __shared__ float sy[SMAX][D];
  __shared__ int sit[SMAX];
  __shared__ int sslot[SMAX];
  __shared__ int sact[SMAX];   // 1: takes updates in this round
  __shared__ int alist[SMAX];
  // rank 0's Early-Stopping decisions: sstop[u & 1][i] == u marks seed i as
  // stopped by the count test of update u, unless it converges or fails in
  // that update (written before the update's cluster barrier, read by every
  // rank after it)
  __shared__ int sstop[2][SMAX];
  __shared__ float wb[kRoundWarps][GMAX][32];
  __shared__ float cpart[2][SMAX][DA];   // this CTA's sums (by update parity), read by every rank
  __shared__ float tot[SMAX][DA];
  __shared__ int sA;

  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int ncl = (int)cluster.num_blocks();
  const int q = blockIdx.x / ncl;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // seeds of the round, split evenly over the clusters of the grid (the host
  // only takes this path when S <= clusters * kSeedsPerCluster)
  const int S = *S_ptr;
  const int nclusters = gridDim.x / ncl;
  const int per_cluster = min(SMAX, (S + nclusters - 1) / nclusters);
  const int s0 = q * per_cluster;
  const int ns = max(0, min(per_cluster, S - s0));

  // the cluster's seeds, replicated in every CTA
  for (int i = threadIdx.x; i < ns; i += blockDim.x) {
    const int slot = list[s0 + i];
    sslot[i] = slot;
    sit[i] = it[slot];
    sact[i] = 1;
    sstop[0][i] = -1;
    sstop[1][i] = -1;
#pragma unroll
    for (int k = 0; k < D; ++k) sy[i][k] = y[(int64_t)slot * DP + k];
  }
  // fixed point slices: rank -> [cb, ce), warp -> [wb0, we)
  const int per_cta = ((n + ncl - 1) / ncl + 31) / 32 * 32;
  const int cb = min(n, rank * per_cta), ce = min(n, cb + per_cta);
  const int per_warp = ((ce - cb + kRoundWarps - 1) / kRoundWarps + 31) / 32 * 32;
  const int w0 = min(ce, cb + warp * per_warp), w1 = min(ce, w0 + per_warp);
  __syncthreads();

  for (int guard = 0; guard <= max_iter; ++guard) {
    // rank 0, warp 1: the convergence counts hist[1..32], read now and used
    // after the pass (the load latency hides behind it)
    int hv = 0;
    if (rank == 0 && warp == 1 && lane < max_iter) hv = *((volatile int32_t*)hist + 1 + lane);
    // active list (identical in every CTA: built from replicated state)
    if (warp == 0) {
      int base = 0;
      for (int b0 = 0; b0 < ns; b0 += 32) {
        const int i = b0 + lane;
        const int take = (i < ns) && sact[i];
        const unsigned m = __ballot_sync(kFull, take);
        if (take) alist[base + __popc(m & ((1u << lane) - 1))] = i;
        base += __popc(m);
      }
      if (lane == 0) sA = base;
    }
    __syncthreads();
    const int A = sA;
    if (A == 0) break;
    const int G = (A + R - 1) / R;

    // partial sums of every active seed over this warp's points, one point
    // pass per block of R seeds; a last block of at most R/2 seeds rides in
    // the previous block's pass; a lone block with fewer than R live seeds
    // keeps only the next power of two in registers
    const int last = A - (G - 1) * R;
    const bool pair = G >= 2 && 2 * last <= R && D < 7;   // (D = 7: registers)
    for (int g = 0; g < G; ++g) {
      if (pair && g == G - 2) {
        float res[2];
        if (last > R / 4 && R >= 4) group_pair<D, DP, DA, R, (R >= 4 ? R / 2 : 1), KF>(Xs, w0, w1, lane, alist, g * R, A, sy, res);
        else if (last > 1 && R >= 8) group_pair<D, DP, DA, R, (R >= 8 ? R / 4 : 1), KF>(Xs, w0, w1, lane, alist, g * R, A, sy, res);
        else group_pair<D, DP, DA, R, 1, KF>(Xs, w0, w1, lane, alist, g * R, A, sy, res);
        wb[warp][g][lane] = res[0];
        wb[warp][g + 1][lane] = res[1];
        break;
      }
      const int cnt = min(R, A - g * R);
      float res;
      if (cnt > 8 && R >= 16) res = group_partial<D, DP, DA, (R >= 16 ? 16 : R), KF>(Xs, w0, w1, lane, alist, g * R, A, sy);
      else if (cnt > 4 && R >= 8) res = group_partial<D, DP, DA, (R >= 8 ? 8 : R), KF>(Xs, w0, w1, lane, alist, g * R, A, sy);
      else if (cnt > 2 && R >= 4) res = group_partial<D, DP, DA, (R >= 4 ? 4 : R), KF>(Xs, w0, w1, lane, alist, g * R, A, sy);
      else if (cnt > 1) res = group_partial<D, DP, DA, 2, KF>(Xs, w0, w1, lane, alist, g * R, A, sy);
      else res = group_partial<D, DP, DA, 1, KF>(Xs, w0, w1, lane, alist, g * R, A, sy);
      wb[warp][g][lane] = res;
    }
    const int par = guard & 1;
    if (rank == 0 && warp == 1) {
      // count test of this update: a seed that will have made t updates and
      // has not converged by then is past t* once count(t) = sum_{u <= t}
      // hist[u] >= target.  count from the values read above (a count read
      // earlier can only be smaller, so a stop can come late, never early)
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y2 = __shfl_up_sync(kFull, hv, o);
        if (lane >= o) hv += y2;
      }
      const int c32 = __shfl_sync(kFull, hv, 31);
      for (int a0 = 0; a0 < A; a0 += 32) {
        const int a = a0 + lane;
        const int i = alist[min(a, A - 1)];
        const int t = sit[i] + 1;
        int c = __shfl_sync(kFull, hv, min(t, 32) - 1);
        if (a < A && t > 32) {
          c = c32;
          for (int u = 33; u <= min(t, max_iter); ++u) c += *((volatile int32_t*)hist + u);
        }
        if (a < A && c >= target) sstop[par][i] = guard;
      }
    }
    __syncthreads();
    // this CTA's sums, warps in order
    for (int t = threadIdx.x; t < G * 32; t += blockDim.x) {
      const int g = t >> 5, l = t & 31;
      float sum = 0.0f;
      for (int w = 0; w < kRoundWarps; ++w) sum += wb[w][g][l];
      const int a = g * R + l / DA;
      if (a < A) cpart[par][a][l % DA] = sum;
    }
    cluster.sync();
    // cluster sums, ranks in order (every CTA computes the same totals); the
    // launch's cluster size is kClusterCtas, so all remote loads are issued
    // before the adds
    for (int t = threadIdx.x; t < A * DA; t += blockDim.x) {
      const int a = t / DA, k = t - a * DA;
      float part[kClusterCtas];
#pragma unroll
      for (int rr = 0; rr < kClusterCtas; ++rr)
        part[rr] = cluster.map_shared_rank(&cpart[par][0][0], rr)[a * DA + k];
      float sum = 0.0f;
#pragma unroll
      for (int rr = 0; rr < kClusterCtas; ++rr) sum += part[rr];
      tot[a][k] = sum;
    }
    __syncthreads();
    // update, convergence test and stop decision of each active seed
    for (int a = threadIdx.x; a < A; a += blockDim.x) {
      const int i = alist[a];
      const float W = tot[a][0];
      bool ok = (W > 0.0f) && isfinite(W);
      float step2 = 0.0f, dl[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        dl[k] = ok ? tot[a][1 + k] / W : 0.0f;
        step2 = fmaf(dl[k], dl[k], step2);
      }
      ok = ok && isfinite(step2);
      if (ok && sphere_r > 0.0f) {
        // cosine metric: the mean scaled back onto the sphere of radius
        // sphere_r; the step is the projected one
        float p[D], nn = 0.0f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          p[k] = sy[i][k] + dl[k];
          nn = fmaf(p[k], p[k], nn);
        }
        const float f = sphere_r / sqrtf(nn);
        step2 = 0.0f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          p[k] *= f;
          const float e = p[k] - sy[i][k];
          step2 = fmaf(e, e, step2);
        }
        ok = nn > 0.0f && isfinite(step2);
        if (ok) {
#pragma unroll
          for (int k = 0; k < D; ++k) sy[i][k] = p[k];
        }
      } else if (ok) {
#pragma unroll
        for (int k = 0; k < D; ++k) sy[i][k] += dl[k];
      }
      const int t = sit[i] + 1;
      sit[i] = t;
      int st = kRunning;
      if (!ok) st = kFailed;
      else if (step2 <= tol2_s) st = kConverged;
      else if (t >= max_iter) st = kExhausted;
      // rank 0's count test of this update stops a seed that is still
      // RUNNING; every rank reads the same decision after the barrier.  A
      // stopped seed stays RUNNING with its update count (a later round may
      // resume it)
      const bool stop = cluster.map_shared_rank(&sstop[par][0], 0)[i] == guard;
      if (st != kRunning || stop) sact[i] = 0;   // decided identically in every rank
      if (rank == 0) {
        const int64_t slot = sslot[i];
#pragma unroll
        for (int k = 0; k < D; ++k) y[slot * DP + k] = sy[i][k];
        // sum w of this update, at the position before its step: the prune's
        // density of a seed whose last update this is
        wlast[slot] = W;
        it[slot] = t;
        if (st == kConverged) {
          conv[slot] = t;
          atomicAdd(hist + t, 1);
        }
        state[slot] = st;
      }
    }
    if (rank == 0 && threadIdx.x == 0) atomicAdd(evals, (unsigned long long)A * (unsigned long long)n);
    __syncthreads();
  }
  // keep this CTA's shared memory alive until no rank can still read it
  cluster.sync();
}

template <int D, int DP, int DA, int KF>
static cudaError_t launch_round_t(const float* Xs, int n, float* y, int32_t* it, int32_t* conv,
                                  int32_t* state, const int32_t* list, const int32_t* S_ptr,
                                  int clusters, int32_t* hist, int target, int max_iter,
                                  float tol2_s, unsigned long long* evals, const RoundCtl* rc,
                                  float* wlast, float sphere_r, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(clusters * kClusterCtas);
  cfg.blockDim = dim3(kRoundWarps * 32);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kClusterCtas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, ms_round_kernel<D, DP, DA, KF>, Xs, n, y, it, conv, state, list,
                            S_ptr, hist, target, max_iter, tol2_s, evals, rc, wlast, sphere_r);
}

template <int D, int DP, int DA>
static int max_clusters_t() {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kClusterCtas);
  cfg.blockDim = dim3(kRoundWarps * 32);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kClusterCtas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int c = 0;
  if (cudaOccupancyMaxActiveClusters(&c, ms_round_kernel<D, DP, DA, kKernelGaussian>, &cfg) !=
      cudaSuccess)
    c = 0;
  return c;
}

int round_max_clusters(int d) {
  static int cache[8] = {0};
  if (d < 1 || d > 7) return 0;
  if (cache[d]) return cache[d];
  int c = 0;
  switch (d) {
    case 1: c = max_clusters_t<1, 4, 2>(); break;
    case 2: c = max_clusters_t<2, 4, 4>(); break;
    case 3: c = max_clusters_t<3, 4, 4>(); break;
    case 4: c = max_clusters_t<4, 4, 8>(); break;
    case 5: c = max_clusters_t<5, 8, 8>(); break;
    case 6: c = max_clusters_t<6, 8, 8>(); break;
    case 7: c = max_clusters_t<7, 8, 8>(); break;
  }
  cache[d] = c > 0 ? c : -1;
  return c;
}

cudaError_t launch_ms_round(const float* Xs, int64_t n, int d, float* y, int32_t* it,
                            int32_t* conv, int32_t* state, const int32_t* list,
                            const int32_t* S_ptr, int clusters, int32_t* hist, int target,
                            int max_iter, float tol2_s, unsigned long long* evals,
                            float* wlast, cudaStream_t st, int kf, const RoundCtl* rc,
                            float sphere_r) {
#define FMS_ROUND(D_, DP_, DA_)                                                                \
  return kf ? launch_round_t<D_, DP_, DA_, 1>(Xs, (int)n, y, it, conv, state, list, S_ptr,     \
                                              clusters, hist, target, max_iter, tol2_s, evals, \
                                              rc, wlast, sphere_r, st)                                          \
            : launch_round_t<D_, DP_, DA_, 0>(Xs, (int)n, y, it, conv, state, list, S_ptr,     \
                                              clusters, hist, target, max_iter, tol2_s, evals, \
                                              rc, wlast, sphere_r, st)
  switch (d) {
    case 1: FMS_ROUND(1, 4, 2);
    case 2: FMS_ROUND(2, 4, 4);
    case 3: FMS_ROUND(3, 4, 4);
    case 4: FMS_ROUND(4, 4, 8);
    case 5: FMS_ROUND(5, 8, 8);
    case 6: FMS_ROUND(6, 8, 8);
    case 7: FMS_ROUND(7, 8, 8);
  }
#undef FMS_ROUND
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// ms_refine: the merged modes take more updates with FP64 positions, on the
// same cluster decomposition.  Each CTA keeps ym (FP64) and yf = fl32(ym) of
// its cluster's modes in shared memory; warps evaluate the FP32 partials
// against yf over their fixed sub-slices (exactly as in ms_round); the warp
// sums are combined in FP64 across warps and across ranks; then
//   ym <- ym + S/W - (ym - yf)   (= m(yf))
// and a mode stops once ||step|| <= tol (FP64) or after max_iter updates.
// The density that orders the second prune is W = sum_j w_j of the mode's
// last update, i.e. at the position one step (<= tol) before the refined
// mode; the density is stationary there, so the difference is O(tol^2)
// relative, far below the FP32 weights' rounding.  Partial buffers are
// double-buffered, so one cluster barrier per update suffices.
// ---------------------------------------------------------------------------
template <int D, int DP, int DA, int KF>
__global__ void __launch_bounds__(kRoundWarps * 32, 1)
    ms_refine_kernel(const float* __restrict__ Xs, int n, const float* __restrict__ y,
                     const int32_t* __restrict__ kept, const int32_t* __restrict__ accepted,
                     const int32_t* __restrict__ M_ptr, double* __restrict__ ym,
                     float* __restrict__ yf, double* __restrict__ mscore, double tol2_s,
                     int max_iter, int32_t* iters_out, unsigned long long* evals,
                     double sphere_r) {
  constexpr int R = 32 / DA;
  constexpr int SMAX = kModesPerCluster;
  constexpr int GMAX = (SMAX + R - 1) / R;
  __shared__ float sy[SMAX][D];
  __shared__ double sym[SMAX][D];
  __shared__ int sact[SMAX];
  __shared__ int alist[SMAX];
  __shared__ float wb[kRoundWarps][GMAX][32];
  __shared__ double cpart[2][SMAX][DA];
  __shared__ double tot[SMAX][DA];
  __shared__ int sA;

  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int ncl = (int)cluster.num_blocks();
  const int q = blockIdx.x / ncl;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int M = *M_ptr;
  const int nclusters = gridDim.x / ncl;
  const int per_cluster = min(SMAX, (M + nclusters - 1) / nclusters);
  const int s0 = q * per_cluster;
  const int ns = max(0, min(per_cluster, M - s0));
  for (int i = threadIdx.x; i < ns; i += blockDim.x) {
    const int64_t src = kept[accepted[s0 + i]];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float v = y[src * DP + k];
      sy[i][k] = v;
      sym[i][k] = (double)v;
    }
    sact[i] = 1;
  }
  const int per_cta = ((n + ncl - 1) / ncl + 31) / 32 * 32;
  const int cb = min(n, rank * per_cta), ce = min(n, cb + per_cta);
  const int per_warp = ((ce - cb + kRoundWarps - 1) / kRoundWarps + 31) / 32 * 32;
  const int w0 = min(ce, cb + warp * per_warp), w1 = min(ce, w0 + per_warp);
  __syncthreads();

  int iters = 0;
  for (int pass = 0; pass < max_iter; ++pass) {
    if (warp == 0) {
      int base = 0;
      for (int b0 = 0; b0 < ns; b0 += 32) {
        const int i = b0 + lane;
        const int take = (i < ns) && sact[i];
        const unsigned m = __ballot_sync(kFull, take);
        if (take) alist[base + __popc(m & ((1u << lane) - 1))] = i;
        base += __popc(m);
      }
      if (lane == 0) sA = base;
    }
    __syncthreads();
    const int A = sA;
    if (A == 0) break;   // every mode has stopped
    const int G = (A + R - 1) / R;
    for (int g = 0; g < G; ++g) {
      const int cnt = min(R, A - g * R);
      float res;
      if (cnt > 8 && R >= 16) res = group_partial<D, DP, DA, (R >= 16 ? 16 : R), KF>(Xs, w0, w1, lane, alist, g * R, A, sy);
      else if (cnt > 4 && R >= 8) res = group_partial<D, DP, DA, (R >= 8 ? 8 : R), KF>(Xs, w0, w1, lane, alist, g * R, A, sy);
      else if (cnt > 2 && R >= 4) res = group_partial<D, DP, DA, (R >= 4 ? 4 : R), KF>(Xs, w0, w1, lane, alist, g * R, A, sy);
      else if (cnt > 1) res = group_partial<D, DP, DA, 2, KF>(Xs, w0, w1, lane, alist, g * R, A, sy);
      else res = group_partial<D, DP, DA, 1, KF>(Xs, w0, w1, lane, alist, g * R, A, sy);
      wb[warp][g][lane] = res;
    }
    __syncthreads();
    const int buf = pass & 1;
    for (int t = threadIdx.x; t < G * 32; t += blockDim.x) {
      const int g = t >> 5, l = t & 31;
      double sum = 0.0;
      for (int w = 0; w < kRoundWarps; ++w) sum += (double)wb[w][g][l];
      const int a = g * R + l / DA;
      if (a < A) cpart[buf][a][l % DA] = sum;
    }
    cluster.sync();
    for (int t = threadIdx.x; t < A * DA; t += blockDim.x) {
      const int a = t / DA, k = t - a * DA;
      double part[kClusterCtas];
#pragma unroll
      for (int rr = 0; rr < kClusterCtas; ++rr)
        part[rr] = cluster.map_shared_rank(&cpart[buf][0][0], rr)[a * DA + k];
      double sum = 0.0;
#pragma unroll
      for (int rr = 0; rr < kClusterCtas; ++rr) sum += part[rr];
      tot[a][k] = sum;
    }
    __syncthreads();
    if (rank == 0 && threadIdx.x == 0 && A > 0)
      atomicAdd(evals, (unsigned long long)A * (unsigned long long)n);
    ++iters;
    for (int a = threadIdx.x; a < A; a += blockDim.x) {
      const int i = alist[a];
      const double W = tot[a][0];
      // the density recorded for the mode: sum w at the position of its last
      // update (the step from there is <= the refinement tolerance, and at a
      // stationary point of the density that moves it by O(step^2))
      if (rank == 0) mscore[s0 + i] = W;
      bool ok = W > 0.0 && isfinite(W);
      double step2 = 0.0, dl[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        dl[k] = ok ? tot[a][1 + k] / W - (sym[i][k] - (double)sy[i][k]) : 0.0;
        step2 += dl[k] * dl[k];
      }
      if (ok && sphere_r > 0.0) {
        // cosine metric: project the FP64 position onto the sphere
        double p[D], nn = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          p[k] = sym[i][k] + dl[k];
          nn += p[k] * p[k];
        }
        const double f = sphere_r / sqrt(nn);
        step2 = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          p[k] *= f;
          dl[k] = p[k] - sym[i][k];
          step2 += dl[k] * dl[k];
        }
        ok = nn > 0.0 && isfinite(step2);
        if (ok) {
#pragma unroll
          for (int k = 0; k < D; ++k) {
            sym[i][k] = p[k];
            sy[i][k] = (float)p[k];
          }
        }
      } else if (ok) {
#pragma unroll
        for (int k = 0; k < D; ++k) {
          sym[i][k] += dl[k];
          sy[i][k] = (float)sym[i][k];
        }
      }
      if (!ok || step2 <= tol2_s) sact[i] = 0;
    }
    __syncthreads();
  }
  if (rank == 0) {
    for (int e = threadIdx.x; e < ns * D; e += blockDim.x) {
      const int i = e / D, k = e - i * D;
      ym[(int64_t)(s0 + i) * DP + k] = sym[i][k];
      yf[(int64_t)(s0 + i) * DP + k] = sy[i][k];
    }
    if (threadIdx.x == 0 && ns > 0) atomicMax(iters_out, iters);
  }
  cluster.sync();
}

template <int D, int DP, int DA, int KF>
static cudaError_t launch_refine_t(const float* Xs, int n, const float* y, const int32_t* kept,
                                   const int32_t* accepted, const int32_t* M_ptr, int clusters,
                                   double* ym, float* yf, double* mscore, double tol2_s,
                                   int max_iter, int32_t* iters_out, unsigned long long* evals,
                                   double sphere_r, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(clusters * kClusterCtas);
  cfg.blockDim = dim3(kRoundWarps * 32);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kClusterCtas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, ms_refine_kernel<D, DP, DA, KF>, Xs, n, y, kept, accepted, M_ptr,
                            ym, yf, mscore, tol2_s, max_iter, iters_out, evals, sphere_r);
}

cudaError_t launch_ms_refine(const float* Xs, int64_t n, int d, const float* y,
                             const int32_t* kept, const int32_t* accepted, const int32_t* M_ptr,
                             int clusters, double* ym, float* yf, double* mscore, double tol2_s,
                             int max_iter, int32_t* iters_out, unsigned long long* evals,
                             cudaStream_t st, int kf, double sphere_r) {
  switch (d) {
    case 1: return kf ? launch_refine_t<1, 4, 2, 1>(Xs, (int)n, y, kept, accepted, M_ptr, clusters, ym, yf, mscore, tol2_s, max_iter, iters_out, evals, sphere_r, st)
                 : launch_refine_t<1, 4, 2, 0>(Xs, (int)n, y, kept, accepted, M_ptr, clusters, ym, yf, mscore, tol2_s, max_iter, iters_out, evals, sphere_r, st);
    case 2: return kf ? launch_refine_t<2, 4, 4, 1>(Xs, (int)n, y, kept, accepted, M_ptr, clusters, ym, yf, mscore, tol2_s, max_iter, iters_out, evals, sphere_r, st)
                 : launch_refine_t<2, 4, 4, 0>(Xs, (int)n, y, kept, accepted, M_ptr, clusters, ym, yf, mscore, tol2_s, max_iter, iters_out, evals, sphere_r, st);
    case 3: return kf ? launch_refine_t<3, 4, 4, 1>(Xs, (int)n, y, kept, accepted, M_ptr, clusters, ym, yf, mscore, tol2_s, max_iter, iters_out, evals, sphere_r, st)
                 : launch_refine_t<3, 4, 4, 0>(Xs, (int)n, y, kept, accepted, M_ptr, clusters, ym, yf, mscore, tol2_s, max_iter, iters_out, evals, sphere_r, st);
    case 4: return kf ? launch_refine_t<4, 4, 8, 1>(Xs, (int)n, y, kept, accepted, M_ptr, clusters, ym, yf, mscore, tol2_s, max_iter, iters_out, evals, sphere_r, st)
                 : launch_refine_t<4, 4, 8, 0>(Xs, (int)n, y, kept, accepted, M_ptr, clusters, ym, yf, mscore, tol2_s, max_iter, iters_out, evals, sphere_r, st);
    case 5: return kf ? launch_refine_t<5, 8, 8, 1>(Xs, (int)n, y, kept, accepted, M_ptr, clusters, ym, yf, mscore, tol2_s, max_iter, iters_out, evals, sphere_r, st)
                 : launch_refine_t<5, 8, 8, 0>(Xs, (int)n, y, kept, accepted, M_ptr, clusters, ym, yf, mscore, tol2_s, max_iter, iters_out, evals, sphere_r, st);
    case 6: return kf ? launch_refine_t<6, 8, 8, 1>(Xs, (int)n, y, kept, accepted, M_ptr, clusters, ym, yf, mscore, tol2_s, max_iter, iters_out, evals, sphere_r, st)
                 : launch_refine_t<6, 8, 8, 0>(Xs, (int)n, y, kept, accepted, M_ptr, clusters, ym, yf, mscore, tol2_s, max_iter, iters_out, evals, sphere_r, st);
    case 7: return kf ? launch_refine_t<7, 8, 8, 1>(Xs, (int)n, y, kept, accepted, M_ptr, clusters, ym, yf, mscore, tol2_s, max_iter, iters_out, evals, sphere_r, st)
                 : launch_refine_t<7, 8, 8, 0>(Xs, (int)n, y, kept, accepted, M_ptr, clusters, ym, yf, mscore, tol2_s, max_iter, iters_out, evals, sphere_r, st);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Round bookkeeping.  round_list: the RUNNING seeds (they take part in the
// round), in slot order.  round_finish: t* from the histogram; the kept list
// (converged by t*), counters for the prune.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
    round_list_kernel(const int32_t* __restrict__ state, int N_arg, int32_t* __restrict__ list,
                      int32_t* S_out, const RoundCtl* __restrict__ rc) {
  __shared__ int scratch[64];
  const int N = rc ? rc->N : N_arg;
  int base = 0;
  for (int b = 0; b < N; b += blockDim.x) {
    const int i = b + threadIdx.x;
    const int take = (i < N) && state[i] == kRunning;
    int tot;
    const int off = block_exclusive_scan(take, &tot, scratch);
    if (take) list[base + off] = i;
    base += tot;
  }
  if (threadIdx.x == 0) *S_out = base;
}

cudaError_t launch_round_list(const int32_t* state, int N, int32_t* list, int32_t* S_out,
                              cudaStream_t st, const RoundCtl* rc) {
  round_list_kernel<<<1, 1024, 0, st>>>(state, N, list, S_out, rc);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(1024)
    round_finish_kernel(const int32_t* __restrict__ hist, int target_arg, int max_iter,
                        const int32_t* __restrict__ state, const int32_t* __restrict__ conv,
                        int N_arg, int keep_exhausted, int32_t* __restrict__ kept, MergeCtl* mctl,
                        IterCtl* ctl, int64_t n, int32_t R, Tiling tl,
                        const RoundCtl* __restrict__ rc, const float* __restrict__ wlast,
                        float* __restrict__ score) {
  __shared__ int scratch[64];
  const int target = rc ? rc->target : target_arg;
  const int N = rc ? rc->N : N_arg;
  // t* = the first update r whose cumulative convergence count reaches the
  // target (max_iter if none does): the histogram is read by the whole block
  // and scanned, so its entries are loaded in parallel
  __shared__ int sh_t;
  if (threadIdx.x == 0) sh_t = target <= 0 ? 1 : max_iter;
  __syncthreads();
  if (target > 0) {
    int carry = 0;
    for (int b0 = 1; b0 <= max_iter; b0 += blockDim.x) {
      const int r = b0 + threadIdx.x;
      const int v = r <= max_iter ? hist[r] : 0;
      int tot;
      const int inc = carry + block_exclusive_scan(v, &tot, scratch) + v;
      // counts are non-negative, so exactly one r crosses the target
      if (r <= max_iter && inc >= target && inc - v < target) sh_t = r;
      carry += tot;
      if (carry >= target) break;   // block-uniform
    }
    __syncthreads();
  }
  const int t_star = sh_t;
  int base = 0, convd = 0;
  for (int b = 0; b < N; b += blockDim.x) {
    const int i = b + threadIdx.x;
    int take = 0;
    if (i < N) {
      const int st = state[i];
      const int ok = st == kConverged && conv[i] <= t_star;
      convd += ok;
      take = keep_exhausted ? (st == kConverged || st == kExhausted) : ok;
    }
    int tot;
    const int off = block_exclusive_scan(take, &tot, scratch);
    if (take) {
      kept[base + off] = i;
      if (wlast) score[base + off] = wlast[i];
    }
    base += tot;
  }
  convd = block_sum(convd, scratch);
  if (threadIdx.x == 0) {
    mctl->K = base;
    mctl->t_star = t_star;
    int C, Lc;
    choose_chunks(n, base, R, tl, &C, &Lc);
    mctl->C = C;
    mctl->Lc = Lc;
    if (!wlast) mctl->evals += (int64_t)base * n;   // the density pass the host then runs
    ctl->N = N;
    ctl->r = t_star;
    ctl->n_converged = convd;
    ctl->done = 1;
    ctl->s = 0;
    ctl->steps += t_star;
  }
}

cudaError_t launch_round_finish(const int32_t* hist, int target, int max_iter,
                                const int32_t* state, const int32_t* conv, int N,
                                int keep_exhausted, int32_t* kept, MergeCtl* mctl, IterCtl* ctl,
                                int64_t n, int32_t R, Tiling tl, cudaStream_t st,
                                const RoundCtl* rc, const float* wlast, float* score) {
  round_finish_kernel<<<1, 1024, 0, st>>>(hist, target, max_iter, state, conv, N, keep_exhausted,
                                          kept, mctl, ctl, n, R, tl, rc, wlast, score);
  return cudaGetLastError();
}

}  // namespace fms
