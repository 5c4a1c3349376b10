// Device body of the sorted prune, shared by the single-set and batched kernels.
#pragma once

#include "fms_internal.cuh"

namespace fms {

// Same prune with the candidates in shared memory, in two parallel stages:
// (1) the block sorts the candidates by (score descending, rank ascending)
// with a bitonic sort; (2) one warp walks the sorted list 32 candidates at a
// time: every lane tests its candidate against the modes accepted so far, and
// the survivors of a batch are resolved in order (the lowest surviving lane is
// accepted and removes the later lanes within r).  The accepted set and its
// order are those of the one-by-one greedy visit.
template <typename PT, typename ST>
__device__ void greedy_sorted_body(const int32_t* __restrict__ cand_row, const int K,
                                   const ST* __restrict__ score, const PT* __restrict__ pos,
                                   int DP, int d, PT r2, int32_t* __restrict__ accepted,
                                   int32_t* __restrict__ M_out, int P, unsigned char* smem) {
  // layout: keys[P] (ST), idx[P] (int), spos[K*d] (PT, sorted order), apos[K*d] (PT)
  ST* keys = reinterpret_cast<ST*>(smem);
  int* idx = reinterpret_cast<int*>(keys + P);
  PT* spos = reinterpret_cast<PT*>(smem + (((size_t)P * (sizeof(ST) + 4) + 15) / 16) * 16);
  PT* apos = spos + (size_t)K * d;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    keys[i] = i < K ? score[i] : (ST)-INFINITY;
    idx[i] = i < K ? i : INT32_MAX;
  }
  __syncthreads();
  // bitonic sort: "a before b" iff a.key > b.key, or equal keys and a.idx < b.idx
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const ST ka = keys[i], kb = keys[l];
          const int ia = idx[i], ib = idx[l];
          const bool a_first = (ka > kb) || (ka == kb && ia < ib);
          const bool up = (i & k) == 0;
          if (up != a_first) {
            keys[i] = kb;
            keys[l] = ka;
            idx[i] = ib;
            idx[l] = ia;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int e = threadIdx.x; e < K * d; e += blockDim.x) {
    const int i = e / d, k = e - i * d;
    const int q = idx[i];
    const int64_t row = cand_row ? cand_row[q] : q;
    spos[e] = pos[row * DP + k];
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  int nacc = 0;
  for (int base = 0; base < K; base += 32) {
    const int i = base + lane;
    bool alive = i < K;
    const PT* cp = spos + (size_t)(alive ? i : 0) * d;
    for (int a = 0; a < nacc && __any_sync(kFull, alive); ++a) {
      if (alive) {
        const PT* ap = apos + (size_t)a * d;
        PT d2 = 0;
        for (int k = 0; k < d; ++k) {
          const PT e = cp[k] - ap[k];
          d2 += e * e;
        }
        if (d2 < r2) alive = false;
      }
    }
    for (;;) {
      const unsigned m = __ballot_sync(kFull, alive);
      if (!m) break;
      const int w = __ffs(m) - 1;
      if (lane == w) {
        accepted[nacc] = idx[i];
        for (int k = 0; k < d; ++k) apos[(size_t)nacc * d + k] = cp[k];
      }
      __syncwarp();
      const PT* wp = apos + (size_t)nacc * d;
      ++nacc;
      if (alive) {
        if (lane == w) {
          alive = false;
        } else {
          PT d2 = 0;
          for (int k = 0; k < d; ++k) {
            const PT e = cp[k] - wp[k];
            d2 += e * e;
          }
          if (d2 < r2) alive = false;
        }
      }
    }
  }
  if (lane == 0) *M_out = nacc;
}

}  // namespace fms
