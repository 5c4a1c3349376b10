// Device body of the sorted prune, shared by the single-set and batched kernels.
#pragma once

#include "fms_internal.cuh"

namespace fms {

// Same prune with the candidates in shared memory, in two parallel stages:
// (1) the block sorts the candidates by (score descending, rank ascending)
// with a bitonic sort; (2) one warp walks the sorted list 32 candidates at a
// time: the batch's coordinates are staged in a transposed, padded tile
// (one candidate per lane, conflict-free per-lane reads), every lane tests its
// candidate against the modes accepted so far, and the survivors of a batch
// are resolved in order (the lowest surviving lane is accepted and removes
// the later lanes within r).  The accepted set and its order are those of the
// one-by-one greedy visit.  With acc_in_smem the accepted modes' coordinates
// are kept in shared memory, else read back from global memory (all lanes
// read the same row).
constexpr int kPruneTileStride = 33;   // padded row of the transposed batch tile
constexpr int kPruneMaxDim = 64;

template <typename PT, typename ST>
__host__ __device__ inline size_t greedy_sorted_smem(int K, int d, int P, bool acc_in_smem) {
  return (((size_t)P * (sizeof(ST) + 4) + 15) / 16) * 16 +
         (size_t)kPruneMaxDim * kPruneTileStride * sizeof(PT) +
         (acc_in_smem ? (size_t)K * d * sizeof(PT) : 0);
}

template <typename PT, typename ST>
__device__ void greedy_sorted_body(const int32_t* __restrict__ cand_row, const int K,
                                   const ST* __restrict__ score, const PT* __restrict__ pos,
                                   int DP, int d, PT r2, int32_t* __restrict__ accepted,
                                   int32_t* __restrict__ M_out, int P, unsigned char* smem,
                                   bool acc_in_smem = true) {
  // layout: keys[P] (ST), idx[P] (int), ctile[64 x 33] (PT), [apos[K*d] (PT)]
  ST* keys = reinterpret_cast<ST*>(smem);
  int* idx = reinterpret_cast<int*>(keys + P);
  PT* ctile = reinterpret_cast<PT*>(smem + (((size_t)P * (sizeof(ST) + 4) + 15) / 16) * 16);
  PT* apos = ctile + kPruneMaxDim * kPruneTileStride;
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
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  auto row_of = [&](int q) -> int64_t { return cand_row ? (int64_t)cand_row[q] : (int64_t)q; };
  // coordinates of accepted mode a (a candidate index in accepted[a])
  auto acc_ptr = [&](int a) -> const PT* {
    if (acc_in_smem) return apos + (size_t)a * d;
    return pos + row_of(accepted[a]) * DP;
  };
  int nacc = 0;
  for (int base = 0; base < K; base += 32) {
    // stage the batch: lane c loads sorted candidate base + c (independent
    // loads in flight across lanes); ctile[k * 33 + c] = its coordinate k
    const int i = base + lane;
    if (i < K) {
      const PT* src = pos + row_of(idx[i]) * DP;
      for (int k = 0; k < d; ++k) ctile[k * kPruneTileStride + lane] = src[k];
    }
    __syncwarp();
    bool alive = i < K;
    for (int a = 0; a < nacc && __any_sync(kFull, alive); ++a) {
      if (alive) {
        const PT* ap = acc_ptr(a);
        PT d2 = 0;
        for (int k = 0; k < d; ++k) {
          const PT e = ctile[k * kPruneTileStride + lane] - ap[k];
          d2 += e * e;
        }
        if (d2 < r2) alive = false;
      }
    }
    for (;;) {
      const unsigned m = __ballot_sync(kFull, alive);
      if (!m) break;
      const int w = __ffs(m) - 1;
      if (lane == w) accepted[nacc] = idx[i];
      if (acc_in_smem)
        for (int k = lane; k < d; k += 32)
          apos[(size_t)nacc * d + k] = ctile[k * kPruneTileStride + w];
      __syncwarp();
      const PT* wp = acc_ptr(nacc);
      ++nacc;
      if (alive) {
        if (lane == w) {
          alive = false;
        } else {
          PT d2 = 0;
          for (int k = 0; k < d; ++k) {
            const PT e = ctile[k * kPruneTileStride + lane] - wp[k];
            d2 += e * e;
          }
          if (d2 < r2) alive = false;
        }
      }
    }
    __syncwarp();   // the tile is rewritten by the next batch
  }
  if (lane == 0) *M_out = nacc;
}

}  // namespace fms
