// Device body of the sorted prune, shared by the single-set and batched kernels.
#pragma once

#include "fms_internal.cuh"

namespace fms {

// Same prune with the candidates in shared memory, in two parallel stages:
// (1) the block sorts the candidates by (score descending, rank ascending):
// up to 512 candidates by counting, for each, the candidates ordered before
// it (FP32 scores as one packed 64-bit key comparison per pair), else with a
// bitonic sort; (2) the sorted list is walked 32 candidates at a time, one
// candidate per lane.  Register visit (d = DT known at compile time, the
// candidates' coordinates preloaded into shared memory): every warp holds the
// batch in registers, tests it against its share of the modes accepted so
// far and computes one member's neighbour mask by shuffles; warp 0 accepts
// the survivors lowest lane first with those masks.  Block visit
// (any d): the batch is staged in a transposed, padded tile (conflict-free
// per-lane reads; two tiles, warp 1 stages the next batch while the current
// one is tested), every warp tests it against its share of the accepted
// modes, warp v records which batch members lie within r of member v (a
// 32-bit mask), and warp 0 resolves the survivors in order with those masks.
// Both use the distance of the test against an accepted mode for every
// suppression, so the accepted set and its order are those of the one-by-one
// greedy visit.  With acc_in_smem the accepted modes' coordinates are kept in
// shared memory, else read back from global memory (all lanes read the same
// row).
constexpr int kPruneTileStride = 33;   // padded row of the transposed batch tile
constexpr int kPruneMaxDim = 64;

// Bytes of the sort keys, indices and 96 scratch ints (batch flags, count,
// the batch's neighbour masks).
constexpr int kPruneScratchInts = 96;
template <typename ST>
__host__ __device__ inline size_t greedy_keys_bytes(int P) {
  return (((size_t)P * (sizeof(ST) + 4) + kPruneScratchInts * 4 + 15) / 16) * 16;
}

// preload: every candidate's coordinates are copied to shared memory once,
// before the sort (P x d values, transposed), so that staging a batch reads
// shared memory instead of two dependent global loads per batch.
template <typename PT, typename ST>
__host__ __device__ inline size_t greedy_sorted_smem(int K, int d, int P, bool acc_in_smem,
                                                     bool preload = false) {
  return greedy_keys_bytes<ST>(P) +
         2 * (size_t)kPruneMaxDim * kPruneTileStride * sizeof(PT) +
         (preload ? (size_t)P * d * sizeof(PT) : 0) +
         (acc_in_smem ? (size_t)K * d * sizeof(PT) : 0);
}

// ---------------------------------------------------------------------------
// The greedy visit for candidate sets too large for the sorted prune's shared
// memory: repeatedly accept the remaining candidate of highest (score, lowest
// index) and drop every candidate within r of it.  The remaining candidates
// are kept as a compacted list (in `list`, K entries of global memory); one
// pass per accepted mode drops the new mode's neighbours and finds the next
// winner, each thread taking kGlobalRun list entries per step with their loads
// issued together.  The winner and every suppression are decided exactly as
// in the one-by-one visit, so the accepted set and order are the same.
// Candidate q has rank q; its row is cand_row[q] (or q when cand_row is
// null).  `sm` holds greedy_global_smem() bytes of shared memory.
// ---------------------------------------------------------------------------
constexpr int kGlobalRun = 8;

template <typename ST>
__device__ __forceinline__ void argmax_merge(ST& best, int& bq, ST os, int oq) {
  if (os > best || (os == best && oq < bq)) {
    best = os;
    bq = oq;
  }
}

// Block-wide (score desc, index asc) winner; INT32_MAX when no candidate
// has a comparable score.  Every thread returns the same value.
template <typename ST>
__device__ int block_argmax(ST best, int bq, ST* sh_s, int* sh_q, int* sh_best) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const ST os = __shfl_xor_sync(kFull, best, o);
    const int oq = __shfl_xor_sync(kFull, bq, o);
    argmax_merge<ST>(best, bq, os, oq);
  }
  if (lane == 0) {
    sh_s[wid] = best;
    sh_q[wid] = bq;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ST b = sh_s[0];
    int bb = sh_q[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) argmax_merge<ST>(b, bb, sh_s[w], sh_q[w]);
    *sh_best = bb;
  }
  __syncthreads();
  const int win = *sh_best;
  __syncthreads();   // sh_best and sh_s / sh_q are reused by the next call
  return win;
}

// shared memory of greedy_global_body: winner scores and indices per warp,
// the winner's coordinates, the winner, the scan's warp sums
template <typename PT, typename ST>
__host__ __device__ constexpr size_t greedy_global_smem() {
  return 32 * sizeof(ST) + 32 * 4 + kPruneMaxDim * sizeof(PT) + 16 + 64 * 4;
}

template <typename PT, typename ST>
__device__ void greedy_global_body(const int32_t* __restrict__ cand_row, const int K,
                                   const ST* __restrict__ score, const PT* __restrict__ pos,
                                   int DP, int d, PT r2, int32_t* __restrict__ list,
                                   int32_t* __restrict__ accepted, int32_t* __restrict__ M_out,
                                   unsigned char* sm) {
  ST* sh_s = reinterpret_cast<ST*>(sm);
  int* sh_q = reinterpret_cast<int*>(sh_s + 32);
  PT* sh_pos = reinterpret_cast<PT*>(sh_q + 32);
  int* sh_best = reinterpret_cast<int*>(sh_pos + kPruneMaxDim);
  int* scratch = sh_best + 4;
  const int T = blockDim.x;
  ST best = (ST)-INFINITY;
  int bq = INT32_MAX;
  for (int b = 0; b < K; b += T * kGlobalRun) {
#pragma unroll
    for (int v = 0; v < kGlobalRun; ++v) {
      const int q = b + v * T + threadIdx.x;
      if (q < K) {
        list[q] = q;
        argmax_merge<ST>(best, bq, score[q], q);
      }
    }
  }
  int win = block_argmax<ST>(best, bq, sh_s, sh_q, sh_best);
  int len = K, M = 0;
  while (win != INT32_MAX) {
    if (threadIdx.x == 0) accepted[M] = win;
    ++M;
    const int64_t wrow = cand_row ? cand_row[win] : win;
    for (int k = threadIdx.x; k < d; k += T) sh_pos[k] = pos[wrow * DP + k];
    __syncthreads();
    best = (ST)-INFINITY;
    bq = INT32_MAX;
    int newlen = 0;
    for (int b = 0; b < len; b += T * kGlobalRun) {
      int q[kGlobalRun];
      int64_t row[kGlobalRun];
      ST sc[kGlobalRun];
      PT d2[kGlobalRun];
#pragma unroll
      for (int v = 0; v < kGlobalRun; ++v) {
        const int idx = b + v * T + threadIdx.x;
        q[v] = idx < len ? list[idx] : -1;
      }
#pragma unroll
      for (int v = 0; v < kGlobalRun; ++v) {
        sc[v] = q[v] >= 0 ? score[q[v]] : (ST)0;
        row[v] = q[v] >= 0 ? (cand_row ? (int64_t)cand_row[q[v]] : (int64_t)q[v]) : 0;
        d2[v] = 0;
      }
      for (int k = 0; k < d; ++k) {
        const PT pk = sh_pos[k];
#pragma unroll
        for (int v = 0; v < kGlobalRun; ++v) {
          if (q[v] >= 0) {
            const PT e = pos[row[v] * DP + k] - pk;
            d2[v] += e * e;
          }
        }
      }
      unsigned keep = 0;
      int cnt = 0;
#pragma unroll
      for (int v = 0; v < kGlobalRun; ++v) {
        if (q[v] >= 0 && q[v] != win && !(d2[v] < r2)) {
          keep |= 1u << v;
          ++cnt;
          argmax_merge<ST>(best, bq, sc[v], q[v]);
        }
      }
      // in-place compaction: this step writes only below the end of what it
      // read, and every read precedes the scan's barriers
      int tot;
      int off = block_exclusive_scan(cnt, &tot, scratch);
#pragma unroll
      for (int v = 0; v < kGlobalRun; ++v)
        if ((keep >> v) & 1u) list[newlen + off++] = q[v];
      newlen += tot;
    }
    len = newlen;
    win = block_argmax<ST>(best, bq, sh_s, sh_q, sh_best);
  }
  if (threadIdx.x == 0) *M_out = M;
}

template <typename PT, typename ST, int DT = 0>
__device__ void greedy_sorted_body(const int32_t* __restrict__ cand_row, const int K,
                                   const ST* __restrict__ score, const PT* __restrict__ pos,
                                   int DP, int d, PT r2, int32_t* __restrict__ accepted,
                                   int32_t* __restrict__ M_out, int P, unsigned char* smem,
                                   bool acc_in_smem = true, bool preload = false) {
  // layout: keys[P] (ST), idx[P] (int), scratch[96] (int), ctile[2][64 x 33] (PT),
  // [cpre[d][P] (PT)], [apos[K*d] (PT)]
  ST* keys = reinterpret_cast<ST*>(smem);
  int* idx = reinterpret_cast<int*>(keys + P);
  PT* ctile2 = reinterpret_cast<PT*>(smem + greedy_keys_bytes<ST>(P));
  constexpr int kTile = kPruneMaxDim * kPruneTileStride;
  PT* cpre = ctile2 + 2 * kTile;
  PT* apos = cpre + (preload ? (size_t)P * d : 0);
  auto row_of = [&](int q) -> int64_t { return cand_row ? (int64_t)cand_row[q] : (int64_t)q; };
  if (preload)   // read by stage() after the sort's barriers
    for (int t = threadIdx.x; t < K; t += blockDim.x) {
      const PT* src = pos + row_of(t) * DP;
      for (int k = 0; k < d; ++k) cpre[(size_t)k * P + t] = src[k];
    }
  // order: "a before b" iff a.key > b.key, or equal keys and a.idx < b.idx
  if (sizeof(ST) == 4 && K <= 512 && K <= (int)blockDim.x) {
    // FP32 scores: (score, index) packed into one 64-bit key whose unsigned
    // order is the visit order (score bits mapped to an unsigned order, the
    // complemented index below them), so the rank count is one comparison
    // per pair; the keys occupy the keys + idx region until the ranks are known
    unsigned long long* vk = reinterpret_cast<unsigned long long*>(smem);
    const int t = threadIdx.x;
    unsigned long long mv = 0;
    if (t < K) {
      float f = (float)score[t];
      if (!(f == f)) f = -INFINITY;   // a NaN score counts as -inf
      if (f == 0.0f) f = 0.0f;        // -0 and +0 are equal scores
      unsigned u = __float_as_uint(f);
      u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
      mv = ((unsigned long long)u << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)t);
      vk[t] = mv;
    }
    __syncthreads();
    int rank = 0;
    if (t < K) {
      int j = 0;
      for (; j + 8 <= K; j += 8) {
        unsigned long long kk[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) kk[u] = vk[j + u];
#pragma unroll
        for (int u = 0; u < 8; ++u) rank += kk[u] > mv ? 1 : 0;
      }
      for (; j < K; ++j) rank += vk[j] > mv ? 1 : 0;
    }
    __syncthreads();
    if (t < K) idx[rank] = t;
    __syncthreads();   // the sorted order is read by other threads below
  } else if (K <= 512 && K <= (int)blockDim.x) {
    // rank of candidate t = number of candidates before it (a permutation:
    // the order is total; a NaN score counts as -inf)
    const int t = threadIdx.x;
    ST mk = (ST)-INFINITY;
    if (t < K) {
      mk = score[t];
      if (!(mk == mk)) mk = (ST)-INFINITY;
      keys[t] = mk;
    }
    __syncthreads();
    int rank = 0;
    if (t < K) {
      // eight independent (broadcast) loads in flight per step
      int j = 0;
      for (; j + 8 <= K; j += 8) {
        ST kk[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) kk[u] = keys[j + u];
#pragma unroll
        for (int u = 0; u < 8; ++u) rank += (kk[u] > mk || (kk[u] == mk && j + u < t)) ? 1 : 0;
      }
      for (; j < K; ++j) {
        const ST kj = keys[j];
        rank += (kj > mk || (kj == mk && j < t)) ? 1 : 0;
      }
    }
    __syncthreads();
    if (t < K) {
      keys[rank] = mk;
      idx[rank] = t;
    }
    __syncthreads();   // the sorted order is read by other threads below
  } else {
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    keys[i] = i < K ? score[i] : (ST)-INFINITY;
    idx[i] = i < K ? i : INT32_MAX;
  }
  __syncthreads();
  // bitonic sort
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
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  // coordinates of accepted mode a (a candidate index in accepted[a])
  auto acc_ptr = [&](int a) -> const PT* {
    if (acc_in_smem) return apos + (size_t)a * d;
    return pos + row_of(accepted[a]) * DP;
  };
  int* s_dead = idx + P;                             // scratch: batch suppression flags
  int* s_nacc = s_dead + 32;                         // scratch: modes accepted so far
  unsigned* s_near = reinterpret_cast<unsigned*>(s_dead + 64);   // scratch: batch masks
  // warp w stages batch `base` (lane c: sorted candidate base + c; tile[k * 33 + c] is
  // its coordinate k)
  auto stage = [&](int base, PT* tile) {
    const int i = base + lane;
    if (i < K) {
      const int c = idx[i];
      if (preload) {
        for (int k = 0; k < d; ++k) tile[k * kPruneTileStride + lane] = cpre[(size_t)k * P + c];
      } else {
        const PT* src = pos + row_of(c) * DP;
        for (int k = 0; k < d; ++k) tile[k * kPruneTileStride + lane] = src[k];
      }
    }
  };
  if constexpr (DT > 0) {
    if (preload && acc_in_smem) {
      // Register visit (d = DT known at compile time): every warp holds the
      // batch's coordinates in registers (lane c: sorted candidate base + c),
      // tests them against its share of the modes accepted so far, and warp v
      // records which members lie within r of member v (shuffles and a
      // ballot); warp 0 then accepts the survivors lowest lane first, each
      // removing its neighbours by mask, and the accepted lanes write their
      // rows in parallel.  The distances are those of the test against an
      // accepted mode, so the accepted set and its order are the greedy
      // visit's.
      if (threadIdx.x == 0) *s_nacc = 0;
      if (warp == 0) s_dead[lane] = 0;
      for (int base = 0; base < K; base += 32) {
        const int i = base + lane;
        const int c = i < K ? idx[i] : 0;
        PT x[DT];
#pragma unroll
        for (int k = 0; k < DT; ++k) x[k] = i < K ? cpre[(size_t)k * P + c] : (PT)0;
        __syncthreads();   // accepted rows, their count and cleared flags are visible
        const int nacc = *s_nacc;
        bool dead = false;
        if (i < K)
          for (int a = warp; a < nacc && !dead; a += nwarps) {
            const PT* ap = apos + (size_t)a * DT;
            PT d2 = 0;
#pragma unroll
            for (int k = 0; k < DT; ++k) {
              const PT e = x[k] - ap[k];
              d2 += e * e;
            }
            dead = d2 < r2;
          }
        if (dead) s_dead[lane] = 1;
        // warp v: the batch members within r of member v (bit l of s_near[v])
        for (int v = warp; v < 32; v += nwarps) {
          PT d2 = 0;
#pragma unroll
          for (int k = 0; k < DT; ++k) {
            const PT e = x[k] - __shfl_sync(kFull, x[k], v);
            d2 += e * e;
          }
          const unsigned m = __ballot_sync(kFull, i < K && d2 < r2);
          if (lane == 0) s_near[v] = m;
        }
        __syncthreads();
        if (warp == 0) {
          // survivors accepted lowest lane first, each removing its neighbours;
          // then every accepted lane writes its own row
          unsigned alive = __ballot_sync(kFull, i < K && !s_dead[lane]);
          unsigned acc = 0;
          while (alive) {
            const int w = __ffs(alive) - 1;
            acc |= 1u << w;
            alive &= ~(s_near[w] | (1u << w));
          }
          if ((acc >> lane) & 1u) {
            const int at = nacc + __popc(acc & ((1u << lane) - 1u));
            accepted[at] = c;
#pragma unroll
            for (int k = 0; k < DT; ++k) apos[(size_t)at * DT + k] = x[k];
          }
          s_dead[lane] = 0;
          if (lane == 0) *s_nacc = nacc + __popc(acc);
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) *M_out = *s_nacc;
      return;
    }
  }
  if (threadIdx.x == 0) *s_nacc = 0;
  if (warp == 0) {
    stage(0, ctile2);
    s_dead[lane] = 0;
  }
  for (int base = 0, b = 0; base < K; base += 32, ++b) {
    const int i = base + lane;
    PT* ctile = ctile2 + (b & 1) * kTile;
    __syncthreads();   // this batch's tile and cleared flags are visible
    const int nacc = *s_nacc;
    // every warp tests the batch against its share of the modes accepted so far
    if (i < K) {
      bool dead = false;
      for (int a = warp; a < nacc && !dead; a += nwarps) {
        const PT* ap = acc_ptr(a);
        PT d2 = 0;
        for (int k = 0; k < d; ++k) {
          const PT e = ctile[k * kPruneTileStride + lane] - ap[k];
          d2 += e * e;
        }
        dead = d2 < r2;
      }
      if (dead) s_dead[lane] = 1;
    }
    // masks: bit l of s_near[v] <=> batch members l and v lie within r (the
    // same FP arithmetic as the test against an accepted mode: the coordinate
    // differences are exact negations of each other)
    for (int v = warp; v < 32; v += nwarps) {
      bool nb = false;
      if (i < K && base + v < K) {
        PT d2 = 0;
        for (int k = 0; k < d; ++k) {
          const PT e = ctile[k * kPruneTileStride + lane] - ctile[k * kPruneTileStride + v];
          d2 += e * e;
        }
        nb = d2 < r2;
      }
      const unsigned m = __ballot_sync(kFull, nb);
      if (lane == 0) s_near[v] = m;
    }
    // the next batch's tile (its last readers finished before this batch's barrier)
    if (warp == (nwarps > 1 ? 1 : 0) && base + 32 < K) stage(base + 32, ctile2 + ((b + 1) & 1) * kTile);
    __syncthreads();
    if (warp == 0) {
      // survivors of the batch, resolved in order by one warp
      unsigned alive = __ballot_sync(kFull, i < K && !s_dead[lane]);
      int na = nacc;
      while (alive) {
        const int w = __ffs(alive) - 1;
        if (lane == w) accepted[na] = idx[i];
        if (acc_in_smem)
          for (int k = lane; k < d; k += 32)
            apos[(size_t)na * d + k] = ctile[k * kPruneTileStride + w];
        alive &= ~(s_near[w] | (1u << w));
        ++na;
      }
      s_dead[lane] = 0;
      if (lane == 0) *s_nacc = na;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *M_out = *s_nacc;
}

}  // namespace fms
