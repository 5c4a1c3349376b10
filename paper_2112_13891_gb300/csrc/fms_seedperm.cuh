// The keyed permutation behind Seed Selection (Alg. 2: N of the n points
// chosen evenly at random), shared by every kernel that draws seeds so that
// the single-set and batched paths produce the same seeds bit for bit.
//
// Entry r of the permutation of [0, n): a balanced Feistel network on 2*hb
// bits (4^hb >= n), whose round function is the SplitMix64 output function of
// (round key XOR right half) truncated to hb bits, cycle-walked into [0, n)
// (Black & Rogaway 2002).  The six round keys are SplitMix64 outputs 0..5 of
// the stream seeded with the caller's rng_seed.
#pragma once

#include <stdint.h>

namespace fms {

// SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014).
__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct FeistelKey {
  uint64_t k[6];
  int hb;   // half width: the network permutes [0, 4^hb)
};

// smallest hb >= 1 with 4^hb >= n
__host__ __device__ inline int feistel_half_bits(int64_t n) {
  int hb = 1;
  while ((int64_t(1) << (2 * hb)) < n) ++hb;
  return hb;
}

inline FeistelKey make_key(int64_t n, uint64_t rng_seed) {
  FeistelKey f;
  for (int r = 0; r < 6; ++r) f.k[r] = mix64(rng_seed + (uint64_t)(r + 1) * 0x9E3779B97F4A7C15ull);
  f.hb = feistel_half_bits(n);
  return f;
}

__device__ __forceinline__ uint64_t feistel(uint64_t x, const FeistelKey& f) {
  const uint64_t mask = (uint64_t(1) << f.hb) - 1;
  uint64_t L = x >> f.hb, R = x & mask;
#pragma unroll
  for (int r = 0; r < 6; ++r) {
    const uint64_t nl = R;
    R = L ^ (mix64(f.k[r] ^ R) & mask);
    L = nl;
  }
  return (L << f.hb) | R;
}

// Entry r of the permutation of [0, n) (f.hb must be feistel_half_bits(n)).
__device__ __forceinline__ int64_t permute(int64_t r, int64_t n, const FeistelKey& f) {
  uint64_t x = feistel((uint64_t)r, f);
  // cycle walking: the walk stays on r's cycle of the bijection of [0, 4^hb)
  // and that cycle contains r < n, so it ends within 4^hb steps
  while (x >= (uint64_t)n) x = feistel(x, f);
  return (int64_t)x;
}

}  // namespace fms
