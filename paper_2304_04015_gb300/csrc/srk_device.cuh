// Device-side building blocks of the walk kernels (sm_103a).
//
// Philox4x32-10 is restated from its defining paper (Salmon, Moraes, Dror,
// Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds,
// each multiplying counter words 0 and 2 by 0xD2511F53 and 0xCD9E8D57 into
// 64-bit products, then
//   x0' = hi(M1 x2) ^ x1 ^ k0,  x1' = lo(M1 x2),
//   x2' = hi(M0 x0) ^ x3 ^ k1,  x3' = lo(M0 x0),
// with the key advanced by the Weyl constants 0x9E3779B9 and 0xBB67AE85
// after every round.  The key is launch-uniform, so the ten round keys are
// computed once per thread.
#pragma once
#include <stdint.h>

namespace srk {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

struct RoundKeys {
  uint32_t k0[10];
  uint32_t k1[10];
};

__device__ __forceinline__ RoundKeys round_keys(uint32_t key0, uint32_t key1) {
  RoundKeys rk;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    rk.k0[r] = key0 + (uint32_t)r * kPhiloxW0;
    rk.k1[r] = key1 + (uint32_t)r * kPhiloxW1;
  }
  return rk;
}

// One Philox4x32-10 block: counter (c0..c3) -> 128 random bits in (x0..x3).
__device__ __forceinline__ void philox(const RoundKeys &rk, uint32_t c0,
                                       uint32_t c1, uint32_t c2, uint32_t c3,
                                       uint32_t &x0, uint32_t &x1,
                                       uint32_t &x2, uint32_t &x3) {
  x0 = c0; x1 = c1; x2 = c2; x3 = c3;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(kPhiloxM0, x0), lo0 = kPhiloxM0 * x0;
    const uint32_t hi1 = __umulhi(kPhiloxM1, x2), lo1 = kPhiloxM1 * x2;
    const uint32_t y0 = hi1 ^ x1 ^ rk.k0[r];
    const uint32_t y2 = hi0 ^ x3 ^ rk.k1[r];
    x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
  }
}

// floor(R * d / 2^64) for a 64-bit draw R = (hi:lo) and 0 < d < 2^32: a
// uniform index in [0, d).  R*d = hi*d*2^32 + lo*d, and adding the fraction
// of lo*d/2^32 cannot carry past a multiple of 2^32, so
// floor(R*d/2^64) = (hi*d + floor(lo*d/2^32)) >> 32.
__device__ __forceinline__ uint32_t draw_index(uint32_t hi, uint32_t lo,
                                               uint32_t d) {
  const uint64_t t = (uint64_t)hi * d + __umulhi(lo, d);
  return (uint32_t)(t >> 32);
}

// Stratum (walk length) of walk index r: the l with P[l] <= r < P[l+1],
// for a prefix array P[0..L+1] held in shared memory.
__device__ __forceinline__ int stratum_of(const int32_t *P, int L, int32_t r) {
  int lo = 0, hi = L;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P[mid] <= r) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace srk
