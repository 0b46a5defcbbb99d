// Counter-based random words for the sweep kernels.
//
// Philox4x32-10 as defined by Salmon, Moraes, Dror and Shaw ("Parallel random
// numbers: as easy as 1, 2, 3", SC'11): ten rounds, each multiplying counter
// words 0 and 2 by two fixed odd constants (32x32 -> 64 bits), exchanging and
// xoring the halves with the other counter words and the round key; the round
// key advances by two Weyl increments between rounds. The sweeps only consume
// output word 0, so the last round's other words are left to dead-code
// elimination.
#pragma once

#include <cstdint>

namespace isingx {

struct PhiloxKey {
  uint32_t lo, hi;
};

__host__ __device__ inline PhiloxKey philox_key(uint64_t seed, uint32_t instance) {
  PhiloxKey k;
  k.lo = static_cast<uint32_t>(seed);
  k.hi = static_cast<uint32_t>(seed >> 32) ^ (instance * 0x9E3779B9u);
  return k;
}

__device__ __forceinline__ uint32_t philox4x32_10_word0(uint32_t x0, uint32_t x1, uint32_t x2,
                                                         uint32_t x3, PhiloxKey key) {
  uint32_t ka = key.lo, kb = key.hi;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t a_lo = 0xD2511F53u * x0;
    const uint32_t a_hi = __umulhi(0xD2511F53u, x0);
    const uint32_t b_lo = 0xCD9E8D57u * x2;
    const uint32_t b_hi = __umulhi(0xCD9E8D57u, x2);
    x0 = b_hi ^ x1 ^ ka;
    x1 = b_lo;
    x2 = a_hi ^ x3 ^ kb;
    x3 = a_lo;
    ka += 0x9E3779B9u;
    kb += 0xBB67AE85u;
  }
  return x0;
}

}  // namespace isingx
