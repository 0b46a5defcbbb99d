// Counter-based random words for the sweep kernels.
//
// Philox4x32-10 as defined by Salmon, Moraes, Dror and Shaw ("Parallel random
// numbers: as easy as 1, 2, 3", SC'11): ten rounds, each multiplying counter
// words 0 and 2 by two fixed odd constants (32x32 -> 64 bits), exchanging and
// xoring the halves with the other counter words and the round key; the round
// key advances by two Weyl increments between rounds. A flip or initial-spin
// draw of vertex o is word o mod 4 of the counter (o / 4, t, replica, stream),
// so four vertices share one evaluation (vertex_word); where only word 0 is
// used, the last round's other words are left to dead-code elimination.
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

// The ten round keys of a key, computed once per launch and passed as kernel
// parameters so that the per-draw rounds read them as constants.
struct PhiloxRounds {
  uint32_t lo[10], hi[10];
};

__host__ __device__ inline PhiloxRounds philox_rounds(PhiloxKey k) {
  PhiloxRounds r;
  uint32_t a = k.lo, b = k.hi;
  for (int i = 0; i < 10; ++i) {
    r.lo[i] = a;
    r.hi[i] = b;
    a += 0x9E3779B9u;
    b += 0xBB67AE85u;
  }
  return r;
}

// Word 0 of Philox4x32-10 for counter (x0, x1, x2, x3). Each round is two
// 32x32 -> 64 products and two three-way xors.
__device__ __forceinline__ uint32_t philox4x32_10_word0(uint32_t x0, uint32_t x1, uint32_t x2,
                                                         uint32_t x3, const PhiloxRounds& rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t pa = static_cast<uint64_t>(0xD2511F53u) * x0;
    const uint64_t pb = static_cast<uint64_t>(0xCD9E8D57u) * x2;
    const uint32_t n0 = static_cast<uint32_t>(pb >> 32) ^ x1 ^ rk.lo[r];
    const uint32_t n2 = static_cast<uint32_t>(pa >> 32) ^ x3 ^ rk.hi[r];
    x1 = static_cast<uint32_t>(pb);
    x3 = static_cast<uint32_t>(pa);
    x0 = n0;
    x2 = n2;
  }
  return x0;
}

// All four words of Philox4x32-10 for counter (x0, x1, x2, x3).
__device__ __forceinline__ uint4 philox4x32_10(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3,
                                               const PhiloxRounds& rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t pa = static_cast<uint64_t>(0xD2511F53u) * x0;
    const uint64_t pb = static_cast<uint64_t>(0xCD9E8D57u) * x2;
    const uint32_t n0 = static_cast<uint32_t>(pb >> 32) ^ x1 ^ rk.lo[r];
    const uint32_t n2 = static_cast<uint32_t>(pa >> 32) ^ x3 ^ rk.hi[r];
    x1 = static_cast<uint32_t>(pb);
    x3 = static_cast<uint32_t>(pa);
    x0 = n0;
    x2 = n2;
  }
  return make_uint4(x0, x1, x2, x3);
}

// The draw of vertex o (original id) in sweep t of replica r on stream s (0
// flips, 1 initial spins): word o mod 4 of counter (o / 4, t, r, s), so the
// four vertices 4q .. 4q + 3 share one evaluation.
// The last round's words 0 and 1 come from one product (B * x2) and words 2
// and 3 from the other (A * x0), so only the product the wanted word needs
// is formed there.
__device__ __forceinline__ uint32_t vertex_word(uint32_t o, uint32_t t, uint32_t replica,
                                                uint32_t stream, const PhiloxRounds& rk) {
  uint32_t x0 = o >> 2, x1 = t, x2 = replica, x3 = stream;
#pragma unroll
  for (int r = 0; r < 9; ++r) {
    const uint64_t pa = static_cast<uint64_t>(0xD2511F53u) * x0;
    const uint64_t pb = static_cast<uint64_t>(0xCD9E8D57u) * x2;
    const uint32_t n0 = static_cast<uint32_t>(pb >> 32) ^ x1 ^ rk.lo[r];
    const uint32_t n2 = static_cast<uint32_t>(pa >> 32) ^ x3 ^ rk.hi[r];
    x1 = static_cast<uint32_t>(pb);
    x3 = static_cast<uint32_t>(pa);
    x0 = n0;
    x2 = n2;
  }
  const uint32_t k = o & 3u;
  const bool low_pair = k < 2u;  // words 0, 1: B * x2; words 2, 3: A * x0
  const uint64_t prod = static_cast<uint64_t>(low_pair ? 0xCD9E8D57u : 0xD2511F53u) * (low_pair ? x2 : x0);
  if (k & 1u) return static_cast<uint32_t>(prod);
  return static_cast<uint32_t>(prod >> 32) ^ (low_pair ? (x1 ^ rk.lo[9]) : (x3 ^ rk.hi[9]));
}

}  // namespace isingx
