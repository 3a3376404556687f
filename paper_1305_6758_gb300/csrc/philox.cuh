// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel
// random numbers: as easy as 1, 2, 3", SC'11), written for the device.
//
// One call maps a 128-bit counter and a 64-bit key to 128 random bits.  Each
// of the ten rounds takes the 32x32->64 products of words 0 and 2 with two
// fixed odd multipliers, swaps the halves into the next state and mixes in the
// other two words and the round key; the key advances by two Weyl constants
// between rounds.  The paper under implementation does not name its generator;
// a counter-based one lets every (path, sweep, site) draw its numbers with no
// stored state, so results do not depend on the launch shape.
#pragma once
#include <cstdint>

namespace mpk {

struct Philox4 {
  uint32_t x, y, z, w;
};

constexpr uint32_t kPhiloxMulA = 0xD2511F53u, kPhiloxMulB = 0xCD9E8D57u;
constexpr uint32_t kPhiloxWeylA = 0x9E3779B9u, kPhiloxWeylB = 0xBB67AE85u;

// The ten round keys of a 64-bit key: (k0 + r*WeylA, k1 + r*WeylB), r = 0..9.
// Computed once on the host and passed as kernel parameters, so that each
// round's key is a constant-memory operand instead of two per-thread adds.
struct PhiloxKeys {
  uint32_t k0[10];
  uint32_t k1[10];
};

inline PhiloxKeys philox_round_keys(uint64_t seed) {
  PhiloxKeys k{};
  uint32_t a = static_cast<uint32_t>(seed & 0xffffffffu), b = static_cast<uint32_t>(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    k.k0[r] = a;
    k.k1[r] = b;
    a += kPhiloxWeylA;
    b += kPhiloxWeylB;
  }
  return k;
}

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                 uint32_t c3, const PhiloxKeys& key) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint64_t pa = static_cast<uint64_t>(kPhiloxMulA) * c0;
    const uint64_t pb = static_cast<uint64_t>(kPhiloxMulB) * c2;
    const uint32_t n0 = static_cast<uint32_t>(pb >> 32) ^ c1 ^ key.k0[round];
    const uint32_t n2 = static_cast<uint32_t>(pa >> 32) ^ c3 ^ key.k1[round];
    c1 = static_cast<uint32_t>(pb);
    c3 = static_cast<uint32_t>(pa);
    c0 = n0;
    c2 = n2;
  }
  return Philox4{c0, c1, c2, c3};
}

// Round 1 of counters that differ only in word 0 (the site): the product of
// word 2 and everything mixed with it depend on words 1..3 and the key alone,
// so a loop over the sites of a sweep computes them once.
struct PhiloxPrefix {
  uint32_t x0, x1, c3k;
};

__device__ __forceinline__ PhiloxPrefix philox_prefix(uint32_t c1, uint32_t c2, uint32_t c3,
                                                      const PhiloxKeys& key) {
  const uint64_t pb = static_cast<uint64_t>(kPhiloxMulB) * c2;
  return PhiloxPrefix{static_cast<uint32_t>(pb >> 32) ^ c1 ^ key.k0[0], static_cast<uint32_t>(pb),
                      c3 ^ key.k1[0]};
}

// philox4x32_10(c0, c1, c2, c3, key) with round 1's fixed part precomputed.
__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, const PhiloxPrefix& pre,
                                                 const PhiloxKeys& key) {
  const uint64_t pa0 = static_cast<uint64_t>(kPhiloxMulA) * c0;
  uint32_t x0 = pre.x0, x1 = pre.x1;
  uint32_t x2 = static_cast<uint32_t>(pa0 >> 32) ^ pre.c3k, x3 = static_cast<uint32_t>(pa0);
#pragma unroll
  for (int round = 1; round < 10; ++round) {
    const uint64_t pa = static_cast<uint64_t>(kPhiloxMulA) * x0;
    const uint64_t pb = static_cast<uint64_t>(kPhiloxMulB) * x2;
    const uint32_t n0 = static_cast<uint32_t>(pb >> 32) ^ x1 ^ key.k0[round];
    const uint32_t n2 = static_cast<uint32_t>(pa >> 32) ^ x3 ^ key.k1[round];
    x1 = static_cast<uint32_t>(pb);
    x3 = static_cast<uint32_t>(pa);
    x0 = n0;
    x2 = n2;
  }
  return Philox4{x0, x1, x2, x3};
}

}  // namespace mpk
