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

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                 uint32_t c3, uint32_t k0, uint32_t k1) {
  constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
  constexpr uint32_t kWeylA = 0x9E3779B9u, kWeylB = 0xBB67AE85u;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint64_t pa = static_cast<uint64_t>(kMulA) * c0;
    const uint64_t pb = static_cast<uint64_t>(kMulB) * c2;
    const uint32_t n0 = static_cast<uint32_t>(pb >> 32) ^ c1 ^ k0;
    const uint32_t n2 = static_cast<uint32_t>(pa >> 32) ^ c3 ^ k1;
    c1 = static_cast<uint32_t>(pb);
    c3 = static_cast<uint32_t>(pa);
    c0 = n0;
    c2 = n2;
    k0 += kWeylA;
    k1 += kWeylB;
  }
  return Philox4{c0, c1, c2, c3};
}

}  // namespace mpk
