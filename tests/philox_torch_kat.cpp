// Known-answer source for the Philox pin: PyTorch's own header-only
// Philox4x32-10 engine (ATen/core/PhiloxRNGEngine.h), an implementation
// written independently of this project.  Reads lines "c0 c1 c2 c3 k0 k1"
// (decimal) on stdin and prints the four output words of each counter.
// The engine's counter is (offset lo, offset hi, subsequence lo, subsequence
// hi) and its key is (seed lo, seed hi); its first four draws are the four
// words of one block.
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdint>
#include <cstdio>

int main() {
  unsigned long long c0, c1, c2, c3, k0, k1;
  while (std::scanf("%llu %llu %llu %llu %llu %llu", &c0, &c1, &c2, &c3, &k0, &k1) == 6) {
    uint64_t seed = (uint64_t)k0 | ((uint64_t)k1 << 32);
    uint64_t subseq = (uint64_t)c2 | ((uint64_t)c3 << 32);
    uint64_t offset = (uint64_t)c0 | ((uint64_t)c1 << 32);
    at::philox_engine eng(seed, subseq, offset);
    uint32_t a = eng(), b = eng(), c = eng(), d = eng();
    std::printf("%u %u %u %u\n", a, b, c, d);
  }
  return 0;
}
