// Independent Philox4x32-10 reference for the oracle's pin: reads lines
// "seed g attempt domain" and prints the four 32-bit outputs of PyTorch's
// host Philox engine for counter (g_lo, g_hi, domain, attempt) and key
// (seed_lo, seed_hi).  The engine maps (seed, subsequence, offset) onto
// key = seed, counter words 2,3 = subsequence and counter words 0,1 = offset.
#include <ATen/core/PhiloxRNGEngine.h>
#include <cinttypes>
#include <cstdio>

int main() {
  unsigned long long seed, g, a, dom;
  while (std::scanf("%llu %llu %llu %llu", &seed, &g, &a, &dom) == 4) {
    at::philox_engine eng(seed, ((uint64_t)a << 32) | (dom & 0xFFFFFFFFull), g);
    uint32_t r0 = eng(), r1 = eng(), r2 = eng(), r3 = eng();
    std::printf("%u %u %u %u\n", r0, r1, r2, r3);
  }
  return 0;
}
