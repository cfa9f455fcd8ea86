/* Search for counters whose packed-keying FP32 first word (32-bit output
 * g & 3 of Philox block g >> 2, counter words (h_lo, h_hi, 0, 0)) has a
 * layer index >= L (byte 0) and U = 0 (bits 9-31): fringe draws whose U is
 * zero (with NEG = 1, also the normal's sign bit 8 set).  Uses only the
 * oracle's Philox4x32-10.  Usage: find_packed_zero SEED L NEG START_BLOCK
 * MAX_BLOCKS -> prints the first counter found, or -1. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

int main(int argc, char** argv) {
  if (argc != 6) return 2;
  const uint64_t seed = strtoull(argv[1], NULL, 0);
  const unsigned L = (unsigned)strtoul(argv[2], NULL, 0);
  const unsigned neg = (unsigned)strtoul(argv[3], NULL, 0);
  const uint64_t h0 = strtoull(argv[4], NULL, 0), nb = strtoull(argv[5], NULL, 0);
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (uint64_t h = h0; h < h0 + nb; h++) {
    const uint32_t ctr[4] = {(uint32_t)h, (uint32_t)(h >> 32), 0u, 0u};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    for (int q = 0; q < 4; q++) {
      if ((r[q] & 0xFFu) >= L && (r[q] >> 9) == 0u && (!neg || (r[q] & 0x100u))) {
        printf("%llu\n", (unsigned long long)(4 * h + (uint64_t)q));
        return 0;
      }
    }
  }
  printf("-1\n");
  return 0;
}
