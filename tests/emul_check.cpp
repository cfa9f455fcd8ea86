// Host build of the library's integer-emulated step-2 product (zig_emul.h)
// for the CPU test: out[k] = bits of RN(m[k] 2^-52 x[k]) by the emulation.
#include <stdint.h>

#include "zig_emul.h"

extern "C" void emul_batch(const uint64_t* m, const uint64_t* xbits, uint64_t* out, uint64_t n) {
  for (uint64_t k = 0; k < n; ++k) out[k] = zig::emul_u_times_x(m[k], xbits[k]);
}
