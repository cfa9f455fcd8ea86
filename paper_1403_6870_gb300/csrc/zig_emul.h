// zig_emul.h -- step 2 of Table 1 (McFarland, arXiv:1403.6870) for FP64
// outputs without the FP64 pipe: RN(U X_i) formed from integers.
//
// U = m 2^-52 (m the 52-bit integer of the word split) and X_i a positive
// normal binary64 with 53-bit significand sig, so U X_i = m sig 2^(E - 1127)
// with E the biased exponent of X_i.  The product m sig is exact in 105
// bits; rounding it to 53 bits, nearest with ties to even, is the IEEE
// product RN(U X_i), the value the fused multiply-add fma(1 + U, X, -X)
// returns.  GB300 runs two FP64 fused multiply-adds per clock per SM, so a
// kernel bound by that pipe can send part of its outputs through this
// integer form (four 32x32->64 multiplies and shifts) instead.
//
// Written for both host and device so that the CPU checks it bit for bit
// against the host's IEEE multiplication.
#ifndef ZIG_EMUL_H
#define ZIG_EMUL_H

#include <stdint.h>

#if defined(__CUDACC__)
#define ZIG_HD __host__ __device__ __forceinline__
#else
#define ZIG_HD inline
#endif

namespace zig {

ZIG_HD int emul_clz64(uint64_t v) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)v);
#else
  return v ? __builtin_clzll(v) : 64;
#endif
}

// Bits of RN(m 2^-52 x) for 0 <= m < 2^52 and x = the binary64 with bits
// xbits, a normal number whose product with U stays normal (|x| >= 2^-960
// suffices).  The sign of x is kept; m = 0 gives +0 for either sign (as
// fma(1 + U, x, -x) does).
ZIG_HD uint64_t emul_u_times_x(uint64_t m, uint64_t xbits) {
  if (m == 0) return 0;
  const int k = emul_clz64(m) - 12;       // m << k in [2^51, 2^52)
  const uint64_t mp = m << k;
  const uint64_t sig = (xbits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int E = (int)(xbits >> 52) & 0x7FF;
  // P = mp sig in [2^103, 2^105), from 32-bit limbs
  const uint32_t a0 = (uint32_t)mp, a1 = (uint32_t)(mp >> 32);
  const uint32_t b0 = (uint32_t)sig, b1 = (uint32_t)(sig >> 32);
  const uint64_t p00 = (uint64_t)a0 * b0;
  const uint64_t mid = (uint64_t)a0 * b1 + (uint64_t)a1 * b0;  // < 2^54
  const uint64_t p11 = (uint64_t)a1 * b1;                      // < 2^41
  const uint64_t lo = p00 + (mid << 32);
  const uint64_t hi = p11 + (mid >> 32) + (lo < p00 ? 1u : 0u);  // P >> 64 in [2^39, 2^41)
  // keep 53 bits: s = 51 or 52 low bits of P go to the rounding
  const int top = (int)(hi >> 40);
  const int s = 51 + top;
  uint64_t mant = (hi << (13 - top)) | (lo >> s);  // in [2^52, 2^53)
  const uint64_t rem = lo & ((1ull << s) - 1);
  const uint64_t half = 1ull << (s - 1);
  mant += (rem > half || (rem == half && (mant & 1u))) ? 1u : 0u;
  // value mant 2^(s + E - 1127 - k): biased exponent s + E - 52 - k; adding
  // mant (with its leading 2^52) to (exponent - 1) << 52 carries into the
  // exponent when rounding reached 2^53
  const uint64_t ex = (uint64_t)(s + E - 52 - k);
  return (xbits & 0x8000000000000000ull) | (((ex - 1) << 52) + mant);
}

}  // namespace zig

#endif
