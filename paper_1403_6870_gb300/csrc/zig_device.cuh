// zig_device.cuh -- device-side pieces of the modified ziggurat shared by
// every kernel of the library: the tables, Philox4x32-10, the word stream of
// one counter and the complete sampler of Table 1 (the "general path").
//
// McFarland, arXiv:1403.6870, Table 1 (modified column):
//   1. generate U_1 and i;  2. if i < L_max return U_1 X_i;
//   3. generate j from A;   4. if j = 0 return a value from the tail;
//   5-8. rejection-sample overhang box j.
// Words: from the 64-bit word w, i = bits 0-7, the normal's sign = bit 8,
// U = bits 12-63 as m 2^-52 (FP32: bits 41-63 as m 2^-23); an alias word
// gives column c = bits 0-7 and threshold t = bits 8-63.  With a 10-bit
// index (i_max = 1024): i = bits 0-9, sign = bit 10, column = bits 0-9,
// threshold = bits 10-63.
#ifndef ZIG_DEVICE_CUH
#define ZIG_DEVICE_CUH

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "zig.h"

namespace zig {

// ---------------------------------------------------------------------------
// Device tables (one set per distribution; index = zig_dist) for an index of
// IB bits: i_max = 2^IB slots (8: the paper's 256; 10: the 1024 of
// Appendix D item 1)
// ---------------------------------------------------------------------------
template <int IB>
struct DevTabT {
  static constexpr int kIMax = 1 << IB;
  static constexpr int kBits = IB;
  double X[kIMax];       // X_i; entries beyond L_max are zero (never returned)
  double f[kIMax + 1];   // heights f_0..f_L (normal: unnormalised)
  double dX[kIMax + 1];  // X_{j-1} - X_j
  double df[kIMax + 1];  // f_j - f_{j-1}
  float X32[kIMax];
  float f32[kIMax + 1];
  float dX32[kIMax + 1];
  float df32[kIMax + 1];
  unsigned long long T[kIMax];  // alias thresholds (scale 2^(64 - IB))
  typename std::conditional<(IB <= 8), unsigned char, unsigned short>::type alias[kIMax];
  // per-box bounds on mx + my: under the curve below acc, over it above rej
  // (exponential: acc covers the always-accept region ux + uy < tau)
  unsigned long long acc52[kIMax + 1], rej52[kIMax + 1];
  unsigned int acc23[kIMax + 1], rej23[kIMax + 1];
  double tau;                  // exponential always-accept bound on ux + uy
  double rinv;                 // RN64(1 / X_0)
  float rinv32;
  int L;
};
typedef DevTabT<8> DevTab;

// This header is included by exactly one translation unit (zig_gen.cu),
// which owns the tables and the status word of each device.
__device__ DevTab g_tab[2];
__device__ DevTabT<10> g_tab10[2];
__device__ unsigned int g_status;

template <int IB>
__device__ __forceinline__ const DevTabT<IB>& dev_tab(int dist);
template <>
__device__ __forceinline__ const DevTabT<8>& dev_tab<8>(int dist) {
  return g_tab[dist];
}
template <>
__device__ __forceinline__ const DevTabT<10>& dev_tab<10>(int dist) {
  return g_tab10[dist];
}

constexpr unsigned kLoopLimitBit = 1u << ZIG_E_LOOP_LIMIT;

struct Limits {
  int max_att;
  int max_tail;
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------
constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
constexpr uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;

// The 64-bit product of a round multiplier and a counter word, as two
// 32-bit multiplies (low and high half).  Measured on GB300 against one
// 32x32->64 multiply: +1.8 % per-index FP64, +3.4 % per-index FP32, the
// packed kernels unchanged; a half nobody reads is dropped by the compiler.
__device__ __forceinline__ uint64_t mul_wide(uint32_t m, uint32_t x) {
  uint32_t lo, hi;
  asm("mul.lo.u32 %0, %1, %2;" : "=r"(lo) : "r"(m), "r"(x));
  asm("mul.hi.u32 %0, %1, %2;" : "=r"(hi) : "r"(m), "r"(x));
  return ((uint64_t)hi << 32) | lo;
}

__device__ __forceinline__ uint4 philox10(uint32_t c0, uint32_t c1, uint32_t c2,
                                          uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = mul_wide(kM0, c0);
    const uint64_t p1 = mul_wide(kM1, c2);
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
    k0 += kW0;
    k1 += kW1;
  }
  return make_uint4(c0, c1, c2, c3);
}

// The ten round keys of one Philox key, (k0 + r W0, k1 + r W1).  Passed to
// kernels by value, they live in the constant bank and enter the XORs as
// operands instead of being recomputed per round.
struct RoundKeys {
  uint32_t k0[10];
  uint32_t k1[10];
};

// Rounds 3..10 of Philox4x32-10 given the state after round 2, returning
// only (r0, r1), the first word of a block.
__device__ __forceinline__ uint2 philox_rounds3to10_first(uint32_t c0, uint32_t c1,
                                                          uint32_t c2, uint32_t c3,
                                                          const RoundKeys& rk) {
#pragma unroll
  for (int r = 2; r < 10; ++r) {
    const uint64_t p0 = mul_wide(kM0, c0);
    const uint64_t p1 = mul_wide(kM1, c2);
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ rk.k0[r];
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk.k1[r];
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
  }
  return make_uint2(c0, c1);
}

// Rounds 3..10 given the state after round 2, returning the whole block.
__device__ __forceinline__ uint4 philox_rounds3to10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                    uint32_t c3, const RoundKeys& rk) {
#pragma unroll
  for (int r = 2; r < 10; ++r) {
    const uint64_t p0 = mul_wide(kM0, c0);
    const uint64_t p1 = mul_wide(kM1, c2);
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ rk.k0[r];
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk.k1[r];
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
  }
  return make_uint4(c0, c1, c2, c3);
}

// Full block k of counter g in domain dom (counter word 2) with the round
// keys: dom 0 is the per-index stream, dom 1 the private stream of packed
// keying.
__device__ __forceinline__ uint4 philox_block(uint64_t g, uint32_t k, const RoundKeys& rk,
                                              uint32_t dom = 0u) {
  uint32_t c0 = (uint32_t)g, c1 = (uint32_t)(g >> 32), c2 = dom, c3 = k;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = mul_wide(kM0, c0);
    const uint64_t p1 = mul_wide(kM1, c2);
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ rk.k0[r];
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk.k1[r];
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
  }
  return make_uint4(c0, c1, c2, c3);
}

// Block 0's first word of counter g (attempt 0) with the round keys.
__device__ __forceinline__ uint2 philox_first(uint64_t g, const RoundKeys& rk) {
  uint32_t c0 = (uint32_t)g, c1 = (uint32_t)(g >> 32), c2 = 0u, c3 = 0u;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const uint64_t p0 = mul_wide(kM0, c0);
    const uint64_t p1 = mul_wide(kM1, c2);
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ rk.k0[r];
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk.k1[r];
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
  }
  return philox_rounds3to10_first(c0, c1, c2, c3, rk);
}

__device__ __forceinline__ uint64_t pack(uint32_t lo, uint32_t hi) {
  return (uint64_t)lo | ((uint64_t)hi << 32);
}

// Word stream of one counter g: block k = Philox((g_lo, g_hi, dom, k), key),
// words r0 | r1 << 32 then r2 | r3 << 32.  dom = 0 is the per-index stream.
struct Words {
  uint32_t glo, ghi, dom, k0, k1, blk, r2, r3;
  bool half;
  __device__ Words(uint64_t seed, uint64_t g, uint32_t domain = 0u)
      : glo((uint32_t)g), ghi((uint32_t)(g >> 32)), dom(domain), k0((uint32_t)seed),
        k1((uint32_t)(seed >> 32)), blk(0), r2(0), r3(0), half(false) {}
  __device__ uint64_t next() {
    if (!half) {
      const uint4 r = philox10(glo, ghi, dom, blk, k0, k1);
      r2 = r.z;
      r3 = r.w;
      half = true;
      return pack(r.x, r.y);
    }
    half = false;
    ++blk;
    return pack(r2, r3);
  }
};

// Packed keying (opt-in; ZIG_KEY_PACKED in zig.h): the first word of
// counter g comes from a block shared with its neighbours, FP64: half
// (g & 1) of block (g >> 1, dom 0, attempt 0); FP32: 32-bit output (g & 3)
// of block (g >> 2, ...), L, as the word (L & 0x1FF) | (L >> 9) << 41 (the
// layer index and sign from L's low 9 bits, U from its top 23).  Every later
// word comes from counter g's private stream Words(seed, g, 1).
template <typename T>
__device__ __forceinline__ uint64_t packed_word_of(uint4 b, uint64_t g) {
  if (sizeof(T) == 8) return (g & 1u) ? pack(b.z, b.w) : pack(b.x, b.y);
  const uint32_t q = (uint32_t)g & 3u;
  const uint32_t lane = q == 0 ? b.x : q == 1 ? b.y : q == 2 ? b.z : b.w;
  return (uint64_t)(lane & 0x1FFu) | ((uint64_t)(lane >> 9) << 41);
}

template <typename T>
__device__ __forceinline__ uint64_t packed_first(uint64_t g, const RoundKeys& rk) {
  return packed_word_of<T>(philox_block(g >> (sizeof(T) == 8 ? 1 : 2), 0u, rk), g);
}

template <typename T>
struct PackedWords {
  Words rest;
  uint64_t first;
  bool started;
  __device__ PackedWords(uint64_t seed, uint64_t g) : rest(seed, g, 1u), started(false) {
    const uint64_t h = g >> (sizeof(T) == 8 ? 1 : 2);
    first = packed_word_of<T>(
        philox10((uint32_t)h, (uint32_t)(h >> 32), 0u, 0u, (uint32_t)seed, (uint32_t)(seed >> 32)),
        g);
  }
  __device__ uint64_t next() {
    if (!started) {
      started = true;
      return first;
    }
    return rest.next();
  }
};

// ---------------------------------------------------------------------------
// Precision traits: integer U, its value, table access, explicit rounding
// ---------------------------------------------------------------------------
template <typename T>
struct Prec;

template <>
struct Prec<double> {
  typedef unsigned long long UInt;
  static constexpr int kBits = 52;
  static constexpr UInt kOne = 1ull << 52;
  static __device__ __forceinline__ UInt ubits(uint64_t w) { return w >> 12; }
  // (1 + U) from the integer: exact
  static __device__ __forceinline__ double one_plus(UInt m) {
    return __hiloint2double((int)(0x3FF00000u | (uint32_t)(m >> 32)), (int)(uint32_t)m);
  }
  static __device__ __forceinline__ double val(UInt m) { return __dsub_rn(one_plus(m), 1.0); }
  // The same U = m 2^-52 (m <= 2^52, exact) from integer operations: the
  // leading one of m moved to bit 52 and the exponent added beneath it,
  // which keeps the subtraction off the FP64 pipe.
  static __device__ __forceinline__ double val_int(UInt m) {
    const int lz = __clzll((long long)m);
    const unsigned long long bits =
        (m << ((lz - 11) & 63)) + ((unsigned long long)(1033 - lz) << 52);
    return m == 0 ? 0.0 : __longlong_as_double((long long)bits);
  }
  static __device__ __forceinline__ double fmat(double a, double b, double c) {
    return __fma_rn(a, b, c);
  }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  template <class Tab>
  static __device__ __forceinline__ double X(const Tab& t, int i) { return t.X[i]; }
  template <class Tab>
  static __device__ __forceinline__ double f(const Tab& t, int i) { return t.f[i]; }
  template <class Tab>
  static __device__ __forceinline__ double dX(const Tab& t, int i) { return t.dX[i]; }
  template <class Tab>
  static __device__ __forceinline__ double df(const Tab& t, int i) { return t.df[i]; }
  template <class Tab>
  static __device__ __forceinline__ double rinv(const Tab& t) { return t.rinv; }
  template <class Tab>
  static __device__ __forceinline__ UInt acc(const Tab& t, int j) { return t.acc52[j]; }
  template <class Tab>
  static __device__ __forceinline__ UInt rej(const Tab& t, int j) { return t.rej52[j]; }
  static __device__ __forceinline__ double nan() {
    return __longlong_as_double(0x7FF8000000000000ll);
  }
};

template <>
struct Prec<float> {
  typedef unsigned int UInt;
  static constexpr int kBits = 23;
  static constexpr UInt kOne = 1u << 23;
  static __device__ __forceinline__ UInt ubits(uint64_t w) { return (UInt)(w >> 41); }
  static __device__ __forceinline__ float one_plus(UInt m) {
    return __int_as_float((int)(0x3F800000u | m));
  }
  static __device__ __forceinline__ float val(UInt m) { return __fsub_rn(one_plus(m), 1.0f); }
  static __device__ __forceinline__ float val_int(UInt m) { return val(m); }
  static __device__ __forceinline__ float fmat(float a, float b, float c) {
    return __fmaf_rn(a, b, c);
  }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  template <class Tab>
  static __device__ __forceinline__ float X(const Tab& t, int i) { return t.X32[i]; }
  template <class Tab>
  static __device__ __forceinline__ float f(const Tab& t, int i) { return t.f32[i]; }
  template <class Tab>
  static __device__ __forceinline__ float dX(const Tab& t, int i) { return t.dX32[i]; }
  template <class Tab>
  static __device__ __forceinline__ float df(const Tab& t, int i) { return t.df32[i]; }
  template <class Tab>
  static __device__ __forceinline__ float rinv(const Tab& t) { return t.rinv32; }
  template <class Tab>
  static __device__ __forceinline__ UInt acc(const Tab& t, int j) { return t.acc23[j]; }
  template <class Tab>
  static __device__ __forceinline__ UInt rej(const Tab& t, int j) { return t.rej23[j]; }
  static __device__ __forceinline__ float nan() { return __int_as_float(0x7FC00000); }
};

// Step 3: j from the alias table.
template <class Tab>
__device__ __forceinline__ int alias_pick(const Tab& t, uint64_t w) {
  const int c = (int)(w & (uint64_t)(Tab::kIMax - 1));
  return (w >> Tab::kBits) < t.T[c] ? c : (int)t.alias[c];
}

// FP32 approximation of U from its integer (top 24 bits at most).
template <typename T>
__device__ __forceinline__ float approx_u(typename Prec<T>::UInt m) {
  if (sizeof(T) == 8)
    return __uint2float_rz((uint32_t)((unsigned long long)m >> 28)) * (1.0f / 16777216.0f);
  return __uint2float_rz((uint32_t)m) * (1.0f / 8388608.0f);
}

// Exact rejection test y < exp(-a), decided first in FP32: xa, ya below are
// FP32 approximations of x and y (from the top 24 bits of U and the binary32
// tables) whose combined error, with that of expf (2 ulp), is at most
// 3.0e-6 (< 2^-18) relative in y / exp(-a) for every box of both
// distributions at either table width, by an a-priori bound on each step.
// With a margin of 2^-17 the FP32 answer, when it is given, is the one the
// FP64 test y < exp(-a) would give, so the decision is always that of the
// FP64 test; only points within the margin (about 7e-4 of the normal's
// attempts, 5e-4 of the exponential's) evaluate the FP64 exp.  Each such
// point costs its warp a double-precision exp on the FP64 pipe, which the
// fast path also needs.
constexpr float kPreTestMargin = 1.0f / 131072.0f;

// One attempt inside overhang box j >= 1 at integer uniforms (mx, my)
// (Table 1 steps 6-7).  Exponential: points above the chord are reflected
// through the anti-diagonal into the lower-left triangle (Appendix C item
// 5); below the chord by more than eps they are accepted without a test
// (Sec. 2, three regions); the rest get the exact test y < e^-x.  Normal:
// the exact test y < e^{-x^2/2}.  On accept x = X_j + ux (X_{j-1} - X_j).
// Before the exact test, the box's own bounds on mx + my (zig.h,
// zig_tables_ex) settle points that lie clearly under or over the curve:
// the per-box eps of Appendix D item 2 for the exponential, and for the
// normal the chord test on either side, which sorts the convex boxes
// (x > 1) and the concave ones (x < 1).  They carry a rounding margin, so
// the answer is the exact test's.  kIntU forms U from integers (val_int)
// instead of with an FP64 subtraction; the packed-keying stages use it
// (their kernel is bound by the FP64 pipe), the per-index ones do not (there
// it measured 1 % slower through register allocation).
template <int DIST, typename T, class Tab, bool kIntU = false>
__device__ __forceinline__ bool overhang_attempt(const Tab& t, int j,
                                                 typename Prec<T>::UInt mx,
                                                 typename Prec<T>::UInt my, T& x) {
  typedef Prec<T> P;
  if (DIST == ZIG_EXP) {
    if (mx + my > P::kOne) {
      const typename P::UInt nx = P::kOne - my, ny = P::kOne - mx;
      mx = nx;
      my = ny;
    }
  }
  {
    const typename P::UInt sum = mx + my;
    if (sum < P::acc(t, j)) {
      x = P::fmat((kIntU ? P::val_int(mx) : P::val(mx)), P::dX(t, j), P::X(t, j));
      return true;
    }
    if (DIST != ZIG_EXP && sum > P::rej(t, j)) return false;
  }
  // FP32 view of x and y for the pre-test
  const float ux = approx_u<T>(mx), uy = approx_u<T>(my);
  const float xa = __fmaf_rn(ux, t.dX32[j], t.X32[j]);
  const float ya = __fmaf_rn(uy, t.df32[j], t.f32[j - 1]);
  const float aa = DIST == ZIG_EXP ? xa : 0.5f * xa * xa;
  const float e = expf(-aa);
  if (ya > e * (1.0f + kPreTestMargin)) return false;
  const T xx = P::fmat((kIntU ? P::val_int(mx) : P::val(mx)), P::dX(t, j), P::X(t, j));
  if (ya < e * (1.0f - kPreTestMargin)) {
    x = xx;
    return true;
  }
  const T y = P::fmat((kIntU ? P::val_int(my) : P::val(my)), P::df(t, j), P::f(t, j - 1));
  const double xd = (double)xx;
  const double a = DIST == ZIG_EXP ? xd : __dmul_rn(__dmul_rn(xd, xd), 0.5);
  if ((double)y < exp(-a)) {
    x = xx;
    return true;
  }
  return false;
}

// Full Table 1 for the exponential from word stream w.  Step 4 uses
// memorylessness: a tail draw is X_0 plus a fresh exponential, evaluated
// innermost first, so depth d adds X_0 d times after the final draw.
// Steps 5-8 keep j on rejection and draw fresh (ux, uy); the first attempt
// reuses U_1 as ux (its bits are disjoint from i).
template <typename T, typename W, class Tab>
__device__ T exp_general(W& w, const Tab& t, Limits lim, bool& err) {
  typedef Prec<T> P;
  int depth = 0;
  T x;
  for (;;) {
    const uint64_t w0 = w.next();
    const int i = (int)(w0 & (uint64_t)(Tab::kIMax - 1));
    const typename P::UInt m1 = P::ubits(w0);
    if (i < t.L) {
      const T X = P::X(t, i);
      x = P::fmat(P::one_plus(m1), X, -X);  // RN(U X_i)
      break;
    }
    const int j = alias_pick(t, w.next());
    if (j == 0) {
      if (++depth > lim.max_tail) {
        err = true;
        return P::nan();
      }
      continue;
    }
    typename P::UInt mx = m1;
    for (int att = 1;; ++att) {
      const typename P::UInt my = P::ubits(w.next());
      if (overhang_attempt<ZIG_EXP, T, Tab>(t, j, mx, my, x)) break;
      if (att >= lim.max_att) {
        err = true;
        return P::nan();
      }
      mx = P::ubits(w.next());
    }
    break;
  }
  for (int d = 0; d < depth; ++d) x = P::add(P::X(t, 0), x);
  return x;
}

// Full Table 1 for the normal: sign from bit 8 of the first word; the tail
// beyond X_0 by Marsaglia-Tsang from two exponential draws (a = E_1 / X_0,
// accept when 2 E_2 > a^2, return X_0 + a); overhangs by rejection against
// e^{-x^2/2}, keeping j and redrawing both uniforms.
template <typename T, typename W, class Tab>
__device__ T normal_general(W& w, const Tab& te, const Tab& tn, Limits lim, bool& err) {
  typedef Prec<T> P;
  const uint64_t w0 = w.next();
  const int i = (int)(w0 & (uint64_t)(Tab::kIMax - 1));
  const bool negative = ((w0 >> Tab::kBits) & 1u) != 0;
  const typename P::UInt m1 = P::ubits(w0);
  T x;
  if (i < tn.L) {
    // the sign on X_i inside the one rounding (a zero is +0)
    const T X = negative ? -P::X(tn, i) : P::X(tn, i);
    return P::fmat(P::one_plus(m1), X, -X);
  } else {
    const int j = alias_pick(tn, w.next());
    if (j == 0) {
      T a;
      for (int att = 1;; ++att) {
        a = P::mul(exp_general<T>(w, te, lim, err), P::rinv(tn));
        const T b = exp_general<T>(w, te, lim, err);
        if (err) return P::nan();
        const double ad = (double)a, bd = (double)b;
        if (__dadd_rn(bd, bd) > __dmul_rn(ad, ad)) break;
        if (att >= lim.max_att) {
          err = true;
          return P::nan();
        }
      }
      x = P::add(P::X(tn, 0), a);
    } else {
      typename P::UInt mx = m1;
      for (int att = 1;; ++att) {
        const typename P::UInt my = P::ubits(w.next());
        if (overhang_attempt<ZIG_NORMAL, T, Tab>(tn, j, mx, my, x)) break;
        if (att >= lim.max_att) {
          err = true;
          return P::nan();
        }
        mx = P::ubits(w.next());
      }
    }
  }
  return negative ? -x : x;
}

// The complete sampler for counter g of key seed; KEY 0: per-index words,
// KEY 1: packed keying; IB: index bits of the tables.
template <int DIST, typename T, int KEY = 0, int IB = 8>
__device__ __noinline__ T sample_general(uint64_t seed, uint64_t g, Limits lim) {
  typename std::conditional<KEY == 0, Words, PackedWords<T>>::type w(seed, g);
  bool err = false;
  T x = (DIST == ZIG_EXP)
            ? exp_general<T>(w, dev_tab<IB>(ZIG_EXP), lim, err)
            : normal_general<T>(w, dev_tab<IB>(ZIG_EXP), dev_tab<IB>(ZIG_NORMAL), lim, err);
  if (err) atomicOr(&g_status, kLoopLimitBit);
  return x;
}

// ---------------------------------------------------------------------------
// Fast path (steps 1-2) on a first word (lo, hi)
// ---------------------------------------------------------------------------
// x = RN(U sX) computed as fma(1 + U, sX, -sX): (1 + U) sX - sX equals
// U sX exactly and the FMA rounds once.  sX is read from a table of
// 2 i_max entries indexed by i | sign << IB: +X_i, then -X_i for the
// normal's negative draws (the exponential reads the first half only), so
// the sign costs nothing; a zero (U = 0) comes out +0 for either sign.
template <int DIST, int IB = 8>
__device__ __forceinline__ double fast_value(uint32_t lo, uint32_t hi, const double* sX) {
  constexpr uint32_t kMask = ((DIST == ZIG_NORMAL ? 2u : 1u) << IB) - 1u;
  const double X = sX[lo & kMask];
  const double one_u = __hiloint2double((int)(0x3FF00000u | (hi >> 12)),
                                        (int)__funnelshift_r(lo, hi, 12));
  return __fma_rn(one_u, X, -X);
}

template <int DIST, int IB = 8>
__device__ __forceinline__ float fast_value(uint32_t lo, uint32_t hi, const float* sX) {
  constexpr uint32_t kMask = ((DIST == ZIG_NORMAL ? 2u : 1u) << IB) - 1u;
  const float X = sX[lo & kMask];
  return __fmaf_rn(__int_as_float((int)(0x3F800000u | (hi >> 9))), X, -X);
}

}  // namespace zig

#endif
