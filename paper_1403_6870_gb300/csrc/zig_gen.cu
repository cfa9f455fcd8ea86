// zig_gen.cu -- sm_103a generation kernels and the C ABI.
//
// McFarland, arXiv:1403.6870, Table 1 (modified column).  Steps 1-2 (the
// common case: 98.4% of exponential and 98.8% of normal draws) run for
// every output without divergence: the Philox block, the word split, one
// shared-memory lookup of X_i, one fused multiply-add and a vector store.
//
// Every warp runs steps 1-2 for its outputs: a draw whose layer index is
// not below L_max is stored like the others (a placeholder) and marked in
// its lane's mask for the tile; a lane with any such draw appends one entry
// (its first position and the mask) to the warp's queue in shared memory.
// Whenever the queue holds 32 entries the warp runs the rest of the
// algorithm in stages, one marked draw per entry and lane, so the 32 lanes
// execute the same step:
//   stage 1: steps 3-7 (alias pick, first attempt in the overhang box);
//   stage 2: one more attempt for each rejected draw (step 8 keeps j);
//   stage 3: tail draws, through the complete sampler of zig_device.cuh.
// Its results overwrite the placeholders.  A warp drains its queues (with
// partial stages) once its tiles are done.  No warp waits for another.
//
// Compiled with --fmad=false: every fused multiply-add is written as one;
// everything else rounds per operation, as the algorithm's readings state.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "zig_device.cuh"
#include "zig_emul.h"
#include "zig_internal.h"

namespace zig {

template <typename T, int V>
struct VecStore;
template <>
struct VecStore<double, 2> {
  static __device__ __forceinline__ void st(double* p, const double* v) {
    asm volatile("st.global.v2.f64 [%0], {%1, %2};" ::"l"(p), "d"(v[0]), "d"(v[1]) : "memory");
  }
};
template <>
struct VecStore<double, 4> {
  static __device__ __forceinline__ void st(double* p, const double* v) {
    asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(p), "d"(v[0]), "d"(v[1]),
                 "d"(v[2]), "d"(v[3])
                 : "memory");
  }
};
template <>
struct VecStore<float, 4> {
  static __device__ __forceinline__ void st(float* p, const float* v) {
    asm volatile("st.global.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v[0]), "f"(v[1]),
                 "f"(v[2]), "f"(v[3])
                 : "memory");
  }
};
template <>
struct VecStore<float, 8> {
  static __device__ __forceinline__ void st(float* p, const float* v) {
    asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p),
                 "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]),
                 "f"(v[7])
                 : "memory");
  }
};

// Launch shape (overridable at build time for tuning sweeps).
#ifndef ZIG_GEN_MINBLOCKS
#define ZIG_GEN_MINBLOCKS 3
#endif
#ifndef ZIG_GEN_V64
#define ZIG_GEN_V64 4
#endif
#ifndef ZIG_GEN_R64
#define ZIG_GEN_R64 8
#endif
#ifndef ZIG_GEN_V32
#define ZIG_GEN_V32 8
#endif
#ifndef ZIG_GEN_R32
#define ZIG_GEN_R32 4
#endif

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kPThreads = kThreads;          // threads making outputs per CTA (all)
constexpr int kQueue = 64;                   // fringe queue slots per warp
constexpr uint64_t kWholeTag = 1ull << 63;   // position needs the whole sampler
constexpr unsigned kWaitBit = 1u << 9;       // status bit: a bounded wait gave up (reserved)

// V elements per vector store, R vector stores per thread per tile.
// A generation shape: V-element vectors (one vector store each), R vectors
// per thread and tile (S = V R outputs per thread and tile), and
// the CTAs per SM the register budget is compiled for.  The outputs do not
// depend on the shape: element t is always the variate of counter
// offset + t.
template <int V_, int R_, int MB_, int U_ = 0, int E_ = 0>
struct Shape {
  // U: vectors whose Philox chains are interleaved (0: the precision's default);
  // E: FP64 outputs per vector whose step-2 product is formed from integers
  // (zig_emul.h) instead of on the FP64 pipe (packed keying only)
  static constexpr int V = V_, R = R_, MB = MB_, U = U_, E = E_;
};

// Default shapes (the batch and fused kernels use these).
template <typename T>
struct GenShape;
template <>
struct GenShape<double> : Shape<ZIG_GEN_V64, ZIG_GEN_R64, ZIG_GEN_MINBLOCKS> {};
template <>
struct GenShape<float> : Shape<ZIG_GEN_V32, ZIG_GEN_R32, ZIG_GEN_MINBLOCKS> {};

// Default shapes of packed keying: a Philox block makes 2 FP64 / 4 FP32
// outputs, so an FP32 thread makes 64 outputs per tile to spread the tile's
// fixed costs, with the register budget of 2 CTAs per SM (measured on GB300
// against R = 2 and 4 and 3 CTAs per SM).
#ifndef ZIG_PACKED_R32
#define ZIG_PACKED_R32 8
#endif
template <typename T>
struct PackedShape;
// Integer-formed products per FP64 vector (0: none).  Measured on GB300 at
// 2^28 packed FP64 normals: 433 Gsamples/s with 0, 339 with 1, 272 with 2
// of 4 (the kernel is not bound by the FP64 pipe alone, and each integer
// product is a long dependent chain), so it is off; kept as a build option.
#ifndef ZIG_PACKED_EM64
#define ZIG_PACKED_EM64 0
#endif
#ifndef ZIG_PACKED_R64
#define ZIG_PACKED_R64 4
#endif
template <>
struct PackedShape<double>
    : Shape<ZIG_GEN_V64, ZIG_PACKED_R64, ZIG_GEN_MINBLOCKS, 0, ZIG_PACKED_EM64> {};
#ifndef ZIG_PACKED_MB32
#define ZIG_PACKED_MB32 2
#endif
template <>
struct PackedShape<float> : Shape<ZIG_GEN_V32, ZIG_PACKED_R32, ZIG_PACKED_MB32> {};

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ double ld_volatile_d(const double* p) {
  return *(const volatile double*)p;
}

// Round 1 of block 0 has counter words 2, 3 equal to zero, so its output
// word 0 is g_hi ^ k0 and round 2's product of that word by M0 is common to
// every counter with the same high word.  For a run of counters whose low
// words do not wrap, round 1's products M0 g_lo are formed by adding
// constants M0 d to one product.
struct RunState {
  uint64_t base;   // M0 g_lo of the run's first counter
  uint32_t uhi;    // hi(M0 (g_hi ^ k0)) ^ k1 of round 2
  uint32_t ulo;    // lo(M0 (g_hi ^ k0))
  __device__ __forceinline__ RunState(uint64_t g0, const RoundKeys& rk) {
    base = (uint64_t)kM0 * (uint32_t)g0;
    const uint64_t u = (uint64_t)kM0 * ((uint32_t)(g0 >> 32) ^ rk.k0[0]);
    uhi = (uint32_t)(u >> 32) ^ rk.k1[1];
    ulo = (uint32_t)u;
  }
  // block 0 (attempt 0) of counter g0 + d (no wrap of the low word)
  __device__ __forceinline__ uint4 block(uint32_t d, const RoundKeys& rk) const {
    const uint64_t p = base + (uint64_t)kM0 * d;
    const uint32_t n2 = (uint32_t)(p >> 32) ^ rk.k1[0], n3 = (uint32_t)p;
    const uint64_t p1 = mul_wide(kM1, n2);  // round 2
    return philox_rounds3to10((uint32_t)(p1 >> 32) ^ rk.k0[1], (uint32_t)p1, uhi ^ n3, ulo, rk);
  }
  // first word of block 0 for counter g0 + d (no wrap of the low word)
  __device__ __forceinline__ uint2 word(uint32_t d, const RoundKeys& rk) const {
    const uint64_t p = base + (uint64_t)kM0 * d;
    const uint32_t n2 = (uint32_t)(p >> 32) ^ rk.k1[0], n3 = (uint32_t)p;
    const uint64_t p1 = mul_wide(kM1, n2);  // round 2
    return philox_rounds3to10_first((uint32_t)(p1 >> 32) ^ rk.k0[1], (uint32_t)p1, uhi ^ n3,
                                    ulo, rk);
  }
};

// Round keys of a key, computed on the device (the batch kernel's requests
// each carry their own key).
__device__ __forceinline__ RoundKeys device_keys(uint64_t seed) {
  RoundKeys rk;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    rk.k0[r] = k0;
    rk.k1[r] = k1;
    k0 += kW0;
    k1 += kW1;
  }
  return rk;
}

// One warp's fringe queues in shared memory: new positions (q), rejected
// attempts waiting for the next one (rp: position, rs: state, rw: saved
// word) and tail draws (tq), with their lengths (warp-uniform).
struct WarpQueues {
  uint64_t q[kQueue];
  uint64_t rp[kQueue], rs[kQueue], rw[kQueue], tq[kQueue];
  // fringe masks: a lane's first output position in a tile (mp) and the
  // mask of its outputs there whose layer index is not below L_max (mm)
  uint64_t mp[kQueue], mm[kQueue];
  int nq, nr, nt, nm;
};

// Shared state of one CTA (X_i of an index of IB bits).
template <typename T, int IB = 8>
struct CtaState {
  T sX[2 << IB];  // +X_i, then -X_i (the normal's negative draws)
  WarpQueues wq[kWarps];
};

// Where values go.  A sink receives the vectors of steps 1-2 (vec, with the
// bits of the outputs the fringe stages will still patch), a per-tile
// notification, and the fringe stages' final values (put).
//
// StoreSink: materialise into out[0, n); vector vi starts at element
// head + vi V.
template <typename T>
struct StoreSink {
  T* out;
  uint64_t head;
  static constexpr bool kReduce = false;
  static constexpr bool kAffine = false;  // step 2 returns U X_i (see BatchSink)
  template <int V>
  __device__ __forceinline__ void vec(uint64_t vi, const T* v, unsigned /*fringe*/) {
    VecStore<T, V>::st(out + head + vi * V, v);
  }
  __device__ __forceinline__ void tile_end() {}
  __device__ __forceinline__ void put(uint64_t p, T x) { out[p] = x; }
};

// Histogram bin of the fused reduction: floor(256 x) + 2048 on [-8, 8);
// 4096 below -8; 4097 at or above 8 and for NaN.  256 x is exact in the
// value's own precision, so the floor is exact.
constexpr int kBins = 4098;
__device__ __forceinline__ int hist_bin(float x) {
  if (x < -8.0f) return 4096;
  if (!(x < 8.0f)) return 4097;
  return __float2int_rd(__fmul_rn(x, 256.0f)) + 2048;
}
__device__ __forceinline__ int hist_bin(double x) {
  if (x < -8.0) return 4096;
  if (!(x < 8.0)) return 4097;
  return __double2int_rd(__dmul_rn(x, 256.0)) + 2048;
}

// MomentSink: the values are never stored; each thread accumulates x, x^2,
// x^3, x^4 (FP32 values in FP32 over one tile, then added to a double-FP32
// accumulator (hi, lo) by an error-free two-sum, which keeps GB300's slow
// FP64 pipe out of the loop; FP64 values in FP64) and counts the value in
// the CTA's shared-memory histogram.  Outputs still to be patched are
// counted when the fringe stages put their final value.
template <typename T>
struct MomentSink {
  unsigned* hist;  // CTA shared histogram, kBins entries and one unused slot
  double acc[4];   // FP64 values: the sums; FP32 values: set by finish()
  T part[4];
  float hi[4], lo[4];  // FP32 values: double-FP32 sums of the tile partials
  static constexpr bool kReduce = true;
  static constexpr bool kAffine = false;
  __device__ __forceinline__ void init(unsigned* h) {
    hist = h;
    placeholders = 0u;
    for (int k = 0; k < 4; ++k) {
      acc[k] = 0.0;
      part[k] = (T)0;
      hi[k] = lo[k] = 0.0f;
    }
  }
  __device__ __forceinline__ void add_powers(T x) {
    typedef Prec<T> P;
    const T x2 = P::mul(x, x);
    part[0] = P::add(part[0], x);
    part[1] = P::add(part[1], x2);
    part[2] = P::fmat(x2, x, part[2]);
    part[3] = P::fmat(x2, x2, part[3]);
  }
  __device__ __forceinline__ void add(T x) {
    add_powers(x);
    atomicAdd(&hist[hist_bin(x)], 1u);
  }
  // Step 2's values lie strictly inside (-8, 8) (|x| < X_0), so their bin
  // needs no range test.  An output still to be patched holds the
  // placeholder +0 (its table entry is zero): it adds nothing to the power
  // sums and one count to bin 2048, which `placeholders` takes back at the
  // end; the fringe stages count its final value.
  unsigned placeholders;
  template <int V>
  __device__ __forceinline__ void vec(uint64_t, const T* v, unsigned fringe) {
    placeholders += __popc(fringe);
#pragma unroll
    for (int k = 0; k < V; ++k) {
      add_powers(v[k]);
      atomicAdd(&hist[inner_bin(v[k])], 1u);
    }
  }
  static __device__ __forceinline__ int inner_bin(float x) {
    return __float2int_rd(__fmul_rn(x, 256.0f)) + 2048;
  }
  static __device__ __forceinline__ int inner_bin(double x) {
    return __double2int_rd(__dmul_rn(x, 256.0)) + 2048;
  }
  __device__ __forceinline__ void tile_end() {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if constexpr (sizeof(T) == 8) {
        acc[k] = __dadd_rn(acc[k], (double)part[k]);
      } else {
        // two-sum (Knuth): s + e == hi + part exactly
        const float s = __fadd_rn(hi[k], (float)part[k]);
        const float b = __fsub_rn(s, hi[k]);
        const float e = __fadd_rn(__fsub_rn(hi[k], __fsub_rn(s, b)), __fsub_rn((float)part[k], b));
        hi[k] = s;
        lo[k] = __fadd_rn(lo[k], e);
      }
      part[k] = (T)0;
    }
  }
  // the thread's sums in FP64 (after its last tile)
  __device__ __forceinline__ void finish() {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[k] = __dadd_rn((double)hi[k], (double)lo[k]);
    }
  }
  __device__ __forceinline__ void put(uint64_t, T x) {
    add(x);
    tile_end();
  }
};

// -x by its sign bit: an integer operation, where a negated double would
// take an instruction on the FP64 pipe (the fast path's busiest unit)
__device__ __forceinline__ double flip_sign(double x) {
  return __hiloint2double(__double2hiint(x) ^ (int)0x80000000, __double2loint(x));
}
__device__ __forceinline__ float flip_sign(float x) { return -x; }

template <int DIST, typename T, typename Sink>
__device__ __forceinline__ void put_signed(Sink& sink, uint64_t p, T x, bool negative) {
  sink.put(p, (DIST == ZIG_NORMAL && negative) ? flip_sign(x) : x);
}

// A retry's state word: overhang j in bits 0-10 (j < 1024 at either index
// width), the normal's sign in bit 11, completed attempts in bits 12-31
// (below the 2^20 cap of zig_set_fringe_limits), the next block in 32-63.
constexpr uint64_t kStateJMask = 0x7FFull;
constexpr int kStateSignBit = 11;
constexpr int kStateAttShift = 12;

// Fringe queue lengths (warp-uniform): retries and tails.
struct SideCounts {
  int retry, tail;
};

// Append one entry per lane with f set, in lane order; returns the slot.
__device__ __forceinline__ int claim(bool f, int& n) {
  const unsigned m = __ballot_sync(0xFFFFFFFFu, f);
  const int k = n + __popc(m & ((1u << (threadIdx.x & 31u)) - 1u));
  n += __popc(m);
  return k;
}

// Step 2 with a request's affine map folded in (batched requests): with
// sB[k] = +-B_i and sD[k] = D for k = i | sign << 8 (the normal's sign bit;
// the exponential uses k = i), the value is RN((1 + U) sB[k] + sD[k]).
template <int DIST>
__device__ __forceinline__ double affine_value(uint32_t lo, uint32_t hi, const double* sB,
                                               const double* sD) {
  const uint32_t k = lo & (DIST == ZIG_NORMAL ? 0x1FFu : 0xFFu);
  const double one_u = __hiloint2double((int)(0x3FF00000u | (hi >> 12)),
                                        (int)__funnelshift_r(lo, hi, 12));
  return __fma_rn(one_u, sB[k], sD[k]);
}
template <int DIST>
__device__ __forceinline__ float affine_value(uint32_t lo, uint32_t hi, const float* sB,
                                              const float* sD) {
  const uint32_t k = lo & (DIST == ZIG_NORMAL ? 0x1FFu : 0xFFu);
  return __fmaf_rn(__int_as_float((int)(0x3F800000u | (hi >> 9))), sB[k], sD[k]);
}

// Queue values.  An item is a queued value, possibly with kWholeTag (the
// draw needs the whole sampler); the value's bits under kPosMask are the
// output position (the batch kernel keeps a request index above them).
// Sinks receive the value.
//
// Stage 1 (one fringe item per lane): steps 3-7 for the first attempt.
// Block 0 gives U_1 (as ux) and the alias word; block 1's first word gives
// uy.  Tail draws (j = 0) and whole-sampler items go to the tail queue;
// rejected attempts to the retry queue with their state.
// KEY 0 (per-index words): block 0 gives U_1 (as ux) and the alias word,
// block 1's first word uy.  KEY 1 (packed keying): U_1 from the packed
// first word, the alias word and uy from private block 0.
template <int DIST, typename T, uint64_t kPosMask, int KEY, int IB, typename Sink, typename State>
__device__ __forceinline__ void stage_new(Sink& sink, uint64_t offset, const RoundKeys& rk,
                                          Limits lim, bool active, uint64_t item, State& sh,
                                          SideCounts& c) {
  typedef Prec<T> P;
  const DevTabT<IB>& t = dev_tab<IB>(DIST);
  const bool whole = (item & kWholeTag) != 0;
  const uint64_t p = item & ~kWholeTag;  // the queued value
  const uint64_t g = offset + (p & kPosMask);
  uint64_t w0, aw;
  uint4 b1 = make_uint4(0u, 0u, 0u, 0u);
  if (KEY == 0) {
    const uint4 b0 = philox_block(g, 0u, rk);
    w0 = pack(b0.x, b0.y);
    aw = pack(b0.z, b0.w);
  } else {
    w0 = packed_first<T>(g, rk);
    b1 = philox_block(g, 0u, rk, 1u);
    aw = pack(b1.x, b1.y);
  }
  const int j = alias_pick(t, aw);
  const bool negative = ((w0 >> IB) & 1u) != 0;
  const bool overhang = active && !whole && j != 0;
  bool retry = false;
  uint64_t state = 0, next = 0;
  if (overhang) {
    if (KEY == 0) b1 = philox_block(g, 1u, rk);
    const uint64_t wy = KEY == 0 ? pack(b1.x, b1.y) : pack(b1.z, b1.w);
    T x;
    if (overhang_attempt<DIST, T, DevTabT<IB>, KEY == 1>(t, j, P::ubits(w0), P::ubits(wy), x)) {
      put_signed<DIST, T>(sink, p, x, negative);
    } else if (1 >= lim.max_att) {
      sink.put(p, P::nan());
      atomicOr(&g_status, kLoopLimitBit);
    } else {
      retry = true;
      // next block: per-index 2 (block 1's second word saved as the next
      // ux); packed: private block 1
      state = (uint64_t)j | ((uint64_t)negative << kStateSignBit) | (1ull << kStateAttShift) |
              ((KEY == 0 ? 2ull : 1ull) << 32);
      next = KEY == 0 ? pack(b1.z, b1.w) : 0ull;
    }
  }
  // a sink with the affine map folded into step 2 takes a whole item's
  // fast-path draw here, in the same form as the producers give it
  bool fast = false;
  if constexpr (Sink::kAffine) {
    if (active && whole && (int)(w0 & ((1u << IB) - 1u)) < t.L) {
      sink.put_mapped(p, affine_value<DIST>((uint32_t)w0, (uint32_t)(w0 >> 32), sink.sB, sink.sD));
      fast = true;
    }
  }
  const bool tl = active && !overhang && !fast;
  int k = claim(tl, c.tail);
  if (tl) sh.tq[k] = p;
  k = claim(retry, c.retry);
  if (retry) {
    sh.rp[k] = p;
    sh.rs[k] = state;
    sh.rw[k] = next;
  }
}

// Stage 2 (one retry per lane): ux is the saved word, uy the first word of
// the next block, whose second word is saved for the following attempt.  j
// is kept (Table 1 step 8 returns to step 4).  State as laid out above
// (kStateJMask, kStateSignBit, kStateAttShift).
template <int DIST, typename T, uint64_t kPosMask, int KEY, int IB, typename Sink, typename State>
__device__ __forceinline__ void stage_retry(Sink& sink, uint64_t offset, const RoundKeys& rk,
                                            Limits lim, bool active, uint64_t p,
                                            uint64_t state, uint64_t word, State& sh,
                                            SideCounts& c) {
  typedef Prec<T> P;
  const DevTabT<IB>& t = dev_tab<IB>(DIST);
  const int j = (int)(state & kStateJMask);
  const bool negative = ((state >> kStateSignBit) & 1u) != 0;
  const uint32_t att = (uint32_t)(state >> kStateAttShift) & 0xFFFFFu;
  const uint32_t blk = (uint32_t)(state >> 32);
  bool retry = false;
  uint64_t nstate = 0, next = 0;
  if (active) {
    // per-index: ux is the saved word, uy block blk's first word; packed:
    // both from private block blk
    const uint4 b = philox_block(offset + (p & kPosMask), blk, rk, KEY == 0 ? 0u : 1u);
    const uint64_t wx = KEY == 0 ? word : pack(b.x, b.y);
    const uint64_t wy = KEY == 0 ? pack(b.x, b.y) : pack(b.z, b.w);
    T x;
    if (overhang_attempt<DIST, T, DevTabT<IB>, KEY == 1>(t, j, P::ubits(wx), P::ubits(wy), x)) {
      put_signed<DIST, T>(sink, p, x, negative);
    } else if ((int)(att + 1) >= lim.max_att) {
      sink.put(p, P::nan());
      atomicOr(&g_status, kLoopLimitBit);
    } else {
      retry = true;
      nstate = (state & ((1ull << kStateAttShift) - 1ull)) |
               ((uint64_t)(att + 1) << kStateAttShift) | ((uint64_t)(blk + 1) << 32);
      next = KEY == 0 ? pack(b.z, b.w) : 0ull;
    }
  }
  const int k = claim(retry, c.retry);
  if (retry) {
    sh.rp[k] = p;
    sh.rs[k] = nstate;
    sh.rw[k] = next;
  }
}

// Run the retry and tail stages while they hold `need` or more
// entries (at most 32 per batch).  Each side queue holds fewer than 32
// entries before a stage-1 batch, so it stays within its 64 slots.
template <int DIST, typename T, int KEY, int IB, typename Sink, typename State>
__device__ __forceinline__ void side_stages(Sink& sink, uint64_t seed, uint64_t offset,
                                            const RoundKeys& rk, Limits lim, int need,
                                            State& sh, SideCounts& c) {
  constexpr uint64_t kPos = ~kWholeTag;
  const int lane = threadIdx.x & 31;
  for (;;) {
    if (c.retry >= need) {
      const int take = c.retry < 32 ? c.retry : 32;
      const bool active = lane < take;
      const int k = c.retry - take + lane;
      const uint64_t p = active ? sh.rp[k] : 0, st = active ? sh.rs[k] : 0,
                     w = active ? sh.rw[k] : 0;
      c.retry -= take;
      __syncwarp();  // slots read before they are refilled
      stage_retry<DIST, T, kPos, KEY, IB>(sink, offset, rk, lim, active, p, st, w, sh, c);
    } else if (c.tail >= need) {
      const int take = c.tail < 32 ? c.tail : 32;
      const bool active = lane < take;
      const uint64_t p = active ? sh.tq[c.tail - take + lane] : 0;
      c.tail -= take;
      __syncwarp();
      if (active) sink.put(p, sample_general<DIST, T, KEY, IB>(seed, offset + p, lim));
    } else {
      break;
    }
    __syncwarp();
  }
}

// Mask of a thread's outputs in one tile whose layer index is not below
// L_max (bit r V + k for output k of vector r): 32 or 64 bits.
template <int S>
using FringeMask = typename std::conditional<(S <= 32), unsigned, unsigned long long>::type;
__device__ __forceinline__ int mask_popc(unsigned m) { return __popc(m); }
__device__ __forceinline__ int mask_popc(unsigned long long m) { return __popcll(m); }
__device__ __forceinline__ int mask_ffs(unsigned m) { return __ffs(m); }
__device__ __forceinline__ int mask_ffs(unsigned long long m) { return __ffsll(m); }

// Vectors of a thread's tile whose Philox chains are interleaved (unrolled):
// FP64 2, FP32 1 (measured on GB300; more only raises register pressure).
#ifndef ZIG_GEN_UNROLL_R64
#define ZIG_GEN_UNROLL_R64 2
#endif
#ifndef ZIG_GEN_UNROLL_R32
#define ZIG_GEN_UNROLL_R32 1
#endif
#ifndef ZIG_PACKED_UNROLL_R
#define ZIG_PACKED_UNROLL_R 4
#endif
constexpr int kPackedUnrollR = ZIG_PACKED_UNROLL_R;

// Fringe flags.  With 8 index bits the flags of four outputs come from one
// byte-wise compare: index_flags gathers the four words' index bytes (byte
// permutes) and, with each byte of add equal to 256 - L (L >= 128), sets
// bit 8 q + 7 exactly when output q's byte is at least L (the byte's low
// seven bits plus 256 - L carry into its top bit when it is >= L, and
// never out of the byte).  Group b of a vector shifts its flags right by
// b; place_flags puts vector r's flags of group bb = r V / 4 + b at bit
// 32 (bb / 8) + 8 q + 7 - bb % 8 of the tile mask (fringe_offset decodes
// it).  Otherwise (10 index bits, packed FP64) output s of the tile is
// bit s (vector s / V, element s % V).
template <typename T, int V, int IB, int KEY>
__host__ __device__ constexpr bool byte_flags() {
  return IB == 8 && V % 4 == 0 && (KEY == 0 || sizeof(T) == 4);
}
__device__ __forceinline__ uint32_t index_flags(const uint32_t* lo, uint32_t add) {
  const uint32_t t =
      __byte_perm(__byte_perm(lo[0], lo[1], 0x0040u), __byte_perm(lo[2], lo[3], 0x0040u), 0x5410u);
  return (((t & 0x7F7F7F7Fu) + add) & t) & 0x80808080u;
}
template <int V, int R, bool BYTES>
__device__ __forceinline__ FringeMask<V * R> place_flags(unsigned f, int r) {
  if (!BYTES) return (FringeMask<V * R>)f << (r * V);
  constexpr int B = V / 4;
  return (FringeMask<V * R>)(f >> ((r * B) % 8)) << (32 * ((r * B) / 8));
}

// Steps 1-2 for one thread's S = V R outputs of a tile: vector r
// holds counters g0 + r kPThreads V + [0, V) and is vector v0 + r kPThreads
// of the output.  The Philox chains of U vectors are interleaved (U from
// the shape, else the precision's default).  Returns the
// mask of outputs (bit r V + k) whose layer index is not below L_max.
// NOWRAP: the low counter words do not wrap inside the run.  full: every
// vector lies inside the output (else vector r exists only if
// v0 + r kPThreads < nvec).
template <int DIST, typename T, typename Shp, bool NOWRAP, int IB, typename Sink>
__device__ __forceinline__ FringeMask<Shp::V * Shp::R> producer_tile(
    Sink& sink, uint64_t g0, uint64_t v0, uint64_t nvec, bool full, const RoundKeys& rk,
    const T* sX, uint32_t L) {
  constexpr int V = Shp::V, R = Shp::R;
  constexpr int kUnrollR =
      Shp::U > 0 ? Shp::U : (sizeof(T) == 8 ? ZIG_GEN_UNROLL_R64 : ZIG_GEN_UNROLL_R32);
  static_assert(V * R <= 64, "at most 64 outputs per thread and tile");
  constexpr bool kBytes = byte_flags<T, V, IB, 0>();
  const uint32_t add = (256u - L) * 0x01010101u;
  FringeMask<V * R> fm = 0;
  const RunState run(g0, rk);
#pragma unroll kUnrollR
  for (int r = 0; r < R; ++r) {
    T v[V];
    uint32_t lo[V];
    unsigned f = 0;
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const uint32_t d = (uint32_t)(r * kPThreads * V + k);
      const uint2 w = NOWRAP ? run.word(d, rk) : philox_first(g0 + d, rk);
      if constexpr (Sink::kAffine)
        v[k] = affine_value<DIST>(w.x, w.y, sink.sB, sink.sD);
      else
        v[k] = fast_value<DIST, IB>(w.x, w.y, sX);
      lo[k] = w.x;
      if (!kBytes) f |= (unsigned)((w.x & ((1u << IB) - 1u)) >= L) << k;
    }
    if (kBytes) {
#pragma unroll
      for (int b = 0; b < V / 4; ++b) f |= index_flags(lo + 4 * b, add) >> b;
    }
    const uint64_t vi = v0 + (uint64_t)(r * kPThreads);
    if (full || vi < nvec) {
      sink.template vec<V>(vi, v, f);
      fm |= place_flags<V, R, kBytes>(f, r);
    }
  }
  sink.tile_end();
  return fm;
}

// Step 2 as fast_value, with the product RN(U sX) formed from integers
// (zig_emul.h): the same bits, without the FP64 pipe.  Placeholders of
// fringe draws (sX = 0) come out as arbitrary bits and are overwritten.
template <int DIST, int IB = 8, typename T>
__device__ __forceinline__ T fast_value_int(uint32_t lo, uint32_t hi, const T* sX) {
  if constexpr (sizeof(T) == 4) {
    return fast_value<DIST, IB>(lo, hi, sX);
  } else {
    constexpr uint32_t kMask = ((DIST == ZIG_NORMAL ? 2u : 1u) << IB) - 1u;
    const uint64_t m = ((uint64_t)(hi >> 12) << 32) | __funnelshift_r(lo, hi, 12);
    return __longlong_as_double(
        (long long)emul_u_times_x(m, (uint64_t)__double_as_longlong(sX[lo & kMask])));
  }
}

// Packed keying (KEY 1) for one thread's tile: each Philox block
// gives B = V / P whole outputs (P = 2 FP64 words or 4 FP32 lanes), so a
// vector takes V / P blocks.  MODE 0: the vector's counters start at a
// multiple of P and the run's block counters do not wrap their low word;
// MODE 1: aligned, with wrap; MODE 2: not aligned (one block per output).
template <int DIST, typename T, typename Shp, int MODE, int IB, typename Sink>
__device__ __forceinline__ FringeMask<Shp::V * Shp::R> producer_tile_packed(
    Sink& sink, uint64_t g0, uint64_t v0, uint64_t nvec, bool full, const RoundKeys& rk,
    const T* sX, uint32_t L) {
  constexpr int V = Shp::V, R = Shp::R;
  constexpr int P = sizeof(T) == 8 ? 2 : 4, SH = sizeof(T) == 8 ? 1 : 2, B = V / P;
  static_assert(V % P == 0, "a vector holds whole blocks");
  static_assert(V * R <= 64, "at most 64 outputs per thread and tile");
  static_assert(IB == 8 || sizeof(T) == 8, "a 32-bit packed word has room for 8 index bits");
  static_assert(Shp::E == 0 || !Sink::kReduce, "integer products leave no +0 placeholders");
  constexpr uint32_t kIM = (1u << IB) - 1u;
  FringeMask<V * R> fm = 0;
  const uint64_t h0 = g0 >> SH;
  const RunState run(h0, rk);
  const uint32_t add = (256u - L) * 0x01010101u;  // FP32: index_flags
#pragma unroll kPackedUnrollR
  for (int r = 0; r < R; ++r) {
    T v[V];
    unsigned f = 0;
    if (MODE != 2) {
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const uint32_t d = (uint32_t)(r * kPThreads * B + b);
        const uint4 w = MODE == 0 ? run.block(d, rk) : philox_block(h0 + d, 0u, rk);
        if (sizeof(T) == 8) {
          v[2 * b] = 2 * b >= V - Shp::E ? fast_value_int<DIST, IB>(w.x, w.y, sX)
                                         : fast_value<DIST, IB>(w.x, w.y, sX);
          v[2 * b + 1] = 2 * b + 1 >= V - Shp::E ? fast_value_int<DIST, IB>(w.z, w.w, sX)
                                                 : fast_value<DIST, IB>(w.z, w.w, sX);
          f |= ((unsigned)((w.x & kIM) >= L) | ((unsigned)((w.z & kIM) >= L) << 1)) << (2 * b);
        } else {
          v[4 * b] = fast_value<DIST, IB>(w.x, w.x, sX);
          v[4 * b + 1] = fast_value<DIST, IB>(w.y, w.y, sX);
          v[4 * b + 2] = fast_value<DIST, IB>(w.z, w.z, sX);
          v[4 * b + 3] = fast_value<DIST, IB>(w.w, w.w, sX);
          const uint32_t lo[4] = {w.x, w.y, w.z, w.w};
          f |= index_flags(lo, add) >> b;
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < V; ++k) {
        const uint64_t g = g0 + (uint64_t)(r * kPThreads * V + k);
        const uint64_t w = packed_word_of<T>(philox_block(g >> SH, 0u, rk), g);
        v[k] = fast_value<DIST, IB>((uint32_t)w, (uint32_t)(w >> 32), sX);
        const unsigned flag = (unsigned)(((uint32_t)w & kIM) >= L);
        f |= sizeof(T) == 8 ? flag << k : flag << (8 * (k % 4) + 7 - k / 4);
      }
    }
    const uint64_t vi = v0 + (uint64_t)(r * kPThreads);
    if (full || vi < nvec) {
      sink.template vec<V>(vi, v, f);
      fm |= place_flags<V, R, byte_flags<T, V, IB, 1>()>(f, r);
    }
  }
  sink.tile_end();
  return fm;
}

// Offset within a lane's tile of the output marked by bit sb of its fringe
// mask (layouts of place_flags).
template <int V, bool BYTES>
__device__ __forceinline__ uint32_t fringe_offset(int sb) {
  if (!BYTES) return (uint32_t)((sb / V) * (kPThreads * V) + sb % V);
  constexpr int B = V / 4;
  const int within = sb & 31;
  const int bb = 8 * (sb >> 5) + 7 - (within & 7);
  return (uint32_t)((bb / B) * (kPThreads * V) + 4 * (bb % B) + (within >> 3));
}
// Scratch of zig_moments_noalloc: the same layout as a caller workspace
// (a 256-byte ticket area, then 4 FP64 partials per CTA), in static device
// memory that every device loading the library holds until exit.  Host
// code must not pass the symbol itself to a kernel: its device address is
// taken once per device with cudaGetSymbolAddress in zig_build_tables.
constexpr size_t kStaticScratchBytes = 64 * 1024;
static __device__ __align__(256) unsigned char g_moment_scratch[kStaticScratchBytes];

// Where the fused reduction's partial results go: per-CTA FP64 partials
// in a caller workspace, the last CTA to finish sums them in CTA order.
struct ReduceOut {
  double* sums;                   // device, 4 values (output)
  unsigned long long* hist;       // device, kBins counts (output, zeroed before launch)
  double* part;                   // workspace: gridDim.x x 4 partial sums
  unsigned* ticket;               // workspace: CTAs finished (zero before launch)
};

// Fringe work of one warp.  Stage 1 runs on the queued fringe masks, 32
// entries at a time while 32 or more are queued (all of them when
// draining): each lane takes the lowest set bit of its entry (output s of
// the lane's tile, at position base + (s / V) kPThreads V + s % V) and
// queues the rest of the entry again.  Whole-sampler items (head and tail
// elements) run when draining.  The retry and tail stages run whenever 32
// or more entries wait (all when draining).  The sink travels by value so
// that the caller keeps its copy in registers.
#ifndef ZIG_FRINGE_ATTR
#define ZIG_FRINGE_ATTR __forceinline__
#endif
template <int DIST, typename T, int KEY, int IB, int V, typename Sink>
__device__ ZIG_FRINGE_ATTR Sink fringe_work(Sink sink, WarpQueues& wq, uint64_t seed,
                                            uint64_t offset, Limits lim, bool drain) {
  const int lane = threadIdx.x & 31;
  const RoundKeys rk = device_keys(seed);
  SideCounts c{wq.nr, wq.nt};
  int nq = wq.nq, nm = wq.nm;
  __syncwarp();  // every lane's placeholder stores come before the fixes
  while (nm >= 32 || (drain && nm > 0)) {
    const int take = nm < 32 ? nm : 32;
    const bool active = lane < take;
    const uint64_t base = active ? wq.mp[nm - take + lane] : 0;
    const uint64_t mask = active ? wq.mm[nm - take + lane] : 0;
    nm -= take;
    __syncwarp();  // entries read before their slots are refilled
    const uint64_t rest = mask & (mask - 1u);
    const int k = claim(rest != 0u, nm);
    if (rest != 0u) {
      wq.mp[k] = base;
      wq.mm[k] = rest;
    }
    const int sb = active ? __ffsll((long long)mask) - 1 : 0;
    const uint64_t item = base + fringe_offset<V, byte_flags<T, V, IB, KEY>()>(sb);
    stage_new<DIST, T, ~kWholeTag, KEY, IB>(sink, offset, rk, lim, active, item, wq, c);
    __syncwarp();
    side_stages<DIST, T, KEY, IB>(sink, seed, offset, rk, lim, 32, wq, c);
  }
  while (nq >= 32 || (drain && nq > 0)) {
    const int take = nq < 32 ? nq : 32;
    const bool active = lane < take;
    const uint64_t item = active ? wq.q[nq - take + lane] : 0;
    nq -= take;
    __syncwarp();
    stage_new<DIST, T, ~kWholeTag, KEY, IB>(sink, offset, rk, lim, active, item, wq, c);
    __syncwarp();
    side_stages<DIST, T, KEY, IB>(sink, seed, offset, rk, lim, 32, wq, c);
  }
  if (drain) side_stages<DIST, T, KEY, IB>(sink, seed, offset, rk, lim, 1, wq, c);
  __syncwarp();
  if (lane == 0) {
    wq.nq = nq;
    wq.nm = nm;
    wq.nr = c.retry;
    wq.nt = c.tail;
  }
  __syncwarp();
  return sink;
}

// One CTA's share of a generation over outputs [0, n): a head of < V
// elements up to the first V-element-aligned address, nvec aligned
// V-vectors, then a tail of < V elements.  Tile t covers vectors
// [t kTile, (t + 1) kTile); thread pt makes vectors t kTile + r kPThreads +
// pt, r < R.  This CTA takes tiles tile, tile + step, ... below tile_end;
// if `ends`, its warp 0 also queues the head and tail elements for the
// whole sampler.  Each lane queues one entry per tile for its draws whose
// layer index is not below L_max (its first position and their mask); the
// warp runs the fringe stages for every 32 entries and drains its queues
// before returning; on return every output of the CTA's tiles has its final
// value (the warps have not synchronised).
template <int DIST, typename T, typename Shp, int KEY, int IB, typename Sink, typename State>
__device__ __forceinline__ void gen_tiles(State& sh, Sink& sink, const T* sX, uint64_t n,
                                          uint64_t head, uint64_t nvec, uint64_t seed,
                                          uint64_t offset, const RoundKeys& rk, Limits lim,
                                          uint64_t tile, uint64_t tile_end, uint64_t step,
                                          bool ends) {
  constexpr int V = Shp::V, R = Shp::R;
  constexpr int kTile = kPThreads * R;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  WarpQueues& wq = sh.wq[tid >> 5];
  const uint32_t L = (uint32_t)dev_tab<IB>(DIST).L;
  const uint64_t body_end = head + nvec * V;
  {
    // head and tail elements (fewer than V each) take the whole sampler
    const int hc = ends && tid < 32 && (uint64_t)lane < head ? 1 : 0;
    const int tc = ends && tid < 32 && (uint64_t)lane < n - body_end ? 1 : 0;
    const int cnt = hc + tc;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += y;
    }
    int slot = incl - cnt;
    if (hc) wq.q[slot++] = kWholeTag | (uint64_t)lane;
    if (tc) wq.q[slot] = kWholeTag | (body_end + (uint64_t)lane);
    const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    if (lane == 0) {
      wq.nq = total;
      wq.nr = 0;
      wq.nt = 0;
      wq.nm = 0;
    }
    __syncwarp();
  }
  constexpr uint32_t kSpan = (uint32_t)((R - 1) * kPThreads * V + (V - 1));
  for (; tile < tile_end; tile += step) {
    const uint64_t v0 = tile * kTile + (uint64_t)tid;  // this thread's first vector
    const uint64_t p0 = head + v0 * V;                   // and its first position
    const uint64_t g0 = offset + p0;
    const bool full = (tile + 1) * kTile <= nvec;
    FringeMask<V * R> fm;  // outputs of this thread whose layer index is >= L_max
    if constexpr (KEY == 0) {
      if ((uint32_t)g0 <= 0xFFFFFFFFu - kSpan)
        fm = producer_tile<DIST, T, Shp, true, IB>(sink, g0, v0, nvec, full, rk, sX, L);
      else
        fm = producer_tile<DIST, T, Shp, false, IB>(sink, g0, v0, nvec, full, rk, sX, L);
    } else {
      constexpr int P = sizeof(T) == 8 ? 2 : 4, SH = sizeof(T) == 8 ? 1 : 2;
      constexpr uint32_t kSpanB = (uint32_t)((R - 1) * kPThreads * (V / P) + (V / P - 1));
      if (g0 % P != 0)
        fm = producer_tile_packed<DIST, T, Shp, 2, IB>(sink, g0, v0, nvec, full, rk, sX, L);
      else if ((uint32_t)(g0 >> SH) <= 0xFFFFFFFFu - kSpanB)
        fm = producer_tile_packed<DIST, T, Shp, 0, IB>(sink, g0, v0, nvec, full, rk, sX, L);
      else
        fm = producer_tile_packed<DIST, T, Shp, 1, IB>(sink, g0, v0, nvec, full, rk, sX, L);
    }
    // queue this lane's fringe mask as one entry; run the fringe stages
    // whenever 32 entries are queued (fewer than 32 are queued here)
    const bool has = fm != 0;
    const unsigned b = __ballot_sync(0xFFFFFFFFu, has);
    if (b != 0u) {
      const int nm = wq.nm;
      if (has) {
        const int k = nm + __popc(b & ((1u << lane) - 1u));
        wq.mp[k] = p0;
        wq.mm[k] = (uint64_t)fm;
      }
      const int total = nm + __popc(b);
      __syncwarp();
      if (lane == 0) wq.nm = total;
      __syncwarp();
      if (total >= 32) sink = fringe_work<DIST, T, KEY, IB, V>(sink, wq, seed, offset, lim, false);
    }
  }
  sink = fringe_work<DIST, T, KEY, IB, V>(sink, wq, seed, offset, lim, true);
}

// One launch covers outputs [0, n) (layout as in gen_tiles); CTA b takes
// tiles b, b + gridDim.x, ... and CTA 0 the head and tail elements.
template <int DIST, typename T, typename Sink, typename Shp = GenShape<T>, int KEY = 0, int IB = 8>
__global__ void __launch_bounds__(kThreads, Shp::MB)
    gen_kernel(Sink sink, uint64_t n, uint32_t head, uint64_t nvec, uint64_t seed,
               uint64_t offset, const RoundKeys rk, Limits lim, ReduceOut red) {
  constexpr int R = Shp::R;
  constexpr int kTile = kPThreads * R;
  __shared__ CtaState<T, IB> sh;
  __shared__ unsigned shist[Sink::kReduce ? kBins + 1 : 1];

  const int tid = threadIdx.x;
  for (int k = tid; k < (2 << IB); k += kThreads) {
    // entries i >= L_max are zero: step 2 leaves the placeholder +0 there
    const int i = k & ((1 << IB) - 1);
    const T X = i < dev_tab<IB>(DIST).L ? Prec<T>::X(dev_tab<IB>(DIST), i) : (T)0;
    sh.sX[k] = (k >> IB) ? -X : X;
  }
  if (Sink::kReduce)
    for (int k = tid; k < kBins; k += kThreads) shist[k] = 0u;
  if constexpr (Sink::kReduce) sink.init(shist);
  __syncthreads();

  const uint64_t ntiles = (nvec + kTile - 1) / kTile;
  gen_tiles<DIST, T, Shp, KEY, IB>(sh, sink, sh.sX, n, head, nvec, seed, offset, rk, lim,
                               blockIdx.x, ntiles, gridDim.x, blockIdx.x == 0);

  if constexpr (Sink::kReduce) {
    // CTA partials in thread order, then the CTA's histogram into the
    // output; the last CTA to finish sums the partials in CTA order.  The
    // partials reuse the warp queues, empty once every warp has drained.
    static_assert(sizeof(sh.wq) >= kThreads * 4 * sizeof(double), "partials fit the queues");
    double (*rsum)[4] = reinterpret_cast<double (*)[4]>(&sh.wq[0]);
    __shared__ bool last_cta;
    sink.finish();
    if (sink.placeholders) atomicSub(&shist[2048], sink.placeholders);
    __syncthreads();
    for (int k = 0; k < 4; ++k) rsum[tid][k] = sink.acc[k];
    __syncthreads();
    if (tid < 4) {
      double a = 0.0;
      for (int t = 0; t < kThreads; ++t) a = __dadd_rn(a, rsum[t][tid]);
      rsum[0][tid] = a;
    }
    for (int k = tid; k < kBins; k += kThreads)
      if (shist[k]) atomicAdd(&red.hist[k], (unsigned long long)shist[k]);
    __syncthreads();
    if (tid < 4) red.part[(size_t)blockIdx.x * 4 + tid] = rsum[0][tid];
    __threadfence();
    __syncthreads();
    if (tid == 0) last_cta = atomicAdd(red.ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last_cta) {
      __threadfence();
      if (tid < 4) {
        double a = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) a = __dadd_rn(a, ld_volatile_d(&red.part[(size_t)b * 4 + tid]));
        red.sums[tid] = a;
      }
      if (tid == 0) *red.ticket = 0u;
    }
  }
}

}  // namespace zig

#include "zig_batch.cuh"

namespace zig {

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

constexpr int kMaxDevices = 64;

std::mutex g_mu;
zig_tables_export g_host[2];
zig_tables_ex g_host8ex[2];  // i_max = 256 in the wide layout
zig_tables_ex g_host10[2];   // i_max = 1024
std::atomic<bool> g_host_ready{false};
std::atomic<int> g_max_att{64};
std::atomic<int> g_max_tail{16};

// Launch shape in use for one (dist, dtype): candidate index, CTAs per SM
// (0 = as many as fit) and the rate it was measured at.
struct Selection {
  std::atomic<int> variant{0};
  std::atomic<int> bps{0};
  std::atomic<double> rate{0.0};
};

struct DeviceState {
  std::atomic<bool> ready{false};
  unsigned int* d_status = nullptr;
  void* d_static_scratch = nullptr;  // device address of g_moment_scratch
  int sms = 0;
  char name[256] = {0};
  Selection sel[2][2];  // [dist][dtype]
  std::atomic<uint32_t> batch_chunk{kBatchChunkDefault};  // zig_batch tiles per claim
  std::atomic<uint32_t> poll_seq{0};  // zig_status_poll's next slot (mod kPollSlots)
};
DeviceState g_dev[kMaxDevices];

zig_status ensure_host_tables() {
  if (g_host_ready.load(std::memory_order_acquire)) return ZIG_OK;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_host_ready.load()) return ZIG_OK;
  if (build_host_tables(&g_host[0], &g_host[1]) != 0) return ZIG_E_TABLE;
  if (build_host_tables_ex(8, &g_host8ex[0], &g_host8ex[1]) != 0) return ZIG_E_TABLE;
  if (build_host_tables_ex(10, &g_host10[0], &g_host10[1]) != 0) return ZIG_E_TABLE;
  g_host_ready.store(true, std::memory_order_release);
  return ZIG_OK;
}

template <class Host, int IB>
void to_device_layout(const Host& h, DevTabT<IB>* d) {
  constexpr int kIMax = 1 << IB;
  std::memset(d, 0, sizeof(*d));
  for (int k = 0; k <= h.L && k < kIMax; ++k) {
    d->X[k] = h.X[k];
    d->X32[k] = h.X32[k];
  }
  for (int k = 0; k <= h.L; ++k) {
    d->f[k] = h.f[k];
    d->dX[k] = h.dX[k];
    d->df[k] = h.df[k];
    d->f32[k] = h.f32[k];
    d->dX32[k] = h.dX32[k];
    d->df32[k] = h.df32[k];
  }
  for (int c = 0; c < kIMax; ++c) {
    d->T[c] = h.T[c];
    d->alias[c] = h.alias[c];
  }
  for (int j = 0; j <= h.L && j <= kIMax; ++j) {
    d->acc52[j] = h.acc52[j];
    d->rej52[j] = h.rej52[j];
    d->acc23[j] = (unsigned int)h.acc23[j];
    d->rej23[j] = (unsigned int)h.rej23[j];
  }
  d->tau = h.tau;
  d->rinv = h.rinv;
  d->rinv32 = h.rinv32;
  d->L = h.L;
}

zig_status current_device(int* dev) {
  if (cudaGetDevice(dev) != cudaSuccess) {
    cudaGetLastError();
    return ZIG_E_CUDA;
  }
  if (*dev < 0 || *dev >= kMaxDevices) return ZIG_E_CUDA;
  return ZIG_OK;
}

RoundKeys round_keys(uint64_t seed) {
  RoundKeys rk;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    rk.k0[r] = k0;
    rk.k1[r] = k1;
    k0 += kW0;
    k1 += kW1;
  }
  return rk;
}

template <int DIST, typename T, typename Sink, typename Shp = GenShape<T>, int KEY = 0, int IB = 8>
int occupancy_blocks(int dev) {
  static std::atomic<int> cache[kMaxDevices];
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gen_kernel<DIST, T, Sink, Shp, KEY, IB>,
                                                    kThreads, 0) != cudaSuccess ||
      occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  cache[dev].store(occ, std::memory_order_relaxed);
  return occ;
}

// Materialising launch of shape Shp with at most bps CTAs per SM (0: as
// many as fit).
template <int DIST, typename T, typename Shp, int KEY = 0, int IB = 8>
zig_status launch_gen(void* out, uint64_t n, uint64_t seed, uint64_t offset,
                      cudaStream_t stream, int dev, int bps) {
  constexpr int V = Shp::V, R = Shp::R;
  const uintptr_t addr = (uintptr_t)out;
  const uint64_t align_elems = (uint64_t)((V - (addr / sizeof(T)) % V) % V);
  const uint64_t head = align_elems < n ? align_elems : n;
  const uint64_t nvec = (n - head) / V;
  const uint64_t tiles = (nvec + (uint64_t)kPThreads * R - 1) / ((uint64_t)kPThreads * R);
  int occ = occupancy_blocks<DIST, T, StoreSink<T>, Shp, KEY, IB>(dev);
  if (bps > 0 && bps < occ) occ = bps;
  const uint64_t cap = (uint64_t)g_dev[dev].sms * (uint64_t)occ;
  uint64_t grid = tiles < cap ? tiles : cap;
  if (grid < 1) grid = 1;
  Limits lim{g_max_att.load(), g_max_tail.load()};
  StoreSink<T> sink{(T*)out, head};
  gen_kernel<DIST, T, StoreSink<T>, Shp, KEY, IB><<<(unsigned)grid, kThreads, 0, stream>>>(
      sink, n, (uint32_t)head, nvec, seed, offset, round_keys(seed), lim, ReduceOut{});
  if (cudaGetLastError() != cudaSuccess) return ZIG_E_CUDA;
  return ZIG_OK;
}

// The autotuner's candidate shapes per precision (index 0 is the default).
// FP64: 16- or 32-byte vectors, 8-16 outputs per thread and tile, register
// budgets for 2-4 CTAs per SM; FP32 likewise with 16- or 32-byte vectors
// and 16-64 outputs per thread and tile.
constexpr int kVariants = 5;
template <typename T>
struct Variants;
template <>
struct Variants<double> {
  static constexpr int V[kVariants] = {GenShape<double>::V, 4, 4, 4, 4};
  static constexpr int R[kVariants] = {GenShape<double>::R, 4, 16, 8, 8};
  static constexpr int MB[kVariants] = {GenShape<double>::MB, 3, 3, 4, 2};
};
template <>
struct Variants<float> {
  static constexpr int V[kVariants] = {GenShape<float>::V, 8, 4, 8, 8};
  static constexpr int R[kVariants] = {GenShape<float>::R, 2, 4, 4, 8};
  static constexpr int MB[kVariants] = {GenShape<float>::MB, 3, 3, 2, 3};
};

template <int DIST, typename T, int K>
using VariantShape = Shape<Variants<T>::V[K], Variants<T>::R[K], Variants<T>::MB[K]>;

template <int DIST, typename T>
zig_status launch_variant(int k, void* out, uint64_t n, uint64_t seed, uint64_t offset,
                          cudaStream_t stream, int dev, int bps) {
  switch (k) {
    case 1: return launch_gen<DIST, T, VariantShape<DIST, T, 1>>(out, n, seed, offset, stream, dev, bps);
    case 2: return launch_gen<DIST, T, VariantShape<DIST, T, 2>>(out, n, seed, offset, stream, dev, bps);
    case 3: return launch_gen<DIST, T, VariantShape<DIST, T, 3>>(out, n, seed, offset, stream, dev, bps);
    case 4: return launch_gen<DIST, T, VariantShape<DIST, T, 4>>(out, n, seed, offset, stream, dev, bps);
    default: return launch_gen<DIST, T, GenShape<T>>(out, n, seed, offset, stream, dev, bps);
  }
}

template <int DIST, typename T>
int variant_occupancy(int k, int dev) {
  switch (k) {
    case 1: return occupancy_blocks<DIST, T, StoreSink<T>, VariantShape<DIST, T, 1>>(dev);
    case 2: return occupancy_blocks<DIST, T, StoreSink<T>, VariantShape<DIST, T, 2>>(dev);
    case 3: return occupancy_blocks<DIST, T, StoreSink<T>, VariantShape<DIST, T, 3>>(dev);
    case 4: return occupancy_blocks<DIST, T, StoreSink<T>, VariantShape<DIST, T, 4>>(dev);
    default: return occupancy_blocks<DIST, T, StoreSink<T>, GenShape<T>>(dev);
  }
}

// Grid of the fused reduction on device dev (one partial per CTA).
template <int DIST, typename T, typename Shp = GenShape<T>, int KEY = 0>
uint64_t moment_grid_cap(int dev) {
  return (uint64_t)g_dev[dev].sms *
         (uint64_t)occupancy_blocks<DIST, T, MomentSink<T>, Shp, KEY>(dev);
}

constexpr size_t kTicketBytes = 256;  // workspace: ticket, then the partials

// zig_status_poll's read-and-clear of the status word, ordered on the
// caller's stream: one atomic exchange, so that a bit set by a kernel on
// another stream in between is kept for the next poll.  Each poll takes
// into a slot of its own (a ring of kPollSlots per device, handed out on
// the host), so that polls running at the same time on different streams
// never read each other's take.
constexpr unsigned kPollSlots = 64;
__device__ unsigned int g_status_taken[kPollSlots];
__global__ void status_take_kernel(unsigned slot) {
  g_status_taken[slot] = atomicExch(&g_status, 0u);
}

template <int DIST, typename T, typename Shp = GenShape<T>, int KEY = 0>
zig_status launch_moments(uint64_t n, uint64_t seed, uint64_t offset, double* d_sums,
                          unsigned long long* d_hist, void* d_ws, size_t ws_bytes,
                          cudaStream_t stream, int dev) {
  constexpr int V = Shp::V, R = Shp::R;
  const uint64_t nvec = n / V;
  const uint64_t tiles = (nvec + (uint64_t)kPThreads * R - 1) / ((uint64_t)kPThreads * R);
  const uint64_t cap = moment_grid_cap<DIST, T, Shp, KEY>(dev);
  uint64_t grid = tiles < cap ? tiles : cap;
  if (grid < 1) grid = 1;
  if (ws_bytes < kTicketBytes + grid * 4 * sizeof(double)) return ZIG_E_NOMEM;
  if (cudaMemsetAsync(d_hist, 0, kBins * sizeof(unsigned long long), stream) != cudaSuccess ||
      cudaMemsetAsync(d_ws, 0, sizeof(unsigned), stream) != cudaSuccess) {
    cudaGetLastError();
    return ZIG_E_CUDA;
  }
  Limits lim{g_max_att.load(), g_max_tail.load()};
  ReduceOut red{d_sums, d_hist, (double*)((char*)d_ws + kTicketBytes), (unsigned*)d_ws};
  MomentSink<T> sink{};
  gen_kernel<DIST, T, MomentSink<T>, Shp, KEY><<<(unsigned)grid, kThreads, 0, stream>>>(
      sink, n, 0u, nvec, seed, offset, round_keys(seed), lim, red);
  if (cudaGetLastError() != cudaSuccess) return ZIG_E_CUDA;
  return ZIG_OK;
}

static_assert(sizeof(zig_request) == 56, "zig_request layout");

size_t batch_ws_bytes(uint32_t count) { return batch_workspace_total(count); }

int batch_occupancy(int dev) {
  static std::atomic<int> cache[kMaxDevices];
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_kernel, kThreads, 0) !=
          cudaSuccess ||
      occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  cache[dev].store(occ, std::memory_order_relaxed);
  return occ;
}

zig_status check_request(const zig_request& q) {
  if (q.dist != ZIG_EXP && q.dist != ZIG_NORMAL) return ZIG_E_INVAL;
  if (q.dtype != ZIG_F32 && q.dtype != ZIG_F64) return ZIG_E_INVAL;
  if (q.n >= (1ull << kBatchPosBits)) return ZIG_E_RANGE;
  if (q.n > 0 && q.out == nullptr) return ZIG_E_INVAL;
  if ((uintptr_t)q.out % (q.dtype == ZIG_F64 ? 8 : 4)) return ZIG_E_ALIGN;
  if (q.n > 0 && q.n - 1 > UINT64_MAX - q.offset) return ZIG_E_RANGE;
  if (q.dist == ZIG_EXP && !(q.p0 > 0.0 && std::isfinite(q.p0))) return ZIG_E_INVAL;
  if (q.dist == ZIG_NORMAL && !(q.p1 > 0.0 && std::isfinite(q.p1) && std::isfinite(q.p0)))
    return ZIG_E_INVAL;
  return ZIG_OK;
}

template <typename T>
int variant_index(const zig_tune_entry& e) {
  for (int k = 0; k < kVariants; ++k)
    if (Variants<T>::V[k] == e.V && Variants<T>::R[k] == e.R && Variants<T>::MB[k] == e.min_blocks)
      return k;
  return -1;
}

int variant_index(int dtype, const zig_tune_entry& e) {
  return dtype == ZIG_F64 ? variant_index<double>(e) : variant_index<float>(e);
}

template <typename T>
zig_tune_entry variant_entry(int k, int bps, double rate) {
  return zig_tune_entry{Variants<T>::V[k], Variants<T>::R[k], Variants<T>::MB[k], bps, rate};
}

zig_tune_entry variant_entry(int dtype, int k, int bps, double rate) {
  return dtype == ZIG_F64 ? variant_entry<double>(k, bps, rate) : variant_entry<float>(k, bps, rate);
}

// Cached choices for device dev (its name and SM count) take effect.
void apply_cached(int dev) {
  for (int d = 0; d < 2; ++d)
    for (int t = 0; t < 2; ++t) {
      zig_tune_entry e;
      if (!tune_cache_get(g_dev[dev].name, g_dev[dev].sms, d, t, &e)) continue;
      const int k = variant_index(t, e);
      if (k < 0 || e.blocks_per_sm < 0) continue;
      Selection& sel = g_dev[dev].sel[d][t];
      sel.variant.store(k);
      sel.bps.store(e.blocks_per_sm);
      sel.rate.store(e.gsamples_s);
    }
}

// The address the kernels write through: device memory of the current
// device and managed memory as given; page-locked host memory
// (cudaHostAlloc, cudaHostRegister) through its device alias, which the
// kernels then write over the host link; anything else (unregistered host
// memory, another device's memory) is refused.
zig_status device_address(void* out, int dev, void** dptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, out) != cudaSuccess) {
    cudaGetLastError();
    return ZIG_E_INVAL;
  }
  switch (a.type) {
    case cudaMemoryTypeDevice:
      if (a.device != dev) return ZIG_E_INVAL;
      *dptr = out;
      return ZIG_OK;
    case cudaMemoryTypeManaged:
      *dptr = out;
      return ZIG_OK;
    case cudaMemoryTypeHost:
      if (a.devicePointer == nullptr) return ZIG_E_INVAL;
      *dptr = a.devicePointer;
      return ZIG_OK;
    default:
      return ZIG_E_INVAL;
  }
}

zig_status generate(int dist, void* out, uint64_t n, uint64_t seed, uint64_t offset,
                    zig_dtype dtype, void* stream, int keying = ZIG_KEY_INDEX,
                    int index_bits = 8) {
  if (dtype != ZIG_F32 && dtype != ZIG_F64) return ZIG_E_INVAL;
  if (dist != ZIG_EXP && dist != ZIG_NORMAL) return ZIG_E_INVAL;
  if (keying != ZIG_KEY_INDEX && keying != ZIG_KEY_PACKED) return ZIG_E_INVAL;
  if (index_bits != 8 && index_bits != 10) return ZIG_E_INVAL;
  // a packed FP32 word (32 bits) holds 8 index bits, a sign and 23 bits of U
  if (index_bits == 10 && keying == ZIG_KEY_PACKED && dtype == ZIG_F32) return ZIG_E_INVAL;
  if (n == 0) return ZIG_OK;
  if (out == nullptr) return ZIG_E_INVAL;
  const size_t es = dtype == ZIG_F64 ? 8 : 4;
  if ((uintptr_t)out % es != 0) return ZIG_E_ALIGN;
  if (n - 1 > UINT64_MAX - offset) return ZIG_E_RANGE;
  if (n > (UINT64_MAX / 16)) return ZIG_E_RANGE;
  int dev;
  zig_status st = current_device(&dev);
  if (st != ZIG_OK) return st;
  if (!g_dev[dev].ready.load(std::memory_order_acquire)) return ZIG_E_NOTINIT;
  st = device_address(out, dev, &out);
  if (st != ZIG_OK) return st;
  if ((uintptr_t)out % es != 0) return ZIG_E_ALIGN;
  cudaStream_t s = (cudaStream_t)stream;
  if (index_bits == 10) {
    if (keying == ZIG_KEY_PACKED)
      return dist == ZIG_EXP ? launch_gen<ZIG_EXP, double, PackedShape<double>, 1, 10>(
                                   out, n, seed, offset, s, dev, 0)
                             : launch_gen<ZIG_NORMAL, double, PackedShape<double>, 1, 10>(
                                   out, n, seed, offset, s, dev, 0);
    if (dist == ZIG_EXP)
      return dtype == ZIG_F64 ? launch_gen<ZIG_EXP, double, GenShape<double>, 0, 10>(
                                    out, n, seed, offset, s, dev, 0)
                              : launch_gen<ZIG_EXP, float, GenShape<float>, 0, 10>(
                                    out, n, seed, offset, s, dev, 0);
    return dtype == ZIG_F64 ? launch_gen<ZIG_NORMAL, double, GenShape<double>, 0, 10>(
                                  out, n, seed, offset, s, dev, 0)
                            : launch_gen<ZIG_NORMAL, float, GenShape<float>, 0, 10>(
                                  out, n, seed, offset, s, dev, 0);
  }
  if (keying == ZIG_KEY_PACKED) {
    if (dist == ZIG_EXP)
      return dtype == ZIG_F64 ? launch_gen<ZIG_EXP, double, PackedShape<double>, 1>(
                                    out, n, seed, offset, s, dev, 0)
                              : launch_gen<ZIG_EXP, float, PackedShape<float>, 1>(
                                    out, n, seed, offset, s, dev, 0);
    return dtype == ZIG_F64 ? launch_gen<ZIG_NORMAL, double, PackedShape<double>, 1>(
                                  out, n, seed, offset, s, dev, 0)
                            : launch_gen<ZIG_NORMAL, float, PackedShape<float>, 1>(
                                  out, n, seed, offset, s, dev, 0);
  }
  const Selection& sel = g_dev[dev].sel[dist == ZIG_EXP ? 0 : 1][dtype == ZIG_F64 ? 1 : 0];
  const int k = sel.variant.load(std::memory_order_relaxed);
  const int bps = sel.bps.load(std::memory_order_relaxed);
  if (dist == ZIG_EXP)
    return dtype == ZIG_F64 ? launch_variant<ZIG_EXP, double>(k, out, n, seed, offset, s, dev, bps)
                            : launch_variant<ZIG_EXP, float>(k, out, n, seed, offset, s, dev, bps);
  return dtype == ZIG_F64 ? launch_variant<ZIG_NORMAL, double>(k, out, n, seed, offset, s, dev, bps)
                          : launch_variant<ZIG_NORMAL, float>(k, out, n, seed, offset, s, dev, bps);
}

int variant_occupancy_any(int dist, int dtype, int k, int dev) {
  if (dist == ZIG_EXP)
    return dtype == ZIG_F64 ? variant_occupancy<ZIG_EXP, double>(k, dev)
                            : variant_occupancy<ZIG_EXP, float>(k, dev);
  return dtype == ZIG_F64 ? variant_occupancy<ZIG_NORMAL, double>(k, dev)
                          : variant_occupancy<ZIG_NORMAL, float>(k, dev);
}

// One empty launch of each fused-reduction kernel zig_moments_noalloc can
// run, on the static scratch (ticket and one CTA's partials at 0, sums at
// 1 KiB, the histogram at 2 KiB), so that the driver loads their code and
// sizes their local memory here, inside zig_build_tables, rather than on a
// later zig_moments_noalloc call (either can take device memory).
zig_status preload_moment_kernels(int dev) {
  static_assert(2048 + kBins * sizeof(unsigned long long) <= kStaticScratchBytes,
                "preload outputs fit the static scratch");
  char* base = (char*)g_dev[dev].d_static_scratch;
  double* sums = (double*)(base + 1024);
  unsigned long long* hist = (unsigned long long*)(base + 2048);
  const size_t ws = 1024;
  zig_status st = launch_moments<ZIG_EXP, float>(0, 0, 0, sums, hist, base, ws, 0, dev);
  if (st == ZIG_OK) st = launch_moments<ZIG_EXP, double>(0, 0, 0, sums, hist, base, ws, 0, dev);
  if (st == ZIG_OK) st = launch_moments<ZIG_NORMAL, float>(0, 0, 0, sums, hist, base, ws, 0, dev);
  if (st == ZIG_OK) st = launch_moments<ZIG_NORMAL, double>(0, 0, 0, sums, hist, base, ws, 0, dev);
  if (st == ZIG_OK && cudaStreamSynchronize(0) != cudaSuccess) st = ZIG_E_CUDA;
  if (st != ZIG_OK) cudaGetLastError();
  return st;
}

// zig_batch's two launches with `chunk` tiles per claim (arguments checked
// by the caller).
zig_status launch_batch(const zig_request* d_reqs, uint32_t count, unsigned long long* d_done_ns,
                        void* d_workspace, cudaStream_t s, int dev, uint32_t chunk) {
  BatchHeader* hdr = (BatchHeader*)d_workspace;
  BatchReq* reqs = (BatchReq*)((char*)d_workspace + batch_header_bytes());
  const uint32_t nranges = (uint32_t)(g_dev[dev].sms < kBatchMaxRanges ? g_dev[dev].sms
                                                                       : kBatchMaxRanges);
  batch_prep_kernel<<<1, 1024, 0, s>>>(d_reqs, count, reqs, hdr, d_done_ns, nranges, chunk);
  if (cudaGetLastError() != cudaSuccess) return ZIG_E_CUDA;
  const unsigned grid = (unsigned)(g_dev[dev].sms * batch_occupancy(dev));
  Limits lim{g_max_att.load(), g_max_tail.load()};
  batch_kernel<<<grid, kThreads, 0, s>>>(reqs, hdr, lim);
  if (cudaGetLastError() != cudaSuccess) return ZIG_E_CUDA;
  return ZIG_OK;
}

// Arguments of zig_batch / zig_batch_autotune; the device on success.
zig_status batch_args(const zig_request* d_reqs, uint32_t count, unsigned long long* d_done_ns,
                      void* d_workspace, size_t workspace_bytes, int* dev) {
  if (d_reqs == nullptr || d_workspace == nullptr) return ZIG_E_INVAL;
  if (count >= (1u << kBatchReqBits)) return ZIG_E_RANGE;
  if ((uintptr_t)d_workspace % 16 || (uintptr_t)d_reqs % 8 || (uintptr_t)d_done_ns % 8)
    return ZIG_E_ALIGN;
  if (workspace_bytes < batch_ws_bytes(count)) return ZIG_E_NOMEM;
  zig_status st = current_device(dev);
  if (st != ZIG_OK) return st;
  if (!g_dev[*dev].ready.load(std::memory_order_acquire)) return ZIG_E_NOTINIT;
  return ZIG_OK;
}

}  // namespace

const zig_tables_export* host_tables(int dist) {
  if (ensure_host_tables() != ZIG_OK) return nullptr;
  return &g_host[dist];
}

bool tune_shape_known(int dtype, const zig_tune_entry& e) { return variant_index(dtype, e) >= 0; }

void tune_apply_loaded() {
  for (int dev = 0; dev < kMaxDevices; ++dev)
    if (g_dev[dev].ready.load(std::memory_order_acquire)) apply_cached(dev);
}

}  // namespace zig

using namespace zig;

extern "C" {

const char* zig_strerror(zig_status s) {
  switch (s) {
    case ZIG_OK: return "ok";
    case ZIG_E_INVAL: return "invalid argument";
    case ZIG_E_NOTINIT: return "tables not built on this device (call zig_build_tables)";
    case ZIG_E_CUDA: return "CUDA runtime error";
    case ZIG_E_NOMEM: return "workspace too small";
    case ZIG_E_ALIGN: return "pointer not aligned to its element size";
    case ZIG_E_RANGE: return "counter range or size out of bounds";
    case ZIG_E_LOOP_LIMIT: return "a fringe loop reached its cap (outputs are NaN)";
    case ZIG_E_TABLE: return "table construction failed";
    case ZIG_E_TIMEOUT: return "a device-side wait exceeded its time limit";
  }
  return "unknown status";
}

zig_status zig_build_tables(void) {
  zig_status st = ensure_host_tables();
  if (st != ZIG_OK) return st;
  int dev;
  st = current_device(&dev);
  if (st != ZIG_OK) return st;
  if (g_dev[dev].ready.load(std::memory_order_acquire)) return ZIG_OK;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_dev[dev].ready.load()) return ZIG_OK;
  static DevTab h[2];
  static DevTabT<10> h10[2];
  to_device_layout(g_host8ex[0], &h[0]);
  to_device_layout(g_host8ex[1], &h[1]);
  to_device_layout(g_host10[0], &h10[0]);
  to_device_layout(g_host10[1], &h10[1]);
  void* status = nullptr;
  void* scratch = nullptr;
  int sms = 0;
  if (cudaMemcpyToSymbol(g_tab, h, sizeof(h)) != cudaSuccess ||
      cudaMemcpyToSymbol(g_tab10, h10, sizeof(h10)) != cudaSuccess ||
      cudaGetSymbolAddress(&status, g_status) != cudaSuccess ||
      cudaGetSymbolAddress(&scratch, g_moment_scratch) != cudaSuccess ||
      cudaMemset(status, 0, sizeof(unsigned int)) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return ZIG_E_CUDA;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return ZIG_E_CUDA;
  }
  g_dev[dev].d_status = (unsigned int*)status;
  g_dev[dev].d_static_scratch = scratch;
  g_dev[dev].sms = sms;
  std::snprintf(g_dev[dev].name, sizeof(g_dev[dev].name), "%s", prop.name);
  st = preload_moment_kernels(dev);
  if (st != ZIG_OK) return st;
  static std::once_flag env_cache;
  std::call_once(env_cache, [] {
    const char* path = std::getenv("ZIG_TUNE_CACHE");
    if (path && *path) tune_cache_load(path);
  });
  apply_cached(dev);
  g_dev[dev].ready.store(true, std::memory_order_release);
  return ZIG_OK;
}

int zig_tune_candidates(zig_dtype dtype, zig_tune_entry* out, int max) {
  if (dtype != ZIG_F32 && dtype != ZIG_F64) return 0;
  for (int k = 0; k < kVariants && out && k < max; ++k) out[k] = variant_entry(dtype, k, 0, 0.0);
  return kVariants;
}

zig_status zig_tune_get(zig_dist dist, zig_dtype dtype, zig_tune_entry* out) {
  if ((dist != ZIG_EXP && dist != ZIG_NORMAL) || (dtype != ZIG_F32 && dtype != ZIG_F64) || !out)
    return ZIG_E_INVAL;
  int dev;
  const zig_status st = current_device(&dev);
  if (st != ZIG_OK) return st;
  const Selection& sel = g_dev[dev].sel[dist][dtype];
  *out = variant_entry(dtype, sel.variant.load(), sel.bps.load(), sel.rate.load());
  return ZIG_OK;
}

zig_status zig_tune_set(zig_dist dist, zig_dtype dtype, const zig_tune_entry* e) {
  if ((dist != ZIG_EXP && dist != ZIG_NORMAL) || (dtype != ZIG_F32 && dtype != ZIG_F64) || !e)
    return ZIG_E_INVAL;
  const int k = variant_index(dtype, *e);
  if (k < 0 || e->blocks_per_sm < 0 || e->blocks_per_sm > 64) return ZIG_E_INVAL;
  int dev;
  const zig_status st = current_device(&dev);
  if (st != ZIG_OK) return st;
  Selection& sel = g_dev[dev].sel[dist][dtype];
  sel.variant.store(k);
  sel.bps.store(e->blocks_per_sm);
  sel.rate.store(e->gsamples_s);
  return ZIG_OK;
}

zig_status zig_autotune(zig_dist dist, zig_dtype dtype, void* d_scratch, size_t scratch_bytes,
                        int reps, void* stream, zig_tune_entry* results, int max_results,
                        int* n_results, zig_tune_entry* chosen) {
  if ((dist != ZIG_EXP && dist != ZIG_NORMAL) || (dtype != ZIG_F32 && dtype != ZIG_F64) ||
      d_scratch == nullptr || reps < 1 || reps > 1000)
    return ZIG_E_INVAL;
  const size_t es = dtype == ZIG_F64 ? 8 : 4;
  const uint64_t n = scratch_bytes / es;
  if (n < (1ull << 20) || (uintptr_t)d_scratch % es) return ZIG_E_INVAL;
  int dev;
  zig_status st = current_device(&dev);
  if (st != ZIG_OK) return st;
  if (!g_dev[dev].ready.load(std::memory_order_acquire)) return ZIG_E_NOTINIT;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return ZIG_E_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return ZIG_E_CUDA;
  }
  int count = 0;
  int best_k = 0, best_b = 0;
  double best = -1.0;
  st = ZIG_OK;
  for (int k = 0; k < kVariants && st == ZIG_OK; ++k) {
    const int occ = variant_occupancy_any(dist, dtype, k, dev);
    // as many CTAs per SM as fit, and one fewer
    for (int b = occ; b >= 1 && b >= occ - 1 && st == ZIG_OK; --b) {
      auto launch = [&] {
        return dist == ZIG_EXP
                   ? (dtype == ZIG_F64
                          ? launch_variant<ZIG_EXP, double>(k, d_scratch, n, 0, 0, s, dev, b)
                          : launch_variant<ZIG_EXP, float>(k, d_scratch, n, 0, 0, s, dev, b))
                   : (dtype == ZIG_F64
                          ? launch_variant<ZIG_NORMAL, double>(k, d_scratch, n, 0, 0, s, dev, b)
                          : launch_variant<ZIG_NORMAL, float>(k, d_scratch, n, 0, 0, s, dev, b));
      };
      st = launch();
      if (st == ZIG_OK && cudaEventRecord(e0, s) != cudaSuccess) st = ZIG_E_CUDA;
      for (int i = 0; i < reps && st == ZIG_OK; ++i) st = launch();
      float ms = 0.0f;
      if (st == ZIG_OK && (cudaEventRecord(e1, s) != cudaSuccess ||
                           cudaEventSynchronize(e1) != cudaSuccess ||
                           cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        st = ZIG_E_CUDA;
      if (st != ZIG_OK) break;
      const double rate = (double)n * reps / ((double)ms * 1e6);
      if (results && count < max_results) results[count] = variant_entry(dtype, k, b, rate);
      ++count;
      if (rate > best) {
        best = rate;
        best_k = k;
        best_b = b;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != ZIG_OK) {
    cudaGetLastError();
    return st;
  }
  Selection& sel = g_dev[dev].sel[dist][dtype];
  sel.variant.store(best_k);
  sel.bps.store(best_b);
  sel.rate.store(best);
  const zig_tune_entry e = variant_entry(dtype, best_k, best_b, best);
  tune_cache_put(g_dev[dev].name, g_dev[dev].sms, dist, dtype, e);
  if (chosen) *chosen = e;
  if (n_results) *n_results = count;
  return ZIG_OK;
}

zig_status zig_export_tables(zig_dist dist, zig_tables_export* h_out) {
  if (h_out == nullptr || (dist != ZIG_EXP && dist != ZIG_NORMAL)) return ZIG_E_INVAL;
  zig_status st = ensure_host_tables();
  if (st != ZIG_OK) return st;
  *h_out = g_host[dist];
  return ZIG_OK;
}

zig_status zig_export_tables_ex(zig_dist dist, int index_bits, zig_tables_ex* h_out) {
  if (h_out == nullptr || (dist != ZIG_EXP && dist != ZIG_NORMAL) ||
      (index_bits != 8 && index_bits != 10))
    return ZIG_E_INVAL;
  zig_status st = ensure_host_tables();
  if (st != ZIG_OK) return st;
  *h_out = index_bits == 10 ? g_host10[dist] : g_host8ex[dist];
  return ZIG_OK;
}

zig_status zig_exponential(void* out, uint64_t n, uint64_t seed, uint64_t offset,
                           zig_dtype dtype, void* stream) {
  return generate(ZIG_EXP, out, n, seed, offset, dtype, stream);
}

zig_status zig_normal(void* out, uint64_t n, uint64_t seed, uint64_t offset, zig_dtype dtype,
                      void* stream) {
  return generate(ZIG_NORMAL, out, n, seed, offset, dtype, stream);
}

zig_status zig_generate(zig_dist dist, zig_keying keying, int index_bits, void* out, uint64_t n,
                        uint64_t seed, uint64_t offset, zig_dtype dtype, void* stream) {
  return generate(dist, out, n, seed, offset, dtype, stream, keying, index_bits);
}

size_t zig_moments_workspace_bytes(zig_dist dist, zig_dtype dtype) {
  int dev;
  if (current_device(&dev) != ZIG_OK || !g_dev[dev].ready.load(std::memory_order_acquire))
    return 0;
  // enough for either keying
  uint64_t cap, cap2;
  if (dist == ZIG_EXP) {
    cap = dtype == ZIG_F64 ? moment_grid_cap<ZIG_EXP, double>(dev)
                           : moment_grid_cap<ZIG_EXP, float>(dev);
    cap2 = dtype == ZIG_F64 ? moment_grid_cap<ZIG_EXP, double, PackedShape<double>, 1>(dev)
                            : moment_grid_cap<ZIG_EXP, float, PackedShape<float>, 1>(dev);
  } else {
    cap = dtype == ZIG_F64 ? moment_grid_cap<ZIG_NORMAL, double>(dev)
                           : moment_grid_cap<ZIG_NORMAL, float>(dev);
    cap2 = dtype == ZIG_F64 ? moment_grid_cap<ZIG_NORMAL, double, PackedShape<double>, 1>(dev)
                            : moment_grid_cap<ZIG_NORMAL, float, PackedShape<float>, 1>(dev);
  }
  if (cap2 > cap) cap = cap2;
  return kTicketBytes + (size_t)cap * 4 * sizeof(double);
}

zig_status zig_moments(zig_dist dist, zig_dtype dtype, uint64_t n, uint64_t seed,
                       uint64_t offset, double* d_sums, unsigned long long* d_hist,
                       void* d_workspace, size_t workspace_bytes, void* stream) {
  return zig_moments_keyed(dist, dtype, ZIG_KEY_INDEX, n, seed, offset, d_sums, d_hist,
                           d_workspace, workspace_bytes, stream);
}

zig_status zig_moments_keyed(zig_dist dist, zig_dtype dtype, int keying, uint64_t n,
                             uint64_t seed, uint64_t offset, double* d_sums,
                             unsigned long long* d_hist, void* d_workspace,
                             size_t workspace_bytes, void* stream) {
  if (keying != ZIG_KEY_INDEX && keying != ZIG_KEY_PACKED) return ZIG_E_INVAL;
  if (dist != ZIG_EXP && dist != ZIG_NORMAL) return ZIG_E_INVAL;
  if (dtype != ZIG_F32 && dtype != ZIG_F64) return ZIG_E_INVAL;
  if (d_sums == nullptr || d_hist == nullptr || d_workspace == nullptr) return ZIG_E_INVAL;
  if ((uintptr_t)d_sums % 8 || (uintptr_t)d_hist % 8 || (uintptr_t)d_workspace % 8)
    return ZIG_E_ALIGN;
  if (n > 0 && n - 1 > UINT64_MAX - offset) return ZIG_E_RANGE;
  if (n > (UINT64_MAX / 16)) return ZIG_E_RANGE;
  int dev;
  zig_status st = current_device(&dev);
  if (st != ZIG_OK) return st;
  if (!g_dev[dev].ready.load(std::memory_order_acquire)) return ZIG_E_NOTINIT;
  cudaStream_t s = (cudaStream_t)stream;
  if (keying == ZIG_KEY_PACKED) {
    if (dist == ZIG_EXP)
      return dtype == ZIG_F64
                 ? launch_moments<ZIG_EXP, double, PackedShape<double>, 1>(
                       n, seed, offset, d_sums, d_hist, d_workspace, workspace_bytes, s, dev)
                 : launch_moments<ZIG_EXP, float, PackedShape<float>, 1>(
                       n, seed, offset, d_sums, d_hist, d_workspace, workspace_bytes, s, dev);
    return dtype == ZIG_F64
               ? launch_moments<ZIG_NORMAL, double, PackedShape<double>, 1>(
                     n, seed, offset, d_sums, d_hist, d_workspace, workspace_bytes, s, dev)
               : launch_moments<ZIG_NORMAL, float, PackedShape<float>, 1>(
                     n, seed, offset, d_sums, d_hist, d_workspace, workspace_bytes, s, dev);
  }
  if (dist == ZIG_EXP)
    return dtype == ZIG_F64 ? launch_moments<ZIG_EXP, double>(n, seed, offset, d_sums, d_hist,
                                                              d_workspace, workspace_bytes, s, dev)
                            : launch_moments<ZIG_EXP, float>(n, seed, offset, d_sums, d_hist,
                                                             d_workspace, workspace_bytes, s, dev);
  return dtype == ZIG_F64 ? launch_moments<ZIG_NORMAL, double>(n, seed, offset, d_sums, d_hist,
                                                               d_workspace, workspace_bytes, s, dev)
                          : launch_moments<ZIG_NORMAL, float>(n, seed, offset, d_sums, d_hist,
                                                              d_workspace, workspace_bytes, s, dev);
}

zig_status zig_moments_noalloc(zig_dist dist, zig_dtype dtype, uint64_t n, uint64_t seed,
                               uint64_t offset, double* d_sums, unsigned long long* d_hist,
                               void* stream) {
  int dev;
  zig_status st = current_device(&dev);
  if (st != ZIG_OK) return st;
  if (!g_dev[dev].ready.load(std::memory_order_acquire)) return ZIG_E_NOTINIT;
  const size_t need = zig_moments_workspace_bytes(dist, dtype);
  if (need == 0) return ZIG_E_INVAL;
  if (need > kStaticScratchBytes) return ZIG_E_NOMEM;  // device needs more blocks than it holds
  return zig_moments(dist, dtype, n, seed, offset, d_sums, d_hist,
                     g_dev[dev].d_static_scratch, kStaticScratchBytes, stream);
}

size_t zig_batch_workspace_bytes(uint32_t count) { return batch_ws_bytes(count); }

zig_status zig_batch_validate(const zig_request* h_reqs, uint32_t count) {
  if (count > 0 && h_reqs == nullptr) return ZIG_E_INVAL;
  if (count >= (1u << kBatchReqBits)) return ZIG_E_RANGE;
  for (uint32_t r = 0; r < count; ++r) {
    const zig_status st = check_request(h_reqs[r]);
    if (st != ZIG_OK) return st;
  }
  return ZIG_OK;
}

zig_status zig_batch(const zig_request* d_reqs, uint32_t count, unsigned long long* d_done_ns,
                     void* d_workspace, size_t workspace_bytes, void* stream) {
  if (count == 0) return ZIG_OK;
  int dev;
  const zig_status st = batch_args(d_reqs, count, d_done_ns, d_workspace, workspace_bytes, &dev);
  if (st != ZIG_OK) return st;
  return launch_batch(d_reqs, count, d_done_ns, d_workspace, (cudaStream_t)stream, dev,
                      g_dev[dev].batch_chunk.load(std::memory_order_relaxed));
}

zig_status zig_batch_autotune(const zig_request* d_reqs, uint32_t count, void* d_workspace,
                              size_t workspace_bytes, int reps, void* stream,
                              zig_batch_tune_entry* results, int max_results, int* n_results,
                              uint32_t* chosen_chunk) {
  if (count == 0 || reps < 1 || reps > 100) return ZIG_E_INVAL;
  int dev;
  zig_status st = batch_args(d_reqs, count, nullptr, d_workspace, workspace_bytes, &dev);
  if (st != ZIG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return ZIG_E_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return ZIG_E_CUDA;
  }
  uint32_t best = kBatchChunkDefault;
  float best_ms = -1.0f;
  for (int k = 0; k < kBatchChunks && st == ZIG_OK; ++k) {
    const uint32_t c = kBatchChunkCand[k];
    st = launch_batch(d_reqs, count, nullptr, d_workspace, s, dev, c);  // warm-up
    if (st == ZIG_OK && cudaEventRecord(e0, s) != cudaSuccess) st = ZIG_E_CUDA;
    for (int i = 0; i < reps && st == ZIG_OK; ++i)
      st = launch_batch(d_reqs, count, nullptr, d_workspace, s, dev, c);
    float ms = 0.0f;
    if (st == ZIG_OK && (cudaEventRecord(e1, s) != cudaSuccess ||
                         cudaEventSynchronize(e1) != cudaSuccess ||
                         cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      st = ZIG_E_CUDA;
    if (st != ZIG_OK) break;
    ms /= (float)reps;
    if (results && k < max_results) results[k] = zig_batch_tune_entry{c, (double)ms};
    if (best_ms < 0.0f || ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != ZIG_OK) {
    cudaGetLastError();
    return st;
  }
  g_dev[dev].batch_chunk.store(best);
  if (chosen_chunk) *chosen_chunk = best;
  if (n_results) *n_results = kBatchChunks;
  return ZIG_OK;
}

zig_status zig_batch_set_chunk(uint32_t chunk) {
  if (chunk < 1 || chunk > 4096) return ZIG_E_INVAL;
  int dev;
  const zig_status st = current_device(&dev);
  if (st != ZIG_OK) return st;
  g_dev[dev].batch_chunk.store(chunk);
  return ZIG_OK;
}

uint32_t zig_batch_get_chunk(void) {
  int dev;
  if (current_device(&dev) != ZIG_OK) return 0;
  return g_dev[dev].batch_chunk.load();
}

zig_status zig_status_poll(void* stream) {
  int dev;
  zig_status st = current_device(&dev);
  if (st != ZIG_OK) return st;
  if (!g_dev[dev].ready.load(std::memory_order_acquire)) return ZIG_E_NOTINIT;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned int h = 0;
  const unsigned slot = g_dev[dev].poll_seq.fetch_add(1u) % kPollSlots;
  status_take_kernel<<<1, 1, 0, s>>>(slot);
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyFromSymbolAsync(&h, g_status_taken, sizeof(h), slot * sizeof(h),
                                cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return ZIG_E_CUDA;
  }
  if (h & kWaitBit) return ZIG_E_TIMEOUT;
  if (h & kBatchInvalidBit) return ZIG_E_INVAL;
  if (h & kLoopLimitBit) return ZIG_E_LOOP_LIMIT;
  return ZIG_OK;
}

zig_status zig_set_fringe_limits(int max_attempts, int max_tail) {
  if (max_attempts < 1 || max_attempts > (1 << 20) || max_tail < 0 || max_tail > (1 << 20))
    return ZIG_E_INVAL;
  g_max_att.store(max_attempts);
  g_max_tail.store(max_tail);
  return ZIG_OK;
}

}  // extern "C"
