// zig_gen.cu -- sm_103a kernels and C ABI for the modified ziggurat.
//
// McFarland, arXiv:1403.6870, Table 1 (modified column):
//   1. generate U_1 and i;  2. if i < L_max return U_1 X_i;
//   3. generate j from A;   4. if j = 0 return a value from the tail;
//   5-8. rejection-sample the overhang box j.
// Steps 1-2 are the common case (98.4% exponential, 98.8% normal).  On the
// GPU every thread runs steps 1-2 for a fixed run of outputs with no
// divergence: the Philox block, the word split, one shared-memory lookup of
// X_i and one fused multiply-add, then one vector store.  A draw with
// i >= L_max is only *recorded*: the warp ballots its fringe lanes into a
// per-CTA shared-memory queue of output positions.  When the queue holds a
// full CTA's worth of work (and at the end), every thread pops one position
// and runs the whole algorithm for it from its counter (steps 1-8 with the
// tail and overhang loops), then overwrites that output.  The fast path
// therefore never diverges and the fringe runs with all lanes busy.
//
// Compiled with --fmad=false: every fused multiply-add below is written as
// one, everything else is rounded per operation, exactly as the algorithm's
// readings state.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "zig_internal.h"

namespace zig {

// ---------------------------------------------------------------------------
// Device tables (one set per distribution; index = zig_dist)
// ---------------------------------------------------------------------------
struct DevTab {
  double X[256];   // X_i; entries beyond L_max are zero (never returned)
  double f[257];   // heights f_0..f_L (normal: unnormalised)
  double dX[257];  // X_{j-1} - X_j
  double df[257];  // f_j - f_{j-1}
  float X32[256];
  float f32[257];
  float dX32[257];
  float df32[257];
  unsigned long long T[256];  // alias thresholds (56-bit scale)
  unsigned char alias[256];
  double tau;   // exponential always-accept bound on ux + uy
  double rinv;  // RN64(1 / X_0)
  float rinv32;
  int L;
};

__device__ DevTab g_tab[2];
__device__ unsigned int g_status;

constexpr unsigned kLoopLimitBit = 1u << ZIG_E_LOOP_LIMIT;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------
constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
constexpr uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox10(uint32_t c0, uint32_t c1, uint32_t c2,
                                          uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)kM0 * c0;
    const uint64_t p1 = (uint64_t)kM1 * c2;
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

__device__ __forceinline__ uint64_t pack(uint32_t lo, uint32_t hi) {
  return (uint64_t)lo | ((uint64_t)hi << 32);
}

// Word stream of one counter g: block k = Philox((g_lo, g_hi, 0, k), key);
// words r0|r1<<32 then r2|r3<<32.
struct Words {
  uint32_t glo, ghi, k0, k1, blk, r2, r3;
  bool half;
  __device__ Words(uint64_t seed, uint64_t g)
      : glo((uint32_t)g), ghi((uint32_t)(g >> 32)), k0((uint32_t)seed),
        k1((uint32_t)(seed >> 32)), blk(0), r2(0), r3(0), half(false) {}
  __device__ uint64_t next() {
    if (!half) {
      const uint4 r = philox10(glo, ghi, 0u, blk, k0, k1);
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

// ---------------------------------------------------------------------------
// Precision traits: U from a word, table access, explicit FMA
// ---------------------------------------------------------------------------
template <typename T>
struct Prec;

template <>
struct Prec<double> {
  // U = (w >> 12) 2^-52, formed as (1 + U) from the bits, minus 1 (exact).
  static __device__ __forceinline__ double one_plus_u(uint32_t lo, uint32_t hi) {
    return __hiloint2double((int)(0x3FF00000u | (hi >> 12)),
                            (int)__funnelshift_r(lo, hi, 12));
  }
  static __device__ __forceinline__ double U(uint64_t w) {
    return __dsub_rn(one_plus_u((uint32_t)w, (uint32_t)(w >> 32)), 1.0);
  }
  static __device__ __forceinline__ double fmat(double a, double b, double c) {
    return __fma_rn(a, b, c);
  }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double X(const DevTab& t, int i) { return t.X[i]; }
  static __device__ __forceinline__ double f(const DevTab& t, int i) { return t.f[i]; }
  static __device__ __forceinline__ double dX(const DevTab& t, int i) { return t.dX[i]; }
  static __device__ __forceinline__ double df(const DevTab& t, int i) { return t.df[i]; }
  static __device__ __forceinline__ double rinv(const DevTab& t) { return t.rinv; }
  static __device__ __forceinline__ double nan() { return __longlong_as_double(0x7FF8000000000000ll); }
  static __device__ __forceinline__ double neg(double x) { return -x; }
};

template <>
struct Prec<float> {
  // U = (w >> 41) 2^-23 (top 23 bits), formed as (1 + U) minus 1.
  static __device__ __forceinline__ float one_plus_u(uint32_t, uint32_t hi) {
    return __int_as_float((int)(0x3F800000u | (hi >> 9)));
  }
  static __device__ __forceinline__ float U(uint64_t w) {
    return __fsub_rn(one_plus_u(0u, (uint32_t)(w >> 32)), 1.0f);
  }
  static __device__ __forceinline__ float fmat(float a, float b, float c) {
    return __fmaf_rn(a, b, c);
  }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float X(const DevTab& t, int i) { return t.X32[i]; }
  static __device__ __forceinline__ float f(const DevTab& t, int i) { return t.f32[i]; }
  static __device__ __forceinline__ float dX(const DevTab& t, int i) { return t.dX32[i]; }
  static __device__ __forceinline__ float df(const DevTab& t, int i) { return t.df32[i]; }
  static __device__ __forceinline__ float rinv(const DevTab& t) { return t.rinv32; }
  static __device__ __forceinline__ float nan() { return __int_as_float(0x7FC00000); }
  static __device__ __forceinline__ float neg(float x) { return -x; }
};

// Step 3: j from the alias table.  Column c = bits 0-7, threshold = bits
// 8-63; j = c when the threshold is below T_c, else alias_c.
__device__ __forceinline__ int alias_pick(const DevTab& t, uint64_t w) {
  const int c = (int)(w & 0xFFu);
  return (w >> 8) < t.T[c] ? c : (int)t.alias[c];
}

struct Limits {
  int max_att;
  int max_tail;
};

// Full Table 1 for the exponential from word stream w (the general path).
// Step 4 uses memorylessness: a tail draw is X_0 plus a fresh exponential,
// evaluated innermost first, so depth d adds X_0 d times after the final
// draw.  Steps 5-8 keep j on rejection and draw fresh (ux, uy); the first
// attempt reuses U_1 as ux (its bits are disjoint from i).
template <typename T>
__device__ T exp_general(Words& w, const DevTab& t, Limits lim, bool& err) {
  typedef Prec<T> P;
  int depth = 0;
  T x;
  for (;;) {
    const uint64_t w0 = w.next();
    const int i = (int)(w0 & 0xFFu);
    const T U1 = P::U(w0);
    if (i < t.L) {
      x = P::mul(U1, P::X(t, i));
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
    T ux = U1;
    for (int att = 1;; ++att) {
      T uy = P::U(w.next());
      // Above the chord never lies under the convex e^-x: reflect through
      // the anti-diagonal (Appendix C item 5).
      if (P::add(ux, uy) > (T)1) {
        const T nx = P::add((T)1, -uy), ny = P::add((T)1, -ux);
        ux = nx;
        uy = ny;
      }
      const T xx = P::fmat(ux, P::dX(t, j), P::X(t, j));
      // Below the chord by more than eps: under P without a test.
      if ((double)P::add(ux, uy) < t.tau) {
        x = xx;
        break;
      }
      const T y = P::fmat(uy, P::df(t, j), P::f(t, j - 1));
      if ((double)y < exp(-(double)xx)) {
        x = xx;
        break;
      }
      if (att >= lim.max_att) {
        err = true;
        return P::nan();
      }
      ux = P::U(w.next());
    }
    break;
  }
  for (int d = 0; d < depth; ++d) x = P::add(P::X(t, 0), x);
  return x;
}

// Full Table 1 for the normal: sign from bit 8 of the first word; the tail
// beyond X_0 by Marsaglia-Tsang from two exponential draws (a = E_1 / X_0,
// accept when 2 E_2 > a^2, return X_0 + a); overhangs by plain rejection
// y < e^{-x^2/2}, keeping j and redrawing both uniforms.
template <typename T>
__device__ T normal_general(Words& w, const DevTab& te, const DevTab& tn, Limits lim,
                            bool& err) {
  typedef Prec<T> P;
  const uint64_t w0 = w.next();
  const int i = (int)(w0 & 0xFFu);
  const bool negative = ((w0 >> 8) & 1u) != 0;
  const T U1 = P::U(w0);
  T x;
  if (i < tn.L) {
    x = P::mul(U1, P::X(tn, i));
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
      T ux = U1;
      for (int att = 1;; ++att) {
        const T uy = P::U(w.next());
        const T xx = P::fmat(ux, P::dX(tn, j), P::X(tn, j));
        const T y = P::fmat(uy, P::df(tn, j), P::f(tn, j - 1));
        const double xd = (double)xx;
        if ((double)y < exp(-__dmul_rn(__dmul_rn(xd, xd), 0.5))) {
          x = xx;
          break;
        }
        if (att >= lim.max_att) {
          err = true;
          return P::nan();
        }
        ux = P::U(w.next());
      }
    }
  }
  return negative ? P::neg(x) : x;
}

template <int DIST, typename T>
__device__ __noinline__ T sample_general(uint64_t seed, uint64_t g, Limits lim) {
  Words w(seed, g);
  bool err = false;
  T x = (DIST == ZIG_EXP) ? exp_general<T>(w, g_tab[ZIG_EXP], lim, err)
                          : normal_general<T>(w, g_tab[ZIG_EXP], g_tab[ZIG_NORMAL], lim, err);
  if (err) atomicOr(&g_status, kLoopLimitBit);
  return x;
}

// ---------------------------------------------------------------------------
// Fast path (steps 1-2) and vector stores
// ---------------------------------------------------------------------------
// x = RN(U X_i) computed as fma(1 + U, X_i, -X_i): (1 + U) X_i - X_i equals
// U X_i exactly, and the FMA rounds once.  The normal's sign (bit 8) is
// applied to the result's sign bit.
template <int DIST, typename T>
__device__ __forceinline__ T fast_value(uint32_t lo, uint32_t hi, const T* sX);

template <>
__device__ __forceinline__ double fast_value<ZIG_EXP, double>(uint32_t lo, uint32_t hi,
                                                              const double* sX) {
  const double X = sX[lo & 0xFFu];
  return __fma_rn(Prec<double>::one_plus_u(lo, hi), X, -X);
}
template <>
__device__ __forceinline__ double fast_value<ZIG_NORMAL, double>(uint32_t lo, uint32_t hi,
                                                                 const double* sX) {
  const double X = sX[lo & 0xFFu];
  const double x = __fma_rn(Prec<double>::one_plus_u(lo, hi), X, -X);
  return __hiloint2double(__double2hiint(x) ^ (int)((lo & 0x100u) << 23), __double2loint(x));
}
template <>
__device__ __forceinline__ float fast_value<ZIG_EXP, float>(uint32_t lo, uint32_t hi,
                                                            const float* sX) {
  const float X = sX[lo & 0xFFu];
  return __fmaf_rn(Prec<float>::one_plus_u(lo, hi), X, -X);
}
template <>
__device__ __forceinline__ float fast_value<ZIG_NORMAL, float>(uint32_t lo, uint32_t hi,
                                                               const float* sX) {
  const float X = sX[lo & 0xFFu];
  const float x = __fmaf_rn(Prec<float>::one_plus_u(lo, hi), X, -X);
  return __int_as_float(__float_as_int(x) ^ (int)((lo & 0x100u) << 23));
}

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

constexpr int kThreads = 256;

template <typename T>
struct GenShape;
template <>
struct GenShape<double> {
  static constexpr int V = 2, R = 2;
};
template <>
struct GenShape<float> {
  static constexpr int V = 4, R = 2;
};

// One launch fills out[0, n): a head of < V elements up to the first
// V-element-aligned address, nvec aligned V-vectors, then a tail.  Head and
// tail go through the general path (queued by CTA 0).
template <int DIST, typename T>
__global__ void __launch_bounds__(kThreads) gen_kernel(T* __restrict__ out, uint64_t n,
                                                       uint32_t head, uint64_t nvec,
                                                       uint64_t seed, uint64_t offset,
                                                       Limits lim) {
  constexpr int V = GenShape<T>::V, R = GenShape<T>::R;
  constexpr int kTile = kThreads * R;  // vectors per tile
  constexpr int kQcap = kThreads * (V * R + 1);
  __shared__ T sX[256];
  __shared__ uint64_t sQ[kQcap];
  __shared__ int sQn;

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  for (int k = tid; k < 256; k += kThreads) sX[k] = Prec<T>::X(g_tab[DIST], k);
  if (tid == 0) sQn = 0;
  __syncthreads();
  const uint32_t L = (uint32_t)g_tab[DIST].L;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const uint64_t body_end = head + nvec * V;
  if (blockIdx.x == 0) {
    if ((uint32_t)tid < head) sQ[atomicAdd(&sQn, 1)] = (uint64_t)tid;
    if ((uint64_t)tid < n - body_end) sQ[atomicAdd(&sQn, 1)] = body_end + (uint64_t)tid;
  }
  const unsigned lt_mask = (1u << lane) - 1u;
  T* body = out + head;
  const uint64_t ntiles = (nvec + kTile - 1) / kTile;

  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint64_t vi = tile * kTile + (uint64_t)(r * kThreads + tid);
      const bool valid = vi < nvec;
      T v[V];
#pragma unroll
      for (int k = 0; k < V; ++k) {
        const uint64_t p = head + vi * V + (uint64_t)k;
        const uint64_t g = offset + p;
        // Step 1: block 0 of counter g; word 0 = r0 | r1 << 32.
        const uint4 b = philox10((uint32_t)g, (uint32_t)(g >> 32), 0u, 0u, k0, k1);
        // Step 2 for every lane; lanes with i >= L_max are queued.
        v[k] = fast_value<DIST, T>(b.x, b.y, sX);
        const bool fringe = valid && (b.x & 0xFFu) >= L;
        const unsigned m = __ballot_sync(0xFFFFFFFFu, fringe);
        if (m) {
          const int leader = __ffs(m) - 1;
          int base = 0;
          if (lane == leader) base = atomicAdd(&sQn, __popc(m));
          base = __shfl_sync(0xFFFFFFFFu, base, leader);
          if (fringe) sQ[base + __popc(m & lt_mask)] = p;
        }
      }
      if (valid) VecStore<T, V>::st(body + vi * V, v);
    }
    __syncthreads();
    int qn = sQn;
    while (qn >= kThreads) {
      const uint64_t p = sQ[qn - kThreads + tid];
      __syncthreads();
      if (tid == 0) sQn = qn - kThreads;
      qn -= kThreads;
      out[p] = sample_general<DIST, T>(seed, offset + p, lim);
    }
    __syncthreads();
  }
  __syncthreads();
  const int qn = sQn;
  for (int base = 0; base < qn; base += kThreads) {
    if (base + tid < qn) {
      const uint64_t p = sQ[base + tid];
      out[p] = sample_general<DIST, T>(seed, offset + p, lim);
    }
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

constexpr int kMaxDevices = 64;

std::mutex g_mu;
zig_tables_export g_host[2];
std::atomic<bool> g_host_ready{false};
std::atomic<int> g_max_att{64};
std::atomic<int> g_max_tail{16};

struct DeviceState {
  std::atomic<bool> ready{false};
  unsigned int* d_status = nullptr;
  int sms = 0;
};
DeviceState g_dev[kMaxDevices];

zig_status ensure_host_tables() {
  if (g_host_ready.load(std::memory_order_acquire)) return ZIG_OK;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_host_ready.load()) return ZIG_OK;
  if (build_host_tables(&g_host[0], &g_host[1]) != 0) return ZIG_E_TABLE;
  g_host_ready.store(true, std::memory_order_release);
  return ZIG_OK;
}

void to_device_layout(const zig_tables_export& h, DevTab* d) {
  std::memset(d, 0, sizeof(*d));
  for (int k = 0; k <= h.L && k < 256; ++k) {
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
  for (int c = 0; c < 256; ++c) {
    d->T[c] = h.T[c];
    d->alias[c] = h.alias[c];
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

template <int DIST, typename T>
int occupancy_blocks(int dev) {
  static std::atomic<int> cache[kMaxDevices];
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gen_kernel<DIST, T>, kThreads, 0) !=
          cudaSuccess ||
      occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  cache[dev].store(occ, std::memory_order_relaxed);
  return occ;
}

template <int DIST, typename T>
zig_status launch_gen(void* out, uint64_t n, uint64_t seed, uint64_t offset,
                      cudaStream_t stream, int dev) {
  constexpr int V = GenShape<T>::V, R = GenShape<T>::R;
  const uintptr_t addr = (uintptr_t)out;
  const uint64_t align_elems = (uint64_t)((V - (addr / sizeof(T)) % V) % V);
  const uint64_t head = align_elems < n ? align_elems : n;
  const uint64_t nvec = (n - head) / V;
  const uint64_t tiles = (nvec + (uint64_t)kThreads * R - 1) / ((uint64_t)kThreads * R);
  const uint64_t cap = (uint64_t)g_dev[dev].sms * (uint64_t)occupancy_blocks<DIST, T>(dev);
  uint64_t grid = tiles < cap ? tiles : cap;
  if (grid < 1) grid = 1;
  Limits lim{g_max_att.load(), g_max_tail.load()};
  gen_kernel<DIST, T><<<(unsigned)grid, kThreads, 0, stream>>>(
      (T*)out, n, (uint32_t)head, nvec, seed, offset, lim);
  if (cudaGetLastError() != cudaSuccess) return ZIG_E_CUDA;
  return ZIG_OK;
}

zig_status generate(int dist, void* out, uint64_t n, uint64_t seed, uint64_t offset,
                    zig_dtype dtype, void* stream) {
  if (dtype != ZIG_F32 && dtype != ZIG_F64) return ZIG_E_INVAL;
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
  cudaStream_t s = (cudaStream_t)stream;
  if (dist == ZIG_EXP)
    return dtype == ZIG_F64 ? launch_gen<ZIG_EXP, double>(out, n, seed, offset, s, dev)
                            : launch_gen<ZIG_EXP, float>(out, n, seed, offset, s, dev);
  return dtype == ZIG_F64 ? launch_gen<ZIG_NORMAL, double>(out, n, seed, offset, s, dev)
                          : launch_gen<ZIG_NORMAL, float>(out, n, seed, offset, s, dev);
}

}  // namespace

const zig_tables_export* host_tables(int dist) {
  if (ensure_host_tables() != ZIG_OK) return nullptr;
  return &g_host[dist];
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
  to_device_layout(g_host[0], &h[0]);
  to_device_layout(g_host[1], &h[1]);
  void* status = nullptr;
  int sms = 0;
  if (cudaMemcpyToSymbol(g_tab, h, sizeof(h)) != cudaSuccess ||
      cudaGetSymbolAddress(&status, g_status) != cudaSuccess ||
      cudaMemset(status, 0, sizeof(unsigned int)) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return ZIG_E_CUDA;
  }
  g_dev[dev].d_status = (unsigned int*)status;
  g_dev[dev].sms = sms;
  g_dev[dev].ready.store(true, std::memory_order_release);
  return ZIG_OK;
}

zig_status zig_export_tables(zig_dist dist, zig_tables_export* h_out) {
  if (h_out == nullptr || (dist != ZIG_EXP && dist != ZIG_NORMAL)) return ZIG_E_INVAL;
  zig_status st = ensure_host_tables();
  if (st != ZIG_OK) return st;
  *h_out = g_host[dist];
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

zig_status zig_status_poll(void* stream) {
  int dev;
  zig_status st = current_device(&dev);
  if (st != ZIG_OK) return st;
  if (!g_dev[dev].ready.load(std::memory_order_acquire)) return ZIG_E_NOTINIT;
  unsigned int h = 0;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess ||
      cudaMemcpy(&h, g_dev[dev].d_status, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(g_dev[dev].d_status, 0, sizeof(h)) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return ZIG_E_CUDA;
  }
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
