// zig_batch.cuh -- one persistent launch for many generation requests.
// Included by zig_gen.cu (shares its tables, sinks and fringe stages).
//
// Each request r asks for n_r variates of its own distribution, precision,
// Philox key (seed_r), counter offset and parameters (exponential rate
// lambda; normal mean mu and standard deviation sigma).  A prep kernel
// splits every request into the tiles zig_exponential / zig_normal would
// use for it, lays the tiles of all requests end to end in request order,
// and cuts that sequence into one contiguous range per SM.  The CTAs of an
// SM claim chunks of tiles (a launch parameter, picked by zig_batch_autotune)
// from their SM's range, so co-resident
// CTAs work on neighbouring tiles (mostly the same request, hence the same
// instruction stream); a CTA whose range is exhausted claims chunks from the
// other ranges in turn.  The tiles of one request inside a chunk form a
// session: all eight warps run the plain kernel's code for the request's
// (dist, dtype) with its key, offset and transform in registers, and meet at
// a barrier once each has finished its fringe draws.  A counter per request
// (its tiles not yet finished) reaches zero when the request is complete;
// the CTA that completes it records %globaltimer minus the batch start.
#ifndef ZIG_BATCH_CUH
#define ZIG_BATCH_CUH

namespace zig {

constexpr int kBatchReqBits = 23;  // requests per batch: below 2^23
constexpr int kBatchPosBits = 40;  // variates per request: below 2^40
constexpr unsigned kBatchInvalidBit = 1u << 10;  // status bit: a request was rejected

// Per-request derived state (workspace).
struct alignas(16) BatchReq {
  uint64_t out;     // device address of the output
  uint64_t seed;
  uint64_t offset;
  uint64_t n;
  uint64_t head;    // elements before the first vector-aligned one
  uint64_t nvec;    // aligned vectors of the body
  uint64_t tile0;   // first global tile
  double a64, b64;  // FP64 transform: exp x*a, normal fma(a, x, b)
  float a32, b32;   // FP32 transform
  uint32_t cls;     // dist | dtype << 1
  uint32_t ntiles;  // tiles of this request (>= 1 when n > 0)
  unsigned long long remaining;  // outstanding units
};

struct BatchHeader {
  uint64_t total_tiles;
  unsigned long long t_start;
  unsigned long long* done_ns;  // completion times (nullable), this batch's own
  uint32_t count;
  uint32_t nranges;        // tile ranges, one per SM
  unsigned range_counter;  // ranges handed to SMs so far
  uint32_t chunk;          // tiles per claim
};

// A tile range of the sequence and its claim cursor.
struct BatchRange {
  unsigned long long cursor;  // next unclaimed tile
  uint64_t end;
};

constexpr int kBatchMaxRanges = 1024;
constexpr int kBatchSmSlots = 1024;  // SM id -> range (by %smid)
// Tiles per claim: the candidates zig_batch_autotune times, and the
// default (measured on GB300 on the 4096-request mix: 16 tiles 10.40 ms,
// 32 tiles 9.95 ms, 128 tiles 9.89 ms, 64 tiles 9.82 ms).
constexpr int kBatchChunks = 4;
constexpr uint32_t kBatchChunkCand[kBatchChunks] = {64, 32, 128, 16};
constexpr uint32_t kBatchChunkDefault = 64;

__host__ __device__ constexpr size_t batch_header_bytes() { return 256; }
static_assert(sizeof(BatchHeader) <= 256, "the header fits its slot of the workspace");
// workspace: header, request states, ranges, SM map
__host__ __device__ constexpr size_t batch_ranges_offset(uint32_t count) {
  return batch_header_bytes() + (((size_t)count * sizeof(BatchReq) + 255) / 256) * 256;
}
__host__ __device__ constexpr size_t batch_smmap_offset(uint32_t count) {
  return batch_ranges_offset(count) + kBatchMaxRanges * sizeof(BatchRange);
}
__host__ __device__ constexpr size_t batch_workspace_total(uint32_t count) {
  return batch_smmap_offset(count) + kBatchSmSlots * sizeof(int);
}

// Shared state of one batch CTA: X_i of both distributions in both
// precisions and the warps' fringe queues (the members gen_tiles uses).
struct BatchCtaState {
  double sX64[2][256];
  float sX32[2][256];
  // the session's folded fast-path tables (+-B_i, D by i | sign << 8)
  double sB64[512], sD64[512];
  float sB32[512], sD32[512];
  WarpQueues wq[kWarps];
};

template <typename T>
__device__ __forceinline__ const T* batch_sx(const BatchCtaState& sh, int dist);
template <>
__device__ __forceinline__ const double* batch_sx<double>(const BatchCtaState& sh, int dist) {
  return sh.sX64[dist];
}
template <>
__device__ __forceinline__ const float* batch_sx<float>(const BatchCtaState& sh, int dist) {
  return sh.sX32[dist];
}
__device__ __forceinline__ double* batch_sb(BatchCtaState& sh, double) { return sh.sB64; }
__device__ __forceinline__ double* batch_sd(BatchCtaState& sh, double) { return sh.sD64; }
__device__ __forceinline__ float* batch_sb(BatchCtaState& sh, float) { return sh.sB32; }
__device__ __forceinline__ float* batch_sd(BatchCtaState& sh, float) { return sh.sD32; }

// Sink of one request: store like StoreSink (vector vi at element
// head + vi V, fringe outputs at their position).  Step 2's values arrive
// already mapped (kAffine: the producers use the session's sB/sD tables);
// the fringe stages' variates are transformed here.
template <int DIST, typename T>
struct BatchSink {
  T* out;
  uint64_t head;
  T a, b;
  const T* sB;
  const T* sD;
  static constexpr bool kReduce = false;
  static constexpr bool kAffine = true;
  __device__ __forceinline__ T tr(T x) const {
    return DIST == ZIG_EXP ? Prec<T>::mul(x, a) : Prec<T>::fmat(a, x, b);
  }
  template <int V>
  __device__ __forceinline__ void vec(uint64_t vi, const T* v, unsigned) {
    VecStore<T, V>::st(out + head + vi * V, v);
  }
  __device__ __forceinline__ void tile_end() {}
  __device__ __forceinline__ void put(uint64_t p, T x) { out[p] = tr(x); }
  __device__ __forceinline__ void put_mapped(uint64_t p, T y) { out[p] = y; }
};

// Subtract `tiles` finished tiles from request r's outstanding count;
// the CTA that brings it to zero records the completion time, against the
// start and into the array that the batch's own header holds (batches on
// other streams have headers of their own).  The caller has made the run's
// outputs visible (fence) before.
__device__ __forceinline__ void settle(const BatchHeader* hdr, BatchReq* reqs, uint32_t r,
                                       unsigned long long tiles) {
  const unsigned long long old =
      atomicAdd(&reqs[r].remaining, (unsigned long long)(-(long long)tiles));
  if (old == tiles && hdr->done_ns) hdr->done_ns[r] = globaltimer() - hdr->t_start;
}

// Prep: derived request state and the exclusive prefix of tile counts
// (one CTA).  Requests that break the batch limits are counted as done with
// no output and flagged in the status word.
__global__ void __launch_bounds__(1024) batch_prep_kernel(const zig_request* __restrict__ in,
                                                           uint32_t count, BatchReq* reqs,
                                                           BatchHeader* hdr,
                                                           unsigned long long* done_ns,
                                                           uint32_t nranges, uint32_t chunk) {
  __shared__ uint64_t part[1024];
  const int tid = threadIdx.x;
  const uint32_t per = (count + 1023u) / 1024u;
  const uint32_t r0 = tid * per, r1 = min(count, r0 + per);
  uint64_t sum = 0;
  for (uint32_t r = r0; r < r1; ++r) {
    const zig_request q = in[r];
    BatchReq b;
    memset(&b, 0, sizeof(b));
    const bool f64 = q.dtype == ZIG_F64;
    const int es = f64 ? 8 : 4;
    const int V = f64 ? GenShape<double>::V : GenShape<float>::V;
    const uint64_t tilev = (uint64_t)kPThreads * (f64 ? GenShape<double>::R : GenShape<float>::R);
    bool ok = (q.dist == ZIG_EXP || q.dist == ZIG_NORMAL) && (q.dtype == ZIG_F32 || f64) &&
              q.n < (1ull << kBatchPosBits) && (q.n == 0 || q.out != nullptr) &&
              (uintptr_t)q.out % es == 0 && (q.n == 0 || q.n - 1 <= ~0ull - q.offset);
    if (q.dist == ZIG_EXP) ok = ok && q.p0 > 0.0 && q.p0 < INFINITY;
    if (q.dist == ZIG_NORMAL) ok = ok && q.p1 > 0.0 && q.p1 < INFINITY && fabs(q.p0) < INFINITY;
    if (!ok) atomicOr(&g_status, kBatchInvalidBit);
    b.out = (uint64_t)q.out;
    b.seed = q.seed;
    b.offset = q.offset;
    b.n = ok ? q.n : 0;
    b.cls = q.dist | (q.dtype << 1);
    if (q.dist == ZIG_EXP) {
      b.a64 = __drcp_rn(q.p0);           // RN(1 / lambda)
      b.a32 = __double2float_rn(b.a64);  // RN32 of it
    } else {
      b.a64 = q.p1;
      b.b64 = q.p0;
      b.a32 = __double2float_rn(q.p1);
      b.b32 = __double2float_rn(q.p0);
    }
    if (b.n > 0) {
      const uint64_t align = (uint64_t)((V - ((uint64_t)q.out / es) % V) % V);
      b.head = align < b.n ? align : b.n;
      b.nvec = (b.n - b.head) / V;
      const uint64_t t = (b.nvec + tilev - 1) / tilev;
      b.ntiles = (uint32_t)(t > 0 ? t : 1);
      b.remaining = b.ntiles;
    } else if (done_ns) {
      done_ns[r] = 0;
    }
    b.tile0 = sum;
    sum += b.ntiles;
    reqs[r] = b;
  }
  part[tid] = sum;
  __syncthreads();
  // exclusive scan of the per-thread tile totals (1024 entries, one thread:
  // the prep is latency-bound anyway and runs once per batch)
  if (tid == 0) {
    uint64_t acc = 0;
    for (int k = 0; k < 1024; ++k) {
      const uint64_t v = part[k];
      part[k] = acc;
      acc += v;
    }
    hdr->total_tiles = acc;
    hdr->count = count;
    hdr->nranges = nranges;
    hdr->range_counter = 0u;
    hdr->chunk = chunk;
  }
  __syncthreads();
  for (uint32_t r = r0; r < r1; ++r) reqs[r].tile0 += part[tid];
  {
    const uint64_t total = hdr->total_tiles;
    BatchRange* rng = (BatchRange*)((char*)hdr + batch_ranges_offset(count));
    int* smmap = (int*)((char*)hdr + batch_smmap_offset(count));
    for (uint32_t i = tid; i < nranges; i += 1024) {
      rng[i].cursor = total * i / nranges;
      rng[i].end = total * (i + 1) / nranges;
    }
    for (int k = tid; k < kBatchSmSlots; k += 1024) smmap[k] = -1;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const unsigned long long t = globaltimer();
    hdr->done_ns = done_ns;
    hdr->t_start = t;
  }
}

// Request of global tile t: the last r with tile0[r] <= t (requests with
// no tiles are skipped automatically since they share tile0 with the next).
__device__ __forceinline__ uint32_t find_request(const BatchReq* reqs, uint32_t count,
                                                 uint64_t t) {
  uint32_t lo = 0, hi = count;  // invariant: tile0[lo] <= t < tile0[hi] (hi virtual)
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) / 2;
    if (reqs[mid].tile0 <= t)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// The batch's tile shape: the default one without interleaved vectors (the
// batch kernel's register budget is set for 2 CTAs per SM; measured).
template <typename T>
using BatchShape = Shape<GenShape<T>::V, GenShape<T>::R, GenShape<T>::MB, 1>;

// One session: tiles [t0, t1) of request r, by the whole CTA, class known
// at compile time.  On return this thread's warp has finished its outputs
// of the session (the warps have not synchronised).
#ifndef ZIG_BATCH_RUN_ATTR
#define ZIG_BATCH_RUN_ATTR __forceinline__
#endif
template <int DIST, typename T>
__device__ ZIG_BATCH_RUN_ATTR void batch_run(BatchCtaState& sh, const BatchReq* reqs, uint32_t r,
                                           uint64_t t0, uint64_t t1, Limits lim) {
  const BatchReq& q = reqs[r];
  BatchSink<DIST, T> sink;
  sink.out = (T*)q.out;
  sink.head = q.head;
  sink.a = sizeof(T) == 8 ? (T)q.a64 : (T)q.a32;
  sink.b = sizeof(T) == 8 ? (T)q.b64 : (T)q.b32;
  const uint64_t seed = q.seed, tile0 = q.tile0;
  // the request's folded fast-path tables: B_i = RN(s X_i), D = RN(m -+ B_i)
  // (exponential s = a, m = 0; normal s = sigma, m = mu; in T precision)
  {
    T* sB = batch_sb(sh, T());
    T* sD = batch_sd(sh, T());
    const T* sX = batch_sx<T>(sh, DIST);
    for (int k = threadIdx.x; k < 512; k += kThreads) {
      const bool neg = k >= 256;
      const T B = Prec<T>::mul(sink.a, sX[k & 255]);
      const T m = DIST == ZIG_EXP ? (T)0 : sink.b;
      sB[k] = neg ? -B : B;
      sD[k] = neg ? Prec<T>::add(m, B) : Prec<T>::add(m, -B);
    }
    sink.sB = sB;
    sink.sD = sD;
    __syncthreads();
  }
  const RoundKeys rk = device_keys(seed);
  gen_tiles<DIST, T, BatchShape<T>, 0, 8>(sh, sink, batch_sx<T>(sh, DIST), q.n, q.head, q.nvec, seed,
                                     q.offset, rk, lim, t0 - tile0, t1 - tile0, 1, t0 == tile0);
}

__device__ __forceinline__ unsigned smid() {
  unsigned v;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(v));
  return v;
}

// This CTA's home range: the first CTA on an SM takes the next range for
// the SM, later ones wait (bounded) for its choice.  A CTA left without a
// range (more SMs than ranges, or the wait gave up) starts from range
// smid mod nranges; every CTA ends up visiting every range, so no range is
// left unclaimed whichever SMs take part.
__device__ unsigned batch_home(BatchHeader* hdr, int* smmap) {
  const unsigned sm = smid(), nr = hdr->nranges;
  if (sm >= (unsigned)kBatchSmSlots) return sm % nr;
  int v = atomicCAS(&smmap[sm], -1, -2);
  if (v == -1) {
    const unsigned id = atomicAdd(&hdr->range_counter, 1u);
    v = id < nr ? (int)id : -3;
    atomicExch(&smmap[sm], v);
  } else {
    const unsigned long long t0 = globaltimer();
    while (v == -2 && globaltimer() - t0 < 1000000ull) {
      __nanosleep(64);
      v = *(volatile int*)&smmap[sm];
    }
  }
  return v >= 0 ? (unsigned)v : sm % nr;
}

// Claim the next chunk: from the home range first, then from the others in
// turn (scan counts the ranges found empty).  Returns false when every
// range is exhausted.
__device__ bool batch_claim(BatchRange* rng, unsigned nr, unsigned home, unsigned& scan,
                            uint64_t chunk, uint64_t& pos, uint64_t& end) {
  while (scan < nr) {
    BatchRange& g = rng[(home + scan) % nr];
    const uint64_t e = g.end;
    if (*(volatile unsigned long long*)&g.cursor < e) {
      const uint64_t b = atomicAdd(&g.cursor, (unsigned long long)chunk);
      if (b < e) {
        pos = b;
        end = b + chunk < e ? b + chunk : e;
        return true;
      }
    }
    ++scan;
  }
  return false;
}

#ifndef ZIG_BATCH_MINBLOCKS
#define ZIG_BATCH_MINBLOCKS 2
#endif
__global__ void __launch_bounds__(kThreads, ZIG_BATCH_MINBLOCKS)
    batch_kernel(BatchReq* reqs, BatchHeader* hdr, Limits lim) {
  __shared__ BatchCtaState sh;
  __shared__ uint64_t s_pos, s_end;  // the CTA's current chunk, [pos, end)
  __shared__ uint32_t s_req;         // request of tile pos
  const int tid = threadIdx.x;
  for (int k = tid; k < 256; k += kThreads) {
    for (int d = 0; d < 2; ++d) {
      sh.sX64[d][k] = g_tab[d].X[k];
      sh.sX32[d][k] = g_tab[d].X32[k];
    }
  }
  const uint32_t count = hdr->count;
  BatchRange* rng = (BatchRange*)((char*)hdr + batch_ranges_offset(count));
  unsigned home = 0, scan = 0;
  uint32_t r = 0;  // thread 0: request of the last session
  if (tid == 0) {
    home = batch_home(hdr, (int*)((char*)hdr + batch_smmap_offset(count)));
    uint64_t pos = 0, end = 0;
    if (batch_claim(rng, hdr->nranges, home, scan, hdr->chunk, pos, end)) r = find_request(reqs, count, pos);
    s_pos = pos;
    s_end = end;
    s_req = r;
  }
  __syncthreads();
  for (;;) {
    const uint64_t t = s_pos, end = s_end;
    if (t >= end) break;
    const uint32_t q = s_req;
    const uint64_t rend = reqs[q].tile0 + reqs[q].ntiles;
    const uint64_t t1 = rend < end ? rend : end;
    switch (reqs[q].cls) {
      case 0: batch_run<ZIG_EXP, float>(sh, reqs, q, t, t1, lim); break;
      case 1: batch_run<ZIG_NORMAL, float>(sh, reqs, q, t, t1, lim); break;
      case 2: batch_run<ZIG_EXP, double>(sh, reqs, q, t, t1, lim); break;
      default: batch_run<ZIG_NORMAL, double>(sh, reqs, q, t, t1, lim); break;
    }
    __threadfence();  // this thread's outputs of the session, before it counts
    __syncthreads();
    if (tid == 0) {
      settle(hdr, reqs, q, t1 - t);
      uint64_t pos = t1, e = end;
      if (pos >= e && !batch_claim(rng, hdr->nranges, home, scan, hdr->chunk, pos, e)) pos = e = 0;
      if (pos < e) {
        // the request of tile pos: walk forward from the last one, else search
        r = q;
        int steps = 0;
        while (r + 1 < count && pos >= reqs[r].tile0 + reqs[r].ntiles && steps < 8) {
          ++r;
          ++steps;
        }
        if (pos < reqs[r].tile0 || pos >= reqs[r].tile0 + reqs[r].ntiles)
          r = find_request(reqs, count, pos);
      }
      s_pos = pos;
      s_end = e;
      s_req = r;
    }
    __syncthreads();
  }
}

}  // namespace zig

#endif
