/*
 * zig.h -- C ABI of the GB300 (sm_103a) modified-ziggurat generator.
 *
 * The library turns counter-based uniform bits into standard exponential
 * and standard normal variates with the modified ziggurat of McFarland,
 * "A modified ziggurat algorithm for generating exponentially- and
 * normally-distributed pseudorandom numbers" (arXiv:1403.6870):
 *   - layers of area 1/256 lie wholly under the density P(x), so a draw
 *     whose layer index i is below L_max returns U * X_i with no rejection
 *     test (Sec. 2; Table 1, modified column, steps 1-2);
 *   - the remaining draws pick an overhang j from the masses A_j with an
 *     alias table (Table 1 step 3), sample the tail (step 4; the exponential
 *     tail by memorylessness, the normal tail by Marsaglia-Tsang, Sec. 2),
 *     or rejection-sample the overhang box (steps 5-8), for the exponential
 *     with the three-region test and the reflection of Appendix C item 5.
 *
 * Uniform source.  Philox4x32-10 (Salmon et al., SC'11).  Output element t
 * of a call with (seed, offset) is the variate for global counter
 * g = offset + t: its k-th uniform block is Philox(counter = (g_lo, g_hi, 0,
 * k), key = (seed_lo, seed_hi)), giving 64-bit words w_{2k} = r0 | r1 << 32
 * and w_{2k+1} = r2 | r3 << 32 consumed in order.  From the first word:
 * layer index i = bits 0-7, normal sign = bit 8, U = bits 12-63 as
 * m * 2^-52 (FP32: bits 41-63 as m * 2^-23); an alias word gives the column
 * from bits 0-7 and a 56-bit threshold from bits 8-63 (Appendix C items
 * 1-2).  A fast-path value is RN(U X_i) with one rounding; the normal's
 * sign is applied to X_i inside that rounding, so a zero (U = 0) is +0 for
 * either sign (the paper does not fix the sign bit of a zero).  Every variate is therefore reproducible from (seed, g) alone, and
 * any split of [offset, offset + n) across calls gives identical bits.
 *
 * Conventions for every entry point below.
 *   - Pointers named d_* or out are DEVICE pointers owned by the caller;
 *     h_* are host pointers.  The library never allocates on a generation
 *     call; its own tables and status word live in static device memory
 *     from zig_build_tables until process exit.
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Generation calls are stream-ordered and return as soon as
 *     the work is enqueued; they do not synchronise.
 *   - Errors are returned as zig_status; nothing aborts or throws across
 *     the ABI.  Conditions detected on the device (a fringe loop reaching
 *     its cap) are recorded in a per-device status word read by
 *     zig_status_poll; the affected outputs are NaN.
 *   - Calls act on the CUDA device current on the calling thread.
 */
#ifndef ZIG_H
#define ZIG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum zig_status {
  ZIG_OK = 0,
  ZIG_E_INVAL = 1,      /* invalid argument (null pointer, bad enum/param) */
  ZIG_E_NOTINIT = 2,    /* zig_build_tables has not run on this device */
  ZIG_E_CUDA = 3,       /* a CUDA runtime call or kernel launch failed */
  ZIG_E_NOMEM = 4,      /* caller-provided workspace too small */
  ZIG_E_ALIGN = 5,      /* pointer not aligned to its element size */
  ZIG_E_RANGE = 6,      /* offset + n wraps past 2^64, or size too large */
  ZIG_E_LOOP_LIMIT = 7, /* device: a fringe loop reached its cap */
  ZIG_E_TABLE = 8,      /* host table construction failed */
  ZIG_E_TIMEOUT = 9     /* device: a bounded internal wait gave up (reserved) */
} zig_status;

typedef enum zig_dtype { ZIG_F32 = 0, ZIG_F64 = 1 } zig_dtype;
typedef enum zig_dist { ZIG_EXP = 0, ZIG_NORMAL = 1 } zig_dist;

/* Human-readable name of a status code (static string, never NULL). */
const char* zig_strerror(zig_status s);

/*
 * zig_build_tables -- build the ziggurat tables and upload them to the
 * current device.
 *
 * Sec. 2: for P(x) = e^-x and the half-normal sqrt(2/pi) e^{-x^2/2}, layer
 * k solves 1/256 = X_k (P(X_k) - P(X_{k-1})) (larger root, P(X_{-1}) = 0)
 * until no layer of area 1/256 fits (L_max = 252 exponential, 253 normal);
 * overhang masses A_j = int_{X_j}^{X_{j-1}} P - P(X_{j-1}) dx (j = 1..L_max,
 * j = L_max the cap above the last layer), A_0 the tail; the alias table
 * for j ~ A (Sec. 2, Smith 2002); the exponential chord deviation eps
 * (Sec. 2, Appendix C item 2).  Values are computed in binary128 and
 * rounded to binary64 and binary32 (Appendix B).
 *
 * Idempotent and thread-safe; the host tables are built once per process
 * and uploaded once per device.  Synchronous (not stream-capturable).
 * Returns ZIG_OK, ZIG_E_TABLE or ZIG_E_CUDA.
 */
zig_status zig_build_tables(void);

/* Flat copy of one distribution's tables, as used on the device.
 * Index conventions (Sec. 2): layer k = 0..L-1 is [0, X_k] x [f_{k-1}, f_k]
 * with f_{-1} = 0; overhang box j = 1..L is [X_j, X_{j-1}] x [f_{j-1}, f_j]
 * with X_L = 0 and f_L = P(0); heights are e^-x (exponential) and the
 * unnormalised e^{-x^2/2} (normal).  dX[j] = X_{j-1} - X_j and
 * df[j] = f_j - f_{j-1} are rounded from binary128 differences.
 * Alias: column c = w & 255 and threshold t = w >> 8 give j = c if
 * t < T[c] else alias[c]. */
typedef struct zig_tables_export {
  int32_t dist;
  int32_t L;
  int32_t imax;
  int32_t reserved;
  double X[257];
  double f[257];
  double dX[257];
  double df[257];
  double A[257];     /* probability masses (informational) */
  double eps;        /* max_j chord deviation over box height (exp) */
  double tau;        /* always-accept threshold on ux + uy (exp) */
  double rinv;       /* RN64(1 / X_0) */
  float X32[257];
  float f32[257];
  float dX32[257];
  float df32[257];
  float rinv32;      /* RN32(1 / X_0) */
  float reserved2;
  uint64_t T[256];
  uint8_t alias[256];
} zig_tables_export;

/* The tables at either index width in one layout: i_max = 2^index_bits
 * columns (index_bits 8: the paper's 256; 10: the 1024 of Appendix D item
 * 1), arrays indexed as in zig_tables_export.  Alias: column c = w &
 * (i_max - 1) and threshold t = w >> index_bits give j = c if t < T[c]
 * else alias[c]; thresholds are on the scale 2^(64 - index_bits). */
typedef struct zig_tables_ex {
  int32_t dist;
  int32_t L;
  int32_t imax;
  int32_t index_bits;
  double X[1025];
  double f[1025];
  double dX[1025];
  double df[1025];
  double A[1025];
  double eps;
  double tau;
  double rinv;
  float X32[1025];
  float f32[1025];
  float dX32[1025];
  float df32[1025];
  float rinv32;
  float reserved;
  uint64_t T[1024];
  uint16_t alias[1024];
  /* Per-box shortcut bounds of the overhang test, box j = 1..L, on the
   * integer sum mx + my of the two uniforms (mx = ux 2^52 for FP64, 2^23 for
   * FP32): a point below acc lies under the curve, one above rej over it,
   * each with a margin for the rounding of x, y and exp, so that skipping
   * the exact test never changes its answer (for the exponential acc also
   * covers the always-accept region ux + uy < tau of Sec. 2).  These bounds
   * give the per-overhang eps of Appendix D item 2 and the normal's
   * convex/concave regions; the outputs are those of the exact test. */
  uint64_t acc52[1025];
  uint64_t rej52[1025];
  uint64_t acc23[1025];
  uint64_t rej23[1025];
} zig_tables_ex;

/*
 * zig_export_tables_ex -- copy the host tables of dist at index_bits (8 or
 * 10) into *h_out.  Builds them if needed (no device is touched).  Returns
 * ZIG_OK, ZIG_E_INVAL (bad dist, index_bits or NULL) or ZIG_E_TABLE.
 */
zig_status zig_export_tables_ex(zig_dist dist, int index_bits, zig_tables_ex* h_out);

/*
 * zig_export_tables -- copy the host tables of dist into *h_out.
 * Builds the host tables if needed (no device is touched).
 * Returns ZIG_OK, ZIG_E_INVAL (bad dist or NULL) or ZIG_E_TABLE.
 */
zig_status zig_export_tables(zig_dist dist, zig_tables_export* h_out);

/*
 * zig_exponential -- n standard exponential variates, Exp(1), into out.
 * zig_normal      -- n standard normal variates, N(0, 1), into out.
 *
 * Table 1 (modified column) with the readings stated above.  out is an
 * array of n float (ZIG_F32) or double (ZIG_F64) elements, aligned to its
 * element size (any further alignment is handled internally), in device or
 * managed memory of the current device, or in page-locked host memory
 * (cudaHostAlloc, cudaHostRegister), which the kernel then writes directly
 * over the host link (NVLink-C2C on Grace systems); other memory (pageable
 * host memory, another device's memory) gives ZIG_E_INVAL.  out[t] is the
 * variate for counter offset + t.  n = 0 is a no-op.
 * FP64: fast-path outputs are the correctly rounded U * X_i.  FP32: the
 * same words, binary32 arithmetic and tables; accept/reject comparisons are
 * made exactly in binary64 against a binary64 exp.
 * Returns ZIG_OK, ZIG_E_INVAL (NULL out with n > 0, bad dtype, memory the
 * kernel cannot write), ZIG_E_ALIGN, ZIG_E_RANGE (offset + n > 2^64),
 * ZIG_E_NOTINIT or ZIG_E_CUDA (launch failure).
 */
zig_status zig_exponential(void* out, uint64_t n, uint64_t seed,
                           uint64_t offset, zig_dtype dtype, void* stream);
zig_status zig_normal(void* out, uint64_t n, uint64_t seed, uint64_t offset,
                      zig_dtype dtype, void* stream);

/*
 * zig_moments -- fused generate-and-reduce: the n variates that
 * zig_exponential / zig_normal would write for (n, seed, offset, dtype)
 * are generated and reduced on the device, never stored.  This is the
 * paper's timing workload, "generating and aggregating" PRNs (Sec. 4).
 *
 * Outputs (device memory, overwritten):
 *   d_sums[k] = sum of x^(k+1), k = 0..3, accumulated per thread in the
 *     variates' precision over one tile of a thread's values (32 at the
 *     default FP32 shape, 64 with packed keying) or directly (FP64) and
 *     then in FP64; every thread adds its values in a fixed order (the
 *     fringe stages' draws when a warp finishes them), each thread block
 *     sums its threads in thread order and the last block the blocks in
 *     block order, so a call repeats bit for bit on the same device;
 *   d_hist[b], b < 4098: count of variates with floor(256 x) + 2048 = b for
 *     -8 <= x < 8, b = 4096 for x < -8, b = 4097 for x >= 8 or NaN (exact).
 * d_workspace: caller-owned device scratch of at least
 *   zig_moments_workspace_bytes(dist, dtype) bytes (8-byte aligned), used
 *   for per-block partial sums; its content need not be initialised.
 * Enqueues two memsets (d_hist, a workspace counter) and one kernel on
 * stream; calls on the same workspace must not overlap.
 * Returns ZIG_OK, ZIG_E_INVAL, ZIG_E_ALIGN, ZIG_E_RANGE, ZIG_E_NOMEM
 * (workspace too small), ZIG_E_NOTINIT or ZIG_E_CUDA.
 */
size_t zig_moments_workspace_bytes(zig_dist dist, zig_dtype dtype);
/* zig_moments_workspace_bytes returns 0 if the current device has no
 * tables yet (call zig_build_tables first). */
zig_status zig_moments(zig_dist dist, zig_dtype dtype, uint64_t n,
                       uint64_t seed, uint64_t offset, double* d_sums,
                       unsigned long long* d_hist, void* d_workspace,
                       size_t workspace_bytes, void* stream);

/* zig_moments over the variates of a keying (zig_keying below): with
 * ZIG_KEY_INDEX exactly zig_moments; with ZIG_KEY_PACKED the variates of
 * zig_generate(dist, ZIG_KEY_PACKED, 8, ...).  The workspace size of
 * zig_moments_workspace_bytes covers both keyings.  Returns as zig_moments,
 * plus ZIG_E_INVAL for an unknown keying. */
zig_status zig_moments_keyed(zig_dist dist, zig_dtype dtype, int keying, uint64_t n,
                             uint64_t seed, uint64_t offset, double* d_sums,
                             unsigned long long* d_hist, void* d_workspace,
                             size_t workspace_bytes, void* stream);

/*
 * zig_moments_noalloc -- zig_moments without a caller workspace.
 *
 * The paper has no counterpart; this is a service for callers that cannot
 * allocate device memory at all: code handed only its output buffers by a
 * host application or inference server that owns the device's memory,
 * code running where the surrounding framework forbids allocation (a
 * locked or exhausted pool, a region whose memory layout must stay fixed),
 * and latency-critical paths that may not enter the allocator.  It computes
 * exactly what zig_moments computes and allocates nothing: no cudaMalloc,
 * no cudaFree, no library routine that allocates.
 *
 * Its scratch (a ticket and 4 FP64 partials per thread block) is a static
 * device array of 64 KiB in the library, present on every device that
 * loads the library until the process exits; its device address is taken
 * by zig_build_tables, which must have run on the current device (as for
 * every entry point).  zig_build_tables also launches each of this entry
 * point's kernels once on an empty range, so that the driver loads their
 * code and sizes their local memory then, not during a later call here
 * (under lazy module loading either could otherwise take device memory on
 * the first call).  All calls share that array and it keeps the last
 * call's contents; each call clears the part that must start at zero.
 * Calls whose executions overlap on the GPU (any device-side concurrency,
 * e.g. two streams) race on the array and give wrong results: serialise
 * them.  A device that would need more than the 64 KiB (more than 2040
 * thread blocks at once) gets ZIG_E_NOMEM; otherwise the returns are
 * those of zig_moments.
 */
zig_status zig_moments_noalloc(zig_dist dist, zig_dtype dtype, uint64_t n,
                               uint64_t seed, uint64_t offset, double* d_sums,
                               unsigned long long* d_hist, void* stream);

/*
 * Batched requests: many generation calls served by one persistent launch.
 * Each request asks for n variates of its own distribution and precision,
 * under its own Philox key and counter offset.  Element t of request r is
 * defined from the standard variate z of counter offset_r + t (exactly what
 * zig_exponential / zig_normal write there) by the standard scale and
 * location change of Exp(1) and N(0, 1):
 *   exponential with rate lambda = p0 > 0:        y = RN(z * RN(1/lambda));
 *   normal with mean mu = p0, sd sigma = p1 > 0:  y = RN(sigma z + mu) (one fma);
 * FP32 requests use s = RN32(RN64(1/lambda)), RN32(mu), RN32(sigma) and
 * binary32 arithmetic.  The paper's method has no batched interface.
 *
 * What the library returns: exactly y for every draw that leaves step 2 of
 * Table 1 (overhang and tail draws).  For a step-2 draw (z = +-RN(U X_i))
 * the map is folded into the step's single rounding, which saves one
 * floating-point operation per value:
 *   y' = RN((1 + U)(+-B_i) + D),  B_i = RN(s X_i),  D = RN(m -+ B_i)
 * (s = RN(1/lambda), m = 0 for the exponential; s = sigma, m = mu for the
 * normal; signs those of the normal's sign bit).  With unit roundoff u
 * (2^-53 for FP64, 2^-24 for FP32) it satisfies
 *   exponential:  |y' - y| <= 4u|y|                       (a few ulp of y);
 *   normal:       |y' - y| <= 4u|y| + 2u|mu| + u|mu -+ sigma X_i|,
 * up to second-order terms: both y and y' are within a few units of
 * roundoff of the exact mu +- sigma U X_i, so where mu cancels sigma z the
 * bound is absolute (in units of |mu|), as for any rounded evaluation of
 * the map.  With rate 1, or mean 0 and sd 1, y' = y bit for bit.
 */
typedef struct zig_request {
  void* out;       /* device array of n float (ZIG_F32) or double elements */
  uint64_t n;      /* < 2^40 */
  uint64_t seed;   /* Philox key */
  uint64_t offset; /* counter of element 0; offset + n must not pass 2^64 */
  uint32_t dist;   /* zig_dist */
  uint32_t dtype;  /* zig_dtype */
  double p0;       /* exponential: rate; normal: mean */
  double p1;       /* normal: standard deviation; exponential: unused */
} zig_request;

/* Bytes of workspace zig_batch needs for count requests. */
size_t zig_batch_workspace_bytes(uint32_t count);

/* Host-side check of a request array (the device checks the same rules and
 * skips a failing request, flagging ZIG_E_INVAL in the status word).
 * Returns ZIG_OK or ZIG_E_INVAL, ZIG_E_ALIGN, ZIG_E_RANGE for the first
 * failing request. */
zig_status zig_batch_validate(const zig_request* h_reqs, uint32_t count);

/*
 * zig_batch -- serve count requests (device array d_reqs, count < 2^23)
 * with one prep kernel and one persistent kernel on stream.  d_workspace is
 * caller-owned device scratch of zig_batch_workspace_bytes(count) bytes
 * (16-byte aligned).  d_done_ns (nullable, device, count entries) receives,
 * per request, the nanoseconds from the batch start (end of the prep
 * kernel) until its last output was written.  The call does not allocate
 * or synchronise.  Calls on the same workspace must not overlap.  Returns
 * ZIG_OK, ZIG_E_INVAL, ZIG_E_NOMEM (workspace too small), ZIG_E_ALIGN,
 * ZIG_E_NOTINIT or ZIG_E_CUDA.
 */
zig_status zig_batch(const zig_request* d_reqs, uint32_t count,
                     unsigned long long* d_done_ns, void* d_workspace,
                     size_t workspace_bytes, void* stream);

/*
 * Batch tuning.  The paper has no batched interface and tunes its CPU code
 * by hand; this is the serving mix's tile scheduling.  The persistent batch
 * kernel's CTAs claim chunks of consecutive tiles (a tile is the plain
 * kernel's unit: 256 threads x V x R outputs of one request); the chunk
 * size changes only the order in which tiles are served, never an output
 * bit.
 */
typedef struct zig_batch_tune_entry {
  uint32_t chunk; /* tiles per claim */
  double ms;      /* measured time of one zig_batch call of the tuned batch */
} zig_batch_tune_entry;

/*
 * zig_batch_autotune -- time zig_batch on the caller's batch (d_reqs,
 * count > 0, d_workspace as for zig_batch) with each candidate chunk size
 * (64, 32, 128, 16 tiles), reps timed calls after one warm-up call each
 * (1 <= reps <= 100), with CUDA events on stream, and select the fastest
 * for later zig_batch calls on the current device.  The calls write the
 * batch's outputs (the same values every time; no completion times).
 * Writes up to max_results entries of results (nullable), the number of
 * candidates to *n_results and the choice to *chosen_chunk (both nullable).
 * Synchronises stream.  Returns ZIG_OK or the errors of zig_batch.
 */
zig_status zig_batch_autotune(const zig_request* d_reqs, uint32_t count, void* d_workspace,
                              size_t workspace_bytes, int reps, void* stream,
                              zig_batch_tune_entry* results, int max_results, int* n_results,
                              uint32_t* chosen_chunk);

/* Set the tiles per claim of later zig_batch calls on the current device
 * (1..4096; default 64).  ZIG_OK, ZIG_E_INVAL or ZIG_E_CUDA. */
zig_status zig_batch_set_chunk(uint32_t chunk);

/* The tiles per claim zig_batch uses on the current device (0 on error). */
uint32_t zig_batch_get_chunk(void);

/*
 * zig_status_poll -- read and clear this device's status word.
 * The read-and-clear is one atomic exchange ordered on stream (after the
 * work queued there), and the call then synchronises that stream only, not
 * the device: a bit set meanwhile by work on another stream is kept for
 * the next poll.  Polls may run at the same time from several threads on
 * several streams (up to 64 in flight at once): each reads its own take,
 * so a recorded condition is returned by exactly one of them.  Returns
 * ZIG_OK if no device-side condition
 * was recorded since the last poll, ZIG_E_LOOP_LIMIT if a fringe loop hit
 * its cap (those outputs are NaN), ZIG_E_INVAL if zig_batch skipped an
 * invalid request, ZIG_E_NOTINIT or ZIG_E_CUDA.  ZIG_E_TIMEOUT is
 * reserved for a bounded device-side wait that gives up; the current
 * kernels have no wait between warps or CTAs that could (the batch kernel's
 * one bounded wait falls back to other work instead).
 */
zig_status zig_status_poll(void* stream);

/*
 * zig_set_fringe_limits -- caps for the rare fringe loops: overhang
 * attempts per variate (default 64) and exponential tail levels (default
 * 16).  Reaching a cap writes NaN and records ZIG_E_LOOP_LIMIT instead of
 * looping on (the chance per variate at the defaults is below 1e-15).
 * Applies to launches enqueued after the call.  max_attempts >= 1,
 * max_tail >= 0, both <= 1<<20, else ZIG_E_INVAL.
 */
zig_status zig_set_fringe_limits(int max_attempts, int max_tail);

/*
 * Keying of the uniform words.  ZIG_KEY_INDEX is the scheme above (every
 * output's words from its own counter: one Philox block per output on the
 * fast path); zig_exponential and zig_normal use it.  ZIG_KEY_PACKED (opt-in,
 * different outputs) shares one block between the fast words of 2 FP64 or
 * 4 FP32 neighbouring outputs, keeping every variate a function of (seed, g)
 * alone:
 *   - the first word of counter g: FP64, half (g & 1) of Philox((h_lo, h_hi,
 *     0, 0)) with h = g >> 1 (half 0 = r0 | r1 << 32, half 1 = r2 | r3 << 32);
 *     FP32, the 32-bit output r_(g & 3) of Philox((h_lo, h_hi, 0, 0)) with
 *     h = g >> 2, whose bits 0-7 are i, bit 8 the normal's sign and bits 9-31
 *     U (m 2^-23);
 *   - every later word (alias pick, overhang attempts, tails): counter g's
 *     private stream, blocks Philox((g_lo, g_hi, 1, a)), a = 0, 1, ..., words
 *     r0 | r1 << 32 then r2 | r3 << 32.
 * The method (Table 1) is unchanged; the paper lets any uniform source feed
 * it (Sec. 2).  Split invariance holds as for ZIG_KEY_INDEX.
 */
typedef enum { ZIG_KEY_INDEX = 0, ZIG_KEY_PACKED = 1 } zig_keying;

/*
 * zig_generate -- zig_exponential (dist ZIG_EXP) or zig_normal (ZIG_NORMAL)
 * with a choice of keying and of table width; (ZIG_KEY_INDEX, 8) gives
 * exactly their outputs.  index_bits 8 uses the paper's i_max = 256 tables;
 * 10 uses i_max = 1024 (Appendix D item 1: a 10-bit layer index, bits 0-9
 * of the first word, the normal's sign in bit 10, alias column bits 0-9 and
 * threshold bits 10-63; U as above), whose fast path covers 1020/1024
 * (exponential) and 1021/1024 (normal) of the draws.  Packed FP32 words hold
 * only 8 index bits, so (ZIG_KEY_PACKED, 10, ZIG_F32) is rejected.
 * Arguments, layout and returns as zig_exponential's, plus ZIG_E_INVAL for
 * an unknown dist, keying or index_bits.  With ZIG_KEY_PACKED a launch whose
 * first vector-aligned counter (offset + the unaligned head) is not a
 * multiple of 2 (FP64) or 4 (FP32) still gives the same outputs, computing
 * one block per output.
 */
zig_status zig_generate(zig_dist dist, zig_keying keying, int index_bits, void* out, uint64_t n,
                        uint64_t seed, uint64_t offset, zig_dtype dtype, void* stream);

/*
 * Launch-shape autotuning.  The paper tunes its CPU code by hand and has
 * no counterpart; the shapes below change only how the work is spread over
 * the GPU, never the outputs (element t is always the variate of counter
 * offset + t).  A shape is V-element vector stores, R vectors per producer
 * thread and tile (V * R outputs per thread and tile), a register budget
 * compiled for min_blocks CTAs per SM, and the CTAs per SM actually
 * launched (blocks_per_sm, 0 = as many as fit).
 */
typedef struct zig_tune_entry {
  int32_t V;
  int32_t R;
  int32_t min_blocks;
  int32_t blocks_per_sm;
  double gsamples_s; /* measured rate of the shape, Gsamples/s (0 if unmeasured) */
} zig_tune_entry;

/* The compiled candidate shapes for dtype (blocks_per_sm 0); the first is
 * the default.  Writes up to max entries to out (host) and returns how
 * many candidates exist. */
int zig_tune_candidates(zig_dtype dtype, zig_tune_entry* out, int max);

/*
 * zig_autotune -- time every candidate shape of zig_exponential (dist
 * ZIG_EXP) or zig_normal (ZIG_NORMAL) at dtype, each at its full and
 * reduced CTAs per SM, on the caller's device scratch d_scratch of
 * scratch_bytes (overwritten; at least 2^20 elements, and larger than the
 * GPU's L2 cache for a write-bound measurement), reps timed launches each
 * after one warm-up, with CUDA events on stream, which it synchronises.
 * Selects the fastest shape for later calls of that (dist, dtype) on this
 * device and records it for zig_tune_save.  Writes up to max_results
 * measured entries to results (host, nullable) and the choice to chosen
 * (host, nullable); *n_results (nullable) receives the number measured.
 * Returns ZIG_OK, ZIG_E_INVAL, ZIG_E_NOTINIT or ZIG_E_CUDA.  Not for use
 * during stream capture.
 */
zig_status zig_autotune(zig_dist dist, zig_dtype dtype, void* d_scratch, size_t scratch_bytes,
                        int reps, void* stream, zig_tune_entry* results, int max_results,
                        int* n_results, zig_tune_entry* chosen);

/* The shape used for (dist, dtype) on the current device (gsamples_s as
 * measured or loaded, else 0).  ZIG_OK, ZIG_E_INVAL or ZIG_E_CUDA. */
zig_status zig_tune_get(zig_dist dist, zig_dtype dtype, zig_tune_entry* out);

/* Use shape e (V, R, min_blocks of a candidate; blocks_per_sm >= 0) for
 * (dist, dtype) on the current device.  ZIG_E_INVAL if e is no candidate. */
zig_status zig_tune_set(zig_dist dist, zig_dtype dtype, const zig_tune_entry* e);

/*
 * Tuning cache, one JSON object per line:
 *   {"device": "<CUDA device name>", "sms": 152, "dist": "normal",
 *    "dtype": "f64", "V": 4, "R": 4, "min_blocks": 4, "blocks_per_sm": 4,
 *    "gsamples_s": 318.2}
 * zig_tune_save writes every entry this process measured or loaded (later
 * entries replace earlier ones with the same device, SM count, dist and
 * dtype).  zig_tune_load reads a file; entries whose device name and SM
 * count match a device take effect on it (now if its tables are built,
 * else at zig_build_tables).  zig_build_tables loads the file named by the
 * environment variable ZIG_TUNE_CACHE, if set, once per process.  Lines
 * that do not parse, or name no candidate shape, are skipped.  ZIG_OK,
 * ZIG_E_INVAL (null path; for load, an unreadable file) or ZIG_E_CUDA
 * (save: the file cannot be written).
 */
zig_status zig_tune_save(const char* path);
zig_status zig_tune_load(const char* path);

#ifdef __cplusplus
}
#endif
#endif /* ZIG_H */
