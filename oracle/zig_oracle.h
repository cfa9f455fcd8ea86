/*
 * zig_oracle.h -- plain, slow CPU oracle for McFarland's modified ziggurat
 * (arXiv:1403.6870).  TEST INFRASTRUCTURE ONLY: the product library never
 * includes, links or calls anything here; only the tests, the bench's CPU
 * baseline leg and the smoke check do.  It shares no code, header or table
 * generator with the CUDA library under paper_1403_6870_gb300/.
 *
 * What it computes, and where the paper defines it:
 *   - Philox4x32-10 uniform blocks (the paper allows any uniform source,
 *     Sec. 2 "Description of the algorithm" and Sec. 3 "Implementation";
 *     the generator itself is Salmon et al., SC'11).
 *   - Layer tables X_i, f_i = P(X_i) from the equal-area condition
 *     1/i_max = X_i (P(X_i) - P(X_{i-1})), solved by bisection (Sec. 2,
 *     equation after "we can solve for X_i"), built in binary128 and rounded
 *     to binary64 (Appendix B, "Demonstration of Quality").
 *   - Overhang masses A_i = int_{X_i}^{X_{i-1}} P(x) - P(X_{i-1}) dx (Sec. 2),
 *     the tail mass A_0, and the cap above the last layer.
 *   - An integer alias table for drawing j ~ A in O(1) (Sec. 2, citing
 *     Smith 2002).
 *   - The chord deviation epsilon of the exponential overhangs (Sec. 2,
 *     three-region partition; Appendix C item 2: one maximal epsilon).
 *   - The sampler of Table 1 (modified column) with the exponential tail by
 *     memorylessness, the normal tail by Marsaglia-Tsang, the three-region
 *     overhang test and the reflection of Appendix C item 5.
 *
 * Readings of the paper that the oracle takes (each is listed in the
 * project's design notes):
 *   R1 larger root of the layer equation; R2 the cap above the last layer is
 *   overhang j = L; R3 on rejection keep j and redraw both uniforms;
 *   R4 reflection (ux,uy) -> (1-uy, 1-ux); R5 overhang test
 *   y = f_{j-1} + uy (f_j - f_{j-1}); R6 word layout (i = low 8 bits,
 *   normal sign = bit 8, U = top 52 bits, alias threshold = top 56 bits);
 *   R7 Philox key/counter layout; R8 deterministic integer Vose alias rule;
 *   R16 the normal's fast path rounds once with the sign on X_i,
 *   RN((1 + U) sX - sX) for sX = +-X_i, so its zero (U = 0) is +0.
 *
 * Parity status: every function here is pinned by tests under tests/
 * (closed forms, numerical quadrature, brute-force enumeration at reduced
 * width, an independent Philox implementation, distribution tests).
 */
#ifndef ZIG_ORACLE_H
#define ZIG_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_EXP = 0, ORC_NORMAL = 1 };
enum { ORC_F32 = 0, ORC_F64 = 1 };

#define ORC_MAXCOLS 1024

/* Tables for one distribution.  Index conventions (Sec. 2):
 *   layer k = 0..L-1 is the rectangle [0, X_k] x [f_{k-1}, f_k], f_{-1} = 0;
 *   overhang j = 1..L is the box [X_j, X_{j-1}] x [f_{j-1}, f_j] with
 *   X_L = 0 and f_L = P(0) (the cap); j = 0 is the tail x > X_0.
 * For the normal the stored heights are unnormalised, f = exp(-X^2/2), so
 * the exact rejection test reads y < exp(-x^2/2). */
typedef struct orc_tables {
  int32_t dist;   /* ORC_EXP or ORC_NORMAL */
  int32_t imax;   /* number of equal-area slots (256 at full width; 1024 for the
                     10-bit index variant of Appendix D item 1) */
  int32_t ibits;  /* log2(imax) */
  int32_t L;      /* L_max, layers wholly under P */
  int32_t ubits;  /* bits of U taken from the top of a word (52 full width) */
  int32_t abits;  /* alias threshold bits from the top of a word (56) */
  int32_t pad0, pad1;
  double X[ORC_MAXCOLS + 1];  /* X[0..L], X[L] = 0 */
  double f[ORC_MAXCOLS + 1];  /* f[0..L], f[L] = P(0) (1 for both here) */
  double dX[ORC_MAXCOLS + 1]; /* dX[j] = X[j-1] - X[j], j = 1..L */
  double df[ORC_MAXCOLS + 1]; /* df[j] = f[j] - f[j-1], j = 1..L */
  double A[ORC_MAXCOLS + 1];  /* probability masses A[0..L] (normalised P) */
  double eps_j[ORC_MAXCOLS + 1]; /* per-overhang chord deviation (exp) */
  double eps;     /* max_j eps_j (exp; 0 for normal) */
  double tau;     /* always-accept threshold on ux + uy (exp) */
  double rinv;    /* RN64(1 / X_0) (normal tail) */
  float X32[ORC_MAXCOLS + 1];
  float f32[ORC_MAXCOLS + 1];
  float dX32[ORC_MAXCOLS + 1];
  float df32[ORC_MAXCOLS + 1];
  float rinv32;   /* RN32(1 / X_0) */
  float padf;
  uint64_t q[ORC_MAXCOLS];     /* integer alias weights, sum = imax * 2^abits */
  uint64_t T[ORC_MAXCOLS];     /* alias thresholds in [0, 2^abits] */
  uint16_t alias[ORC_MAXCOLS]; /* alias targets */
} orc_tables;

/* Philox4x32-10 block: out = Philox(ctr, key). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]);

/* Build tables for dist with imax = 2^ibits slots (ibits <= 10), U taken
 * from the top ubits of a word, alias thresholds from the top abits.  Full
 * width is (ibits, ubits, abits) = (8, 52, 56); the 10-bit index variant is
 * (10, 52, 54).  Returns 0 on success. */
int orc_build_tables(int dist, int ibits, int ubits, int abits,
                     orc_tables* t);

/* Word sources.  A Philox source yields, for global counter g, the words
 * w_{2a} = r0 | r1<<32, w_{2a+1} = r2 | r3<<32 of block a with counter
 * (g_lo, g_hi, 0, a) and key (seed_lo, seed_hi).  A scripted source yields
 * a fixed list and flags an overrun when it runs out. */
typedef struct orc_words {
  int kind; /* 0 = philox, 1 = scripted, 2 = packed (K2) */
  int dtype; /* packed source: the precision whose first word it forms */
  uint32_t dom; /* philox: counter word 2 of every block */
  uint64_t seed, g;
  uint32_t block;
  int half;
  uint32_t r[4];
  const uint64_t* script;
  int nscript, pos, overrun;
  int used; /* words consumed so far */
} orc_words;

void orc_words_philox(orc_words* w, uint64_t seed, uint64_t g);
/* Packed keying (K2, opt-in; not the paper's, which allows any uniform
 * source).  The first word of counter g comes from a block shared by
 * neighbouring counters: FP64 -- half (g & 1) of block (h_lo, h_hi, 0, 0)
 * with h = g >> 1 (half 0 = r0 | r1<<32, half 1 = r2 | r3<<32); FP32 --
 * the 32-bit output r_(g & 3) of block (h_lo, h_hi, 0, 0) with h = g >> 2,
 * L, presented as the word (L & 0x1FF) | (L >> 9) << 41 (layer index and
 * sign from its low 9 bits, U from its top 23).  Every later word comes
 * from counter g's private domain: blocks (g_lo, g_hi, 1, a), a = 0, 1, ...,
 * words r0 | r1<<32 then r2 | r3<<32. */
void orc_words_packed(orc_words* w, uint64_t seed, uint64_t g, int dtype);
void orc_words_script(orc_words* w, const uint64_t* script, int n);
uint64_t orc_next(orc_words* w);

/* Per-sample diagnostics. */
typedef struct orc_diag {
  int words;        /* words consumed */
  int err;          /* 1 if a loop limit was hit (value is NaN) */
  double margin;    /* min over exact tests of |y - bound| in FP64 ulps of
                       the bound (+inf if no exact test was made) */
} orc_diag;

/* Loop limits (defaults 64 overhang attempts, 16 tail levels). */
void orc_set_limits(int max_attempts, int max_tail);

/* One attempt inside overhang j >= 1 at uniforms (ux, uy) in FP64
 * (Table 1 steps 6-7 with the three-region test and reflection for the
 * exponential).  Returns 1 on accept and stores x. */
int orc_overhang_attempt64(const orc_tables* t, int j, double ux, double uy,
                           double* x, double* margin);

/* Alias pick j from a word: column c = low ibits, threshold from the top
 * abits; j = c if t < T_c else alias_c. */
int orc_alias_pick(const orc_tables* t, uint64_t w);

/* Samplers of Table 1 (modified column).  te are the exponential tables
 * (also used by the normal tail), tn the normal ones. */
double orc_exp64(const orc_tables* te, orc_words* w, orc_diag* d);
double orc_normal64(const orc_tables* te, const orc_tables* tn, orc_words* w,
                    orc_diag* d);
float orc_exp32(const orc_tables* te, orc_words* w, orc_diag* d);
float orc_normal32(const orc_tables* te, const orc_tables* tn, orc_words* w,
                   orc_diag* d);

/* Bulk: out[k] = sample at counter offset + pos_k where pos_k = idx[k] if
 * idx is given, else k.  dtype selects float/double output.  words and
 * margin (nullable) receive per-sample diagnostics.  Returns the number of
 * loop-limit errors. */
int64_t orc_fill(const orc_tables* te, const orc_tables* tn, int dist,
                 int dtype, uint64_t seed, uint64_t offset, uint64_t n,
                 const uint64_t* idx, void* out, uint8_t* words,
                 double* margin, int nthreads);
/* orc_fill with a choice of keying: 0 = per-index words (orc_words_philox),
 * 1 = packed keying (orc_words_packed). */
int64_t orc_fill_keyed(const orc_tables* te, const orc_tables* tn, int dist,
                       int dtype, int keying, uint64_t seed, uint64_t offset,
                       uint64_t n, const uint64_t* idx, void* out,
                       uint8_t* words, double* margin, int nthreads);

/* Fused reduction reference: sums[k] = sum x^(k+1), abssums[k] =
 * sum |x|^(k+1) for k = 0..3 accumulated in binary128, and a histogram of
 * 4096 bins over [-8, 8) with bin = floor(256 x + 2048), bin 4096 for
 * x < -8 and bin 4097 for x >= 8 (and NaN). */
int64_t orc_moments(const orc_tables* te, const orc_tables* tn, int dist,
                    int dtype, uint64_t seed, uint64_t offset, uint64_t n,
                    double sums[4], double abssums[4], uint64_t hist[4098],
                    int nthreads);
/* orc_moments with a choice of keying (0 per index, 1 packed). */
int64_t orc_moments_keyed(const orc_tables* te, const orc_tables* tn, int dist,
                          int dtype, int keying, uint64_t seed, uint64_t offset,
                          uint64_t n, double sums[4], double abssums[4],
                          uint64_t hist[4098], int nthreads);

/* Enumerate the 2^bits x 2^bits grid (ux, uy) = (a 2^-bits, b 2^-bits),
 * the values U takes at bits-bit resolution, through
 * orc_overhang_attempt64 for overhang j: writes accepted x values into xs
 * (capacity 4^bits) and returns their count. */
int64_t orc_enum_overhang(const orc_tables* t, int j, int bits, double* xs);

/* Batched requests: the parameter transform of a request's variate x
 * (exponential with rate lambda: x * RN(1/lambda); normal with mean mu and
 * standard deviation sigma: fma(sigma, x, mu)); FP32 requests use
 * RN32(RN64(1/lambda)), RN32(mu), RN32(sigma) and binary32 arithmetic. */
double orc_transform64(int dist, double x, double p0, double p1);
float orc_transform32(int dist, float x, double p0, double p1);

/* out[k] = variate idx[k] of a request (dist, dtype, seed, offset, p0, p1):
 * the standard variate of counter offset + idx[k] (orc_fill) mapped by
 * orc_transform64/32, for every draw; values as double (FP32 results
 * widened exactly).  Returns the number of draws that hit a loop cap, or
 * -1 if scratch memory could not be allocated. */
int64_t orc_request_values(const orc_tables* te, const orc_tables* tn, int dist, int dtype,
                           uint64_t seed, uint64_t offset, double p0, double p1,
                           const uint64_t* idx, uint64_t m, double* out, int nthreads);

/* out[k] = the first word of counter offset + idx[k] under key seed (block
 * 0, words r0 | r1 << 32 of C-1): the word that carries the layer index, the
 * normal's sign and U_1. */
void orc_first_words(uint64_t seed, uint64_t offset, const uint64_t* idx, uint64_t m,
                     uint64_t* out);

size_t orc_tables_size(void);

#ifdef __cplusplus
}
#endif
#endif
