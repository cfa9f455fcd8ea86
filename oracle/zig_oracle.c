/*
 * zig_oracle.c -- plain, slow CPU oracle for the modified ziggurat of
 * McFarland (arXiv:1403.6870).  TEST INFRASTRUCTURE ONLY (see zig_oracle.h):
 * nothing in the product library includes or calls this file.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared zig_oracle.c -lm -lpthread
 * -ffp-contract=off matters: every a*b+c below is rounded twice unless it is
 * written as fma(), exactly as the readings of the algorithm state.
 *
 * Tables are built in binary128 (_Float128) and rounded to binary64 and
 * binary32 at the end (Appendix B: tables computed at 128 bits, rounded to
 * 64).  Sampling arithmetic is binary64 (FP64 samplers) or binary32 (FP32
 * samplers, with the exact rejection comparisons made in binary64).
 */
#define _GNU_SOURCE
#define __STDC_WANT_IEC_60559_TYPES_EXT__ 1
#include "zig_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

typedef _Float128 q128;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 as published by Salmon, Moraes, Dror and Shaw (SC'11):      */
/* each round multiplies counter words 0 and 2 by M0 and M1 (32x32->64),     */
/* then the new counter is (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1,     */
/* lo(M0*c0)); the key is bumped by the Weyl constants W0, W1 per round.     */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; r++) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* Word sources                                                             */
/* ------------------------------------------------------------------------ */
void orc_words_philox(orc_words* w, uint64_t seed, uint64_t g) {
  memset(w, 0, sizeof(*w));
  w->kind = 0;
  w->seed = seed;
  w->g = g;
}

void orc_words_packed(orc_words* w, uint64_t seed, uint64_t g, int dtype) {
  memset(w, 0, sizeof(*w));
  w->kind = 2;
  w->dtype = dtype;
  w->seed = seed;
  w->g = g;
}

void orc_words_script(orc_words* w, const uint64_t* script, int n) {
  memset(w, 0, sizeof(*w));
  w->kind = 1;
  w->script = script;
  w->nscript = n;
}

uint64_t orc_next(orc_words* w) {
  w->used++;
  if (w->kind == 1) {
    if (w->pos >= w->nscript) {
      w->overrun = 1;
      return 0;
    }
    return w->script[w->pos++];
  }
  if (w->kind == 2) {
    uint32_t key[2] = {(uint32_t)w->seed, (uint32_t)(w->seed >> 32)};
    /* packed keying: the first word from the block shared with the
     * neighbouring counters, then counter g's private stream (domain 1) */
    w->kind = 0;
    w->dom = 1u;
    uint32_t r[4];
    if (w->dtype == ORC_F64) {
      uint64_t h = w->g >> 1;
      uint32_t ctr[4] = {(uint32_t)h, (uint32_t)(h >> 32), 0u, 0u};
      orc_philox4x32_10(ctr, key, r);
      int half = (int)(w->g & 1u);
      return (uint64_t)r[2 * half] | ((uint64_t)r[2 * half + 1] << 32);
    }
    uint64_t h = w->g >> 2;
    uint32_t ctr[4] = {(uint32_t)h, (uint32_t)(h >> 32), 0u, 0u};
    orc_philox4x32_10(ctr, key, r);
    uint32_t lane = r[w->g & 3u];
    return (uint64_t)(lane & 0x1FFu) | ((uint64_t)(lane >> 9) << 41);
  }
  if (w->half == 0) {
    /* Block a = w->block of counter g: (g_lo, g_hi, dom, a), key = seed. */
    uint32_t ctr[4] = {(uint32_t)w->g, (uint32_t)(w->g >> 32), w->dom, w->block};
    uint32_t key[2] = {(uint32_t)w->seed, (uint32_t)(w->seed >> 32)};
    orc_philox4x32_10(ctr, key, w->r);
    w->half = 1;
    return (uint64_t)w->r[0] | ((uint64_t)w->r[1] << 32);
  }
  w->half = 0;
  w->block++;
  return (uint64_t)w->r[2] | ((uint64_t)w->r[3] << 32);
}

/* ------------------------------------------------------------------------ */
/* Table construction (Sec. 2) in binary128                                 */
/* ------------------------------------------------------------------------ */
static q128 q_pi(void) { return acosf128((q128)-1); }

/* Normalised density on x >= 0: exponential e^-x, half-normal
 * sqrt(2/pi) e^{-x^2/2}. */
static q128 dens(int dist, q128 x) {
  if (dist == ORC_EXP) return expf128(-x);
  return sqrtf128((q128)2 / q_pi()) * expf128(-x * x / 2);
}

/* g(X) = X (P(X) - f_prev): area of the layer whose upper-right corner is
 * (X, P(X)) and whose bottom is at height f_prev (Sec. 2). */
static q128 layer_area(int dist, q128 X, q128 fprev) {
  return X * (dens(dist, X) - fprev);
}

/* g'(X) = P(X) + X P'(X) - f_prev. */
static q128 layer_area_deriv(int dist, q128 X, q128 fprev) {
  if (dist == ORC_EXP) return dens(dist, X) * (1 - X) - fprev;
  return dens(dist, X) * (1 - X * X) - fprev;
}

/* Bisection on a bracket [lo, hi] where pred(lo) holds and pred(hi) fails,
 * until the midpoint equals an endpoint; returns the last point where the
 * predicate holds. */
static q128 bisect_area(int dist, q128 lo, q128 hi, q128 fprev, q128 area) {
  for (int it = 0; it < 1000; it++) {
    q128 mid = (lo + hi) / 2;
    if (mid == lo || mid == hi) break;
    if (layer_area(dist, mid, fprev) >= area)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

static q128 bisect_argmax(int dist, q128 lo, q128 hi, q128 fprev) {
  for (int it = 0; it < 1000; it++) {
    q128 mid = (lo + hi) / 2;
    if (mid == lo || mid == hi) break;
    if (layer_area_deriv(dist, mid, fprev) > 0)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

/* Round a binary128 value down to binary64. */
static double q_to_double_rd(q128 v) {
  double d = (double)v;
  if ((q128)d > v) d = nextafter(d, -INFINITY);
  return d;
}

static void build_alias(orc_tables* t, const q128* A, int nmass) {
  const int cols = t->imax;
  const uint64_t K = (uint64_t)1 << t->abits; /* capacity per column */
  /* Integer weights: q_j = RN(A_j / sum(A) * cols * K); the rounding
   * residual goes on the largest weight so that sum(q) = cols * K. */
  q128 sumA = 0;
  for (int j = 0; j < nmass; j++) sumA += A[j];
  q128 total = (q128)cols * (q128)K;
  unsigned __int128 acc = 0;
  int big = 0;
  for (int j = 0; j < cols; j++) {
    if (j < nmass) {
      q128 qq = rintf128(A[j] / sumA * total);
      t->q[j] = (uint64_t)qq;
    } else {
      t->q[j] = 0;
    }
    acc += t->q[j];
    if (t->q[j] > t->q[big]) big = j;
  }
  unsigned __int128 want = (unsigned __int128)cols * K;
  if (acc > want)
    t->q[big] -= (uint64_t)(acc - want);
  else
    t->q[big] += (uint64_t)(want - acc);

  /* Vose's construction with FIFO work lists, each filled in increasing j:
   * pair the head of "small" with the head of "large"; the small column
   * keeps its own weight as threshold and aliases to the large entry, whose
   * weight drops by the column's remaining capacity; a large entry that
   * falls below capacity moves to the back of "small". */
  uint64_t w[ORC_MAXCOLS];
  int small[ORC_MAXCOLS], large[ORC_MAXCOLS];
  int ns = 0, nl = 0, hs = 0, hl = 0;
  for (int j = 0; j < cols; j++) {
    w[j] = t->q[j];
    if (w[j] < K)
      small[ns++] = j;
    else
      large[nl++] = j;
  }
  while (hs < ns && hl < nl) {
    int s = small[hs++];
    int l = large[hl];
    t->T[s] = w[s];
    t->alias[s] = (uint16_t)l;
    w[l] -= (K - w[s]);
    if (w[l] < K) {
      hl++;
      small[ns++] = l;
    }
  }
  while (hl < nl) {
    int l = large[hl++];
    t->T[l] = K;
    t->alias[l] = (uint16_t)l;
  }
  while (hs < ns) {
    int s = small[hs++];
    t->T[s] = K;
    t->alias[s] = (uint16_t)s;
  }
}

int orc_build_tables(int dist, int ibits, int ubits, int abits,
                     orc_tables* t) {
  if (dist != ORC_EXP && dist != ORC_NORMAL) return 1;
  if (ibits < 1 || ibits > 10 || ubits < 1 || ubits > 52) return 1;
  if (abits < 1 || abits > 64 - ibits) return 1;
  memset(t, 0, sizeof(*t));
  t->dist = dist;
  t->ibits = ibits;
  t->imax = 1 << ibits;
  t->ubits = ubits;
  t->abits = abits;

  const q128 area = (q128)1 / (q128)t->imax;
  q128 Xq[ORC_MAXCOLS + 1], fq[ORC_MAXCOLS + 1]; /* normalised heights */
  /* Layers: solve 1/imax = X_k (P(X_k) - P(X_{k-1})) for the larger root,
   * starting from the origin (f_{-1} = 0), until no layer of area 1/imax
   * fits under P (Sec. 2). */
  int L = 0;
  q128 fprev = 0;
  q128 Xprev = (dist == ORC_EXP) ? (q128)64 : (q128)40; /* g < area there */
  for (int k = 0; k < t->imax; k++) {
    q128 hi = Xprev < 1 ? Xprev : (q128)1;
    q128 xs = bisect_argmax(dist, 0, hi, fprev);
    if (layer_area(dist, xs, fprev) < area) break;
    q128 Xk = bisect_area(dist, xs, Xprev, fprev, area);
    Xq[k] = Xk;
    fq[k] = dens(dist, Xk);
    fprev = fq[k];
    Xprev = Xk;
    L = k + 1;
  }
  t->L = L;
  Xq[L] = 0;
  fq[L] = dens(dist, 0);

  /* Overhang masses: A_0 is the tail beyond X_0; A_j = int_{X_j}^{X_{j-1}}
   * P - f_{j-1} dx for j = 1..L, the last (j = L) being the cap. */
  q128 A[ORC_MAXCOLS + 1];
  if (dist == ORC_EXP) {
    A[0] = expf128(-Xq[0]);
    for (int j = 1; j <= L; j++)
      A[j] = (fq[j] - fq[j - 1]) - fq[j - 1] * (Xq[j - 1] - Xq[j]);
  } else {
    q128 r2 = sqrtf128((q128)2);
    A[0] = erfcf128(Xq[0] / r2);
    for (int j = 1; j <= L; j++)
      A[j] = (erfcf128(Xq[j] / r2) - erfcf128(Xq[j - 1] / r2)) -
             fq[j - 1] * (Xq[j - 1] - Xq[j]);
  }

  /* Stored heights: exponential e^-X; normal unnormalised e^{-X^2/2}. */
  q128 hq[ORC_MAXCOLS + 1];
  for (int k = 0; k <= L; k++)
    hq[k] = (dist == ORC_EXP) ? fq[k] : expf128(-Xq[k] * Xq[k] / 2);

  for (int k = 0; k <= L; k++) {
    t->X[k] = (double)Xq[k];
    t->f[k] = (double)hq[k];
    t->A[k] = (double)A[k];
    t->X32[k] = (float)Xq[k];
    t->f32[k] = (float)hq[k];
  }
  for (int j = 1; j <= L; j++) {
    t->dX[j] = (double)(Xq[j - 1] - Xq[j]);
    t->df[j] = (double)(hq[j] - hq[j - 1]);
    t->dX32[j] = (float)(Xq[j - 1] - Xq[j]);
    t->df32[j] = (float)(hq[j] - hq[j - 1]);
  }

  /* Chord deviation (exponential only; Sec. 2 three-region partition).  In
   * box j the chord joins (X_j, f_j) and (X_{j-1}, f_{j-1}); its slope is
   * s = -(f_j - f_{j-1}) / (X_{j-1} - X_j); chord - e^-x is maximal where
   * e^-x = -s, i.e. x* = ln(dX/df); eps_j is that gap over the box height. */
  if (dist == ORC_EXP) {
    q128 emax = 0;
    for (int j = 1; j <= L; j++) {
      q128 dX = Xq[j - 1] - Xq[j], dfq = fq[j] - fq[j - 1];
      q128 s = -dfq / dX;
      q128 xs = logf128(dX / dfq);
      q128 chord = fq[j] + (xs - Xq[j]) * s;
      q128 e = (chord - expf128(-xs)) / dfq;
      t->eps_j[j] = (double)e;
      if (e > emax) emax = e;
    }
    t->eps = (double)emax;
    /* Always-accept threshold: ux + uy < tau guarantees the point lies
     * under P; tau = RD64(1 - eps (1 + 2^-40)) keeps a safety margin. */
    t->tau = q_to_double_rd((q128)1 - emax * ((q128)1 + ldexpf128(1, -40)));
  }
  t->rinv = (double)((q128)1 / Xq[0]);
  t->rinv32 = (float)((q128)1 / Xq[0]);

  build_alias(t, A, L + 1);
  return 0;
}

size_t orc_tables_size(void) { return sizeof(orc_tables); }

/* ------------------------------------------------------------------------ */
/* Sampler (Table 1, modified column)                                       */
/* ------------------------------------------------------------------------ */
static int g_max_att = 64;
static int g_max_tail = 16;

void orc_set_limits(int max_attempts, int max_tail) {
  g_max_att = max_attempts;
  g_max_tail = max_tail;
}

/* U in [0,1) from the top ubits of a word (Appendix C items 1-2). */
static double u64_of(const orc_tables* t, uint64_t w) {
  uint64_t m = w >> (64 - t->ubits);
  return ldexp((double)m, -t->ubits);
}

/* FP32 U in [0,1): top 23 bits of the word. */
static float u32_of(uint64_t w) { return ldexpf((float)(w >> 41), -23); }

int orc_alias_pick(const orc_tables* t, uint64_t w) {
  int c = (int)(w & (uint64_t)(t->imax - 1));
  uint64_t th = w >> (64 - t->abits);
  return th < t->T[c] ? c : (int)t->alias[c];
}

static void note_margin(double* margin, double y, double bound) {
  if (!margin) return;
  double ulp = nextafter(bound, INFINITY) - bound;
  double m = fabs(y - bound) / ulp;
  if (m < *margin) *margin = m;
}

int orc_overhang_attempt64(const orc_tables* t, int j, double ux, double uy,
                           double* x, double* margin) {
  if (t->dist == ORC_EXP) {
    /* Points above the chord never lie under the convex e^-x; reflect them
     * through the anti-diagonal into the lower-left triangle. */
    if (ux + uy > 1.0) {
      double nx = 1.0 - uy, ny = 1.0 - ux;
      ux = nx;
      uy = ny;
    }
    /* Step 6: x = X_j + U (X_{j-1} - X_j). */
    double xx = fma(ux, t->dX[j], t->X[j]);
    /* Below the chord by more than eps: always under P. */
    if (ux + uy < t->tau) {
      *x = xx;
      return 1;
    }
    /* Step 7 in the narrow band: exact test y < P(x). */
    double y = fma(uy, t->df[j], t->f[j - 1]);
    double bound = exp(-xx);
    note_margin(margin, y, bound);
    if (y < bound) {
      *x = xx;
      return 1;
    }
    return 0;
  }
  double xx = fma(ux, t->dX[j], t->X[j]);
  double y = fma(uy, t->df[j], t->f[j - 1]);
  double bound = exp(-((xx * xx) * 0.5));
  note_margin(margin, y, bound);
  if (y < bound) {
    *x = xx;
    return 1;
  }
  return 0;
}

static double exp64_rec(const orc_tables* t, orc_words* w, orc_diag* d,
                        int depth) {
  /* Step 1: U_1 and i from one word. */
  uint64_t w0 = orc_next(w);
  int i = (int)(w0 & (uint64_t)(t->imax - 1));
  double U1 = u64_of(t, w0);
  /* Step 2: layer i lies wholly under P: return U_1 X_i. */
  if (i < t->L) return U1 * t->X[i];
  /* Step 3: overhang index j ~ A. */
  int j = orc_alias_pick(t, orc_next(w));
  /* Step 4: the tail of an exponential is X_0 plus an exponential. */
  if (j == 0) {
    if (depth + 1 > g_max_tail) {
      d->err = 1;
      return NAN;
    }
    double inner = exp64_rec(t, w, d, depth + 1);
    return t->X[0] + inner;
  }
  /* Steps 5-8 in overhang j; the first attempt reuses U_1 as U_x. */
  double ux = U1;
  for (int att = 0;; att++) {
    double uy = u64_of(t, orc_next(w));
    double x;
    if (orc_overhang_attempt64(t, j, ux, uy, &x, &d->margin)) return x;
    if (att + 1 >= g_max_att) {
      d->err = 1;
      return NAN;
    }
    ux = u64_of(t, orc_next(w));
  }
}

static void diag_init(orc_diag* d) {
  d->words = 0;
  d->err = 0;
  d->margin = INFINITY;
}

double orc_exp64(const orc_tables* te, orc_words* w, orc_diag* d) {
  orc_diag local;
  if (!d) d = &local;
  diag_init(d);
  double x = exp64_rec(te, w, d, 0);
  d->words = w->used;
  return x;
}

double orc_normal64(const orc_tables* te, const orc_tables* tn, orc_words* w,
                    orc_diag* d) {
  orc_diag local;
  if (!d) d = &local;
  diag_init(d);
  uint64_t w0 = orc_next(w);
  int i = (int)(w0 & (uint64_t)(tn->imax - 1));
  int neg = (int)((w0 >> tn->ibits) & 1u);
  double U1 = u64_of(tn, w0);
  double x;
  if (i < tn->L) {
    /* Step 2: U X_i, one rounding, with the sign bit applied (reading
     * R16: the sign of a zero is not fixed; parity compares it by value). */
    const double x2 = U1 * tn->X[i];
    d->words = w->used;
    return neg ? -x2 : x2;
  } else {
    int j = orc_alias_pick(tn, orc_next(w));
    if (j == 0) {
      /* Tail beyond X_0 from two exponential variates (Marsaglia-Tsang):
       * a = E_1 / X_0, accept when 2 E_2 > a^2, return X_0 + a. */
      double a;
      for (int att = 0;; att++) {
        a = exp64_rec(te, w, d, 0) * tn->rinv;
        double b = exp64_rec(te, w, d, 0);
        if (d->err) {
          d->words = w->used;
          return NAN;
        }
        if (b + b > a * a) break;
        if (att + 1 >= g_max_att) {
          d->err = 1;
          d->words = w->used;
          return NAN;
        }
      }
      x = tn->X[0] + a;
    } else {
      double ux = U1;
      for (int att = 0;; att++) {
        double uy = u64_of(tn, orc_next(w));
        if (orc_overhang_attempt64(tn, j, ux, uy, &x, &d->margin)) break;
        if (att + 1 >= g_max_att) {
          d->err = 1;
          d->words = w->used;
          return NAN;
        }
        ux = u64_of(tn, orc_next(w));
      }
    }
  }
  d->words = w->used;
  return neg ? -x : x;
}

/* FP32 samplers: the same words and decisions with binary32 arithmetic;
 * every exact accept/reject comparison promotes its binary32 operands to
 * binary64 (exactly) and compares against a binary64 exp. */
static float exp32_rec(const orc_tables* t, orc_words* w, orc_diag* d,
                       int depth) {
  uint64_t w0 = orc_next(w);
  int i = (int)(w0 & (uint64_t)(t->imax - 1));
  float U1 = u32_of(w0);
  if (i < t->L) return U1 * t->X32[i];
  int j = orc_alias_pick(t, orc_next(w));
  if (j == 0) {
    if (depth + 1 > g_max_tail) {
      d->err = 1;
      return NAN;
    }
    float inner = exp32_rec(t, w, d, depth + 1);
    return t->X32[0] + inner;
  }
  float ux = U1;
  for (int att = 0;; att++) {
    float uy = u32_of(orc_next(w));
    if (ux + uy > 1.0f) {
      float nx = 1.0f - uy, ny = 1.0f - ux;
      ux = nx;
      uy = ny;
    }
    float xx = fmaf(ux, t->dX32[j], t->X32[j]);
    if ((double)(ux + uy) < t->tau) return xx;
    float y = fmaf(uy, t->df32[j], t->f32[j - 1]);
    double bound = exp(-(double)xx);
    note_margin(&d->margin, (double)y, bound);
    if ((double)y < bound) return xx;
    if (att + 1 >= g_max_att) {
      d->err = 1;
      return NAN;
    }
    ux = u32_of(orc_next(w));
  }
}

float orc_exp32(const orc_tables* te, orc_words* w, orc_diag* d) {
  orc_diag local;
  if (!d) d = &local;
  diag_init(d);
  float x = exp32_rec(te, w, d, 0);
  d->words = w->used;
  return x;
}

float orc_normal32(const orc_tables* te, const orc_tables* tn, orc_words* w,
                   orc_diag* d) {
  orc_diag local;
  if (!d) d = &local;
  diag_init(d);
  uint64_t w0 = orc_next(w);
  int i = (int)(w0 & (uint64_t)(tn->imax - 1));
  int neg = (int)((w0 >> tn->ibits) & 1u);
  float U1 = u32_of(w0);
  float x;
  if (i < tn->L) {
    /* as in orc_normal64, in binary32 */
    const float x2 = U1 * tn->X32[i];
    d->words = w->used;
    return neg ? -x2 : x2;
  } else {
    int j = orc_alias_pick(tn, orc_next(w));
    if (j == 0) {
      float a;
      for (int att = 0;; att++) {
        a = exp32_rec(te, w, d, 0) * tn->rinv32;
        float b = exp32_rec(te, w, d, 0);
        if (d->err) {
          d->words = w->used;
          return NAN;
        }
        if ((double)b + (double)b > (double)a * (double)a) break;
        if (att + 1 >= g_max_att) {
          d->err = 1;
          d->words = w->used;
          return NAN;
        }
      }
      x = tn->X32[0] + a;
    } else {
      float ux = U1;
      for (int att = 0;; att++) {
        float uy = u32_of(orc_next(w));
        float xx = fmaf(ux, tn->dX32[j], tn->X32[j]);
        float y = fmaf(uy, tn->df32[j], tn->f32[j - 1]);
        double bound = exp(-(((double)xx * (double)xx) * 0.5));
        note_margin(&d->margin, (double)y, bound);
        if ((double)y < bound) {
          x = xx;
          break;
        }
        if (att + 1 >= g_max_att) {
          d->err = 1;
          d->words = w->used;
          return NAN;
        }
        ux = u32_of(orc_next(w));
      }
    }
  }
  d->words = w->used;
  return neg ? -x : x;
}

/* ------------------------------------------------------------------------ */
/* Bulk drivers (threads only split the index range)                        */
/* ------------------------------------------------------------------------ */
typedef struct {
  const orc_tables *te, *tn;
  int dist, dtype;
  uint64_t seed, offset, lo, hi;
  const uint64_t* idx;
  void* out;
  uint8_t* words;
  double* margin;
  int keying; /* 0 = per index, 1 = packed */
  int64_t errs;
  /* moments */
  int moments;
  q128 sums[4], abssums[4];
  uint64_t hist[4098];
} fill_job;

static double sample_one(const fill_job* jb, uint64_t pos, orc_diag* d) {
  orc_words w;
  if (jb->keying == 1)
    orc_words_packed(&w, jb->seed, jb->offset + pos, jb->dtype);
  else
    orc_words_philox(&w, jb->seed, jb->offset + pos);
  if (jb->dtype == ORC_F64) {
    return jb->dist == ORC_EXP ? orc_exp64(jb->te, &w, d)
                               : orc_normal64(jb->te, jb->tn, &w, d);
  }
  return (double)(jb->dist == ORC_EXP ? orc_exp32(jb->te, &w, d)
                                      : orc_normal32(jb->te, jb->tn, &w, d));
}

/* Histogram bin of Sec. "fused" reduction: floor(256 x) + 2048 on
 * [-8, 8); 4096 below -8; 4097 at or above 8 (and NaN). */
static int hist_bin(double x) {
  if (x < -8.0) return 4096;
  if (!(x < 8.0)) return 4097;
  return (int)floor(256.0 * x) + 2048;
}

static void* fill_worker(void* arg) {
  fill_job* jb = (fill_job*)arg;
  for (uint64_t k = jb->lo; k < jb->hi; k++) {
    uint64_t pos = jb->idx ? jb->idx[k] : k;
    orc_diag d;
    double x = sample_one(jb, pos, &d);
    if (d.err) jb->errs++;
    if (jb->moments) {
      q128 xq = (q128)x, p = xq, ap = fabsf128(xq);
      for (int m = 0; m < 4; m++) {
        jb->sums[m] += p;
        jb->abssums[m] += ap;
        p *= xq;
        ap *= fabsf128(xq);
      }
      jb->hist[hist_bin(x)]++;
      continue;
    }
    if (jb->dtype == ORC_F64)
      ((double*)jb->out)[k] = x;
    else
      ((float*)jb->out)[k] = (float)x;
    if (jb->words) jb->words[k] = (uint8_t)(d.words > 255 ? 255 : d.words);
    if (jb->margin) jb->margin[k] = d.margin;
  }
  return NULL;
}

static int64_t run_jobs(fill_job* proto, uint64_t n, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if ((uint64_t)nthreads > n) nthreads = n ? (int)n : 1;
  fill_job* jobs = (fill_job*)calloc((size_t)nthreads, sizeof(fill_job));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  for (int t = 0; t < nthreads; t++) {
    jobs[t] = *proto;
    jobs[t].lo = n * (uint64_t)t / (uint64_t)nthreads;
    jobs[t].hi = n * (uint64_t)(t + 1) / (uint64_t)nthreads;
    if (nthreads == 1)
      fill_worker(&jobs[t]);
    else
      pthread_create(&th[t], NULL, fill_worker, &jobs[t]);
  }
  int64_t errs = 0;
  for (int t = 0; t < nthreads; t++) {
    if (nthreads > 1) pthread_join(th[t], NULL);
    errs += jobs[t].errs;
  }
  if (proto->moments) {
    for (int m = 0; m < 4; m++) {
      proto->sums[m] = 0;
      proto->abssums[m] = 0;
    }
    memset(proto->hist, 0, sizeof(proto->hist));
    for (int t = 0; t < nthreads; t++) {
      for (int m = 0; m < 4; m++) {
        proto->sums[m] += jobs[t].sums[m];
        proto->abssums[m] += jobs[t].abssums[m];
      }
      for (int b = 0; b < 4098; b++) proto->hist[b] += jobs[t].hist[b];
    }
  }
  free(jobs);
  free(th);
  return errs;
}

int64_t orc_fill(const orc_tables* te, const orc_tables* tn, int dist,
                 int dtype, uint64_t seed, uint64_t offset, uint64_t n,
                 const uint64_t* idx, void* out, uint8_t* words,
                 double* margin, int nthreads) {
  return orc_fill_keyed(te, tn, dist, dtype, 0, seed, offset, n, idx, out, words, margin,
                        nthreads);
}

int64_t orc_fill_keyed(const orc_tables* te, const orc_tables* tn, int dist,
                       int dtype, int keying, uint64_t seed, uint64_t offset,
                       uint64_t n, const uint64_t* idx, void* out,
                       uint8_t* words, double* margin, int nthreads) {
  fill_job* jb = (fill_job*)calloc(1, sizeof(fill_job));
  jb->keying = keying;
  jb->te = te;
  jb->tn = tn;
  jb->dist = dist;
  jb->dtype = dtype;
  jb->seed = seed;
  jb->offset = offset;
  jb->idx = idx;
  jb->out = out;
  jb->words = words;
  jb->margin = margin;
  int64_t e = run_jobs(jb, n, nthreads);
  free(jb);
  return e;
}

int64_t orc_moments(const orc_tables* te, const orc_tables* tn, int dist,
                    int dtype, uint64_t seed, uint64_t offset, uint64_t n,
                    double sums[4], double abssums[4], uint64_t hist[4098],
                    int nthreads) {
  return orc_moments_keyed(te, tn, dist, dtype, 0, seed, offset, n, sums, abssums, hist,
                           nthreads);
}

int64_t orc_moments_keyed(const orc_tables* te, const orc_tables* tn, int dist,
                          int dtype, int keying, uint64_t seed, uint64_t offset,
                          uint64_t n, double sums[4], double abssums[4],
                          uint64_t hist[4098], int nthreads) {
  fill_job* jb = (fill_job*)calloc(1, sizeof(fill_job));
  jb->keying = keying;
  jb->te = te;
  jb->tn = tn;
  jb->dist = dist;
  jb->dtype = dtype;
  jb->seed = seed;
  jb->offset = offset;
  jb->moments = 1;
  int64_t e = run_jobs(jb, n, nthreads);
  for (int m = 0; m < 4; m++) {
    sums[m] = (double)jb->sums[m];
    abssums[m] = (double)jb->abssums[m];
  }
  memcpy(hist, jb->hist, sizeof(jb->hist));
  free(jb);
  return e;
}

int64_t orc_enum_overhang(const orc_tables* t, int j, int bits, double* xs) {
  int64_t cnt = 0;
  const int64_t side = (int64_t)1 << bits;
  for (int64_t a = 0; a < side; a++) {
    double ux = ldexp((double)a, -bits);
    for (int64_t b = 0; b < side; b++) {
      double uy = ldexp((double)b, -bits);
      double x;
      if (orc_overhang_attempt64(t, j, ux, uy, &x, NULL)) xs[cnt++] = x;
    }
  }
  return cnt;
}

/* ------------------------------------------------------------------------ */
/* Batched requests: parameter transforms                                   */
/* ------------------------------------------------------------------------ */
double orc_transform64(int dist, double x, double p0, double p1) {
  if (dist == ORC_EXP) return x * (1.0 / p0);
  return fma(p1, x, p0);
}

float orc_transform32(int dist, float x, double p0, double p1) {
  if (dist == ORC_EXP) return x * (float)(1.0 / p0);
  return fmaf((float)p1, x, (float)p0);
}

int64_t orc_request_values(const orc_tables* te, const orc_tables* tn, int dist, int dtype,
                           uint64_t seed, uint64_t offset, double p0, double p1,
                           const uint64_t* idx, uint64_t m, double* out, int nthreads) {
  /* the standard variate of each counter, then the request's map */
  int64_t errs;
  if (dtype == ORC_F64) {
    errs = orc_fill(te, tn, dist, dtype, seed, offset, m, idx, out, NULL, NULL, nthreads);
    for (uint64_t k = 0; k < m; k++) out[k] = orc_transform64(dist, out[k], p0, p1);
  } else {
    float* tmp = (float*)malloc((m ? m : 1) * sizeof(float));
    if (tmp == NULL) return -1;
    errs = orc_fill(te, tn, dist, dtype, seed, offset, m, idx, tmp, NULL, NULL, nthreads);
    for (uint64_t k = 0; k < m; k++) out[k] = (double)orc_transform32(dist, tmp[k], p0, p1);
    free(tmp);
  }
  return errs;
}

void orc_first_words(uint64_t seed, uint64_t offset, const uint64_t* idx, uint64_t m,
                     uint64_t* out) {
  for (uint64_t k = 0; k < m; k++) {
    orc_words w;
    orc_words_philox(&w, seed, offset + (idx ? idx[k] : k));
    out[k] = orc_next(&w);
  }
}
