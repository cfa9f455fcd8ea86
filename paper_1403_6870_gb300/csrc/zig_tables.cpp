// zig_tables.cpp -- host construction of the modified-ziggurat tables.
//
// McFarland, arXiv:1403.6870, Sec. 2: the layers of the modified ziggurat
// lie wholly under the density P; layer k has its upper-right corner on P at
// (X_k, P(X_k)), its bottom at the previous layer's height, and area
// 1/i_max:  1/i_max = X_k (P(X_k) - P(X_{k-1})).  Layers are stacked until
// none fits (L_max of them); the overhangs A_j to the right of each layer,
// the tail A_0 beyond X_0 and the cap above the last layer hold the rest of
// the mass.  The tables are computed in binary128 and rounded to binary64
// (Appendix B) and, for the FP32 generator, to binary32.  i_max is 256 (the
// paper's tables) or 1024 (the variant of Appendix D item 1).
//
// Root finding here is a bracketed Newton iteration (Newton step when it
// stays inside the bracket and shrinks it, bisection otherwise); both roots
// of the layer equation lie on either side of the area's maximum, and the
// larger one is the layer edge.
#include <math.h>

#include <cstdint>
#include <cstring>
#include <deque>
#include <vector>

#include "zig_internal.h"

namespace zig {
namespace {

typedef _Float128 quad;

struct Density {
  int dist;
  quad c;  // normalising constant of the half-normal
  explicit Density(int d) : dist(d) {
    c = (d == ZIG_EXP) ? (quad)1 : sqrtf128((quad)2 / acosf128((quad)-1));
  }
  quad p(quad x) const {
    return dist == ZIG_EXP ? expf128(-x) : c * expf128(-(x * x) / 2);
  }
  // d/dx of P
  quad dp(quad x) const { return dist == ZIG_EXP ? -p(x) : -x * p(x); }
  // d2/dx2 of P
  quad d2p(quad x) const {
    return dist == ZIG_EXP ? p(x) : (x * x - 1) * p(x);
  }
  // unnormalised height stored for the rejection test
  quad height(quad x) const {
    return dist == ZIG_EXP ? expf128(-x) : expf128(-(x * x) / 2);
  }
  // mass of P on [a, b]
  quad mass(quad a, quad b) const {
    if (dist == ZIG_EXP) return expf128(-a) - expf128(-b);
    const quad s = sqrtf128((quad)2);
    return erfcf128(a / s) - erfcf128(b / s);
  }
  quad tail(quad a) const {
    if (dist == ZIG_EXP) return expf128(-a);
    return erfcf128(a / sqrtf128((quad)2));
  }
};

// Root of h on [lo, hi] with sign(h(lo)) != sign(h(hi)); h and its
// derivative dh are callables.  Newton steps are kept only if they land
// strictly inside the current bracket.
template <class H, class D>
quad safe_newton(H h, D dh, quad lo, quad hi) {
  quad hlo = h(lo);
  bool lo_pos = hlo > 0;
  quad x = (lo + hi) / 2;
  for (int it = 0; it < 400; ++it) {
    quad hx = h(x);
    if (hx == 0) return x;
    if ((hx > 0) == lo_pos)
      lo = x;
    else
      hi = x;
    quad d = dh(x);
    quad nx = (d != 0) ? x - hx / d : (lo + hi) / 2;
    if (!(nx > lo && nx < hi)) nx = (lo + hi) / 2;
    if (nx == x || hi - lo <= ldexpf128(fabsf128(x), -112)) return nx;
    x = nx;
  }
  return x;
}

double round_down(quad v) {
  double d = (double)v;
  if ((quad)d > v) d = nextafter(d, -INFINITY);
  return d;
}

// Deterministic integer alias table (Walker/Vose; the paper cites Smith
// 2002 for O(1) sampling of j ~ A).  cols = i_max columns of capacity
// K = 2^64 / cols, weights summing to 2^64.  Worklists are FIFO queues
// filled in increasing index order; the head of "small" is paired with the
// head of "large"; a large entry whose remaining weight drops below K moves
// to the back of "small".
void vose(const std::vector<uint64_t>& q, int cols, uint64_t K, uint64_t* T, uint16_t* alias) {
  std::vector<uint64_t> rem(q);
  std::deque<int> small, large;
  for (int j = 0; j < cols; ++j) (rem[j] < K ? small : large).push_back(j);
  while (!small.empty() && !large.empty()) {
    const int s = small.front();
    small.pop_front();
    const int l = large.front();
    T[s] = rem[s];
    alias[s] = (uint16_t)l;
    rem[l] -= K - rem[s];
    if (rem[l] < K) {
      large.pop_front();
      small.push_back(l);
    }
  }
  for (int l : large) {
    T[l] = K;
    alias[l] = (uint16_t)l;
  }
  for (int s : small) {
    T[s] = K;
    alias[s] = (uint16_t)s;
  }
}

// Tables of dist for i_max = 2^ibits (ibits 8 or 10).
int build_one(int dist, int ibits, zig_tables_ex* out) {
  std::memset(out, 0, sizeof(*out));
  const int imax = 1 << ibits;
  const Density P(dist);
  const quad area = (quad)1 / imax;
  std::vector<quad> X(imax + 1), F(imax + 1);  // abscissae and normalised heights
  int L = 0;
  quad fprev = 0;
  quad xprev = dist == ZIG_EXP ? (quad)64 : (quad)40;  // area << 1/i_max there
  for (int k = 0; k < imax; ++k) {
    // area of the layer with corner at x and bottom fprev, and derivatives
    auto g = [&](quad x) { return x * (P.p(x) - fprev); };
    auto g1 = [&](quad x) { return P.p(x) - fprev + x * P.dp(x); };
    auto g2 = [&](quad x) { return 2 * P.dp(x) + x * P.d2p(x); };
    // The maximum of g: g' > 0 at 0 and g' < 0 at min(1, xprev).
    quad top = xprev < 1 ? xprev : (quad)1;
    quad xs = (g1(top) >= 0) ? top : safe_newton(g1, g2, (quad)0, top);
    if (g(xs) < area) break;
    quad xk = safe_newton([&](quad x) { return g(x) - area; }, g1, xs, xprev);
    X[k] = xk;
    F[k] = P.p(xk);
    fprev = F[k];
    xprev = xk;
    L = k + 1;
  }
  if (L < 2) return 1;
  X[L] = 0;
  F[L] = P.p(0);

  // Masses: tail beyond X_0, then overhang j = 1..L (j = L is the cap).
  std::vector<quad> A(L + 1);
  A[0] = P.tail(X[0]);
  for (int j = 1; j <= L; ++j)
    A[j] = P.mass(X[j], X[j - 1]) - F[j - 1] * (X[j - 1] - X[j]);

  out->dist = dist;
  out->L = L;
  out->imax = imax;
  out->index_bits = ibits;
  std::vector<quad> H(L + 1);
  for (int k = 0; k <= L; ++k) H[k] = (k == L) ? (quad)1 : P.height(X[k]);
  for (int k = 0; k <= L; ++k) {
    out->X[k] = (double)X[k];
    out->f[k] = (double)H[k];
    out->A[k] = (double)A[k];
    out->X32[k] = (float)X[k];
    out->f32[k] = (float)H[k];
  }
  for (int j = 1; j <= L; ++j) {
    out->dX[j] = (double)(X[j - 1] - X[j]);
    out->df[j] = (double)(H[j] - H[j - 1]);
    out->dX32[j] = (float)(X[j - 1] - X[j]);
    out->df32[j] = (float)(H[j] - H[j - 1]);
  }
  out->rinv = (double)((quad)1 / X[0]);
  out->rinv32 = (float)((quad)1 / X[0]);

  if (dist == ZIG_EXP) {
    // Chord of box j from (X_j, f_j) to (X_{j-1}, f_{j-1}) lies above the
    // convex e^-x; its largest gap to the curve, where e^-x equals minus
    // the slope, over the box height is eps_j; one eps = max_j eps_j
    // serves all boxes (Appendix C item 2).
    quad emax = 0;
    for (int j = 1; j <= L; ++j) {
      const quad w = X[j - 1] - X[j], h = F[j] - F[j - 1];
      const quad xm = logf128(w / h);
      const quad gap = F[j] - (xm - X[j]) * h / w - expf128(-xm);
      const quad e = gap / h;
      if (e > emax) emax = e;
    }
    out->eps = (double)emax;
    out->tau = round_down((quad)1 - emax * ((quad)1 + ldexpf128((quad)1, -40)));
  }

  // Integer alias weights, total 2^64 (i_max columns of capacity 2^64 / i_max).
  quad sum = 0;
  for (int j = 0; j <= L; ++j) sum += A[j];
  std::vector<uint64_t> q(imax, 0);
  const quad scale = ldexpf128((quad)1, 64);
  unsigned __int128 tot = 0;
  int imax_w = 0;
  for (int j = 0; j <= L; ++j) {
    q[j] = (uint64_t)rintf128(A[j] / sum * scale);
    tot += q[j];
    if (q[j] > q[imax_w]) imax_w = j;
  }
  const unsigned __int128 want = (unsigned __int128)1 << 64;
  if (tot > want)
    q[imax_w] -= (uint64_t)(tot - want);
  else
    q[imax_w] += (uint64_t)(want - tot);
  vose(q, imax, (uint64_t)1 << (64 - ibits), out->T, out->alias);
  return 0;
}

// The 256-column tables in the original export layout.
void narrow(const zig_tables_ex& w, zig_tables_export* out) {
  std::memset(out, 0, sizeof(*out));
  out->dist = w.dist;
  out->L = w.L;
  out->imax = w.imax;
  for (int k = 0; k < 257; ++k) {
    out->X[k] = w.X[k];
    out->f[k] = w.f[k];
    out->dX[k] = w.dX[k];
    out->df[k] = w.df[k];
    out->A[k] = w.A[k];
    out->X32[k] = w.X32[k];
    out->f32[k] = w.f32[k];
    out->dX32[k] = w.dX32[k];
    out->df32[k] = w.df32[k];
  }
  out->eps = w.eps;
  out->tau = w.tau;
  out->rinv = w.rinv;
  out->rinv32 = w.rinv32;
  for (int c = 0; c < 256; ++c) {
    out->T[c] = w.T[c];
    out->alias[c] = (uint8_t)w.alias[c];
  }
}

}  // namespace

int build_host_tables(zig_tables_export* exp_tab, zig_tables_export* nrm_tab) {
  static zig_tables_ex w;  // ~55 KB: not on the stack
  if (build_one(ZIG_EXP, 8, &w) != 0) return 1;
  narrow(w, exp_tab);
  if (build_one(ZIG_NORMAL, 8, &w) != 0) return 1;
  narrow(w, nrm_tab);
  return 0;
}

namespace {

// Largest value of the smooth function g on [0, 1]: the best of a uniform
// grid, refined by golden-section search around it.
template <class G>
quad max_on_unit(G g) {
  const int N = 2048;
  int best = 0;
  quad bv = g((quad)0);
  for (int k = 1; k <= N; ++k) {
    const quad v = g((quad)k / N);
    if (v > bv) {
      bv = v;
      best = k;
    }
  }
  quad a = (quad)(best > 0 ? best - 1 : 0) / N, b = (quad)(best < N ? best + 1 : N) / N;
  const quad r = (sqrtf128((quad)5) - 1) / 2;
  quad c = b - r * (b - a), d = a + r * (b - a);
  quad gc = g(c), gd = g(d);
  for (int it = 0; it < 120; ++it) {
    if (gc > gd) {
      b = d;
      d = c;
      gd = gc;
      c = b - r * (b - a);
      gc = g(c);
    } else {
      a = c;
      c = d;
      gc = gd;
      d = a + r * (b - a);
      gd = g(d);
    }
  }
  const quad m = gc > gd ? gc : gd;
  return m > bv ? m : bv;
}

// Shortcut bounds of one box at one precision (b bits of U).  X, dX, f0
// (= f_{j-1}) and df are the rounded table values the device uses; the
// curve h is exact.  In box coordinates (ux, uy) in [0, 1)^2 the curve is
// uy_c(ux) = (h(X + ux dX) - f0) / df; Dm and Dp are the largest distances
// of the curve below and above the chord uy = 1 - ux.  A point with
// ux + uy < 1 - Dm - margin lies under the curve, one with
// ux + uy > 1 + Dp + margin above it, with a margin that exceeds what the
// rounding of x and y to the precision and of exp can move the exact test
// y < h(x).  Returns the integer bounds on mx + my (mx = ux 2^b): accept
// when below acc, reject when above rej.
void box_bounds(int dist, quad X, quad dX, quad f0, quad df, int b, uint64_t* acc, uint64_t* rej) {
  auto h = [&](quad x) { return dist == ZIG_EXP ? expf128(-x) : expf128(-(x * x) / 2); };
  auto dev = [&](quad u) { return (h(X + u * dX) - f0) / df - (1 - u); };
  const quad Dp = max_on_unit(dev);
  const quad Dm = max_on_unit([&](quad u) { return -dev(u); });
  // rounding of x and y to b + 1 significant bits, of the FP64 exp, and the
  // refinement error: in box-height units, with a factor 8 to spare
  const quad ulp_y = ldexpf128((quad)1, -(b + 1)) * (f0 + df);
  const quad xmax = X + dX;
  const quad slope = dist == ZIG_EXP ? h(X) : (X > 1 ? X * h(X) : (xmax > 1 ? expf128((quad)-0.5) : xmax * h(xmax)));
  const quad ulp_x = ldexpf128((quad)1, -(b + 1)) * xmax;
  const quad r = (ulp_y + slope * ulp_x + ldexpf128((quad)1, -50) * (f0 + df)) / df;
  const quad margin = 8 * r + ldexpf128((quad)1, -(b - 4));
  const quad scale = ldexpf128((quad)1, b);
  const quad lo = (1 - (Dm > 0 ? Dm : 0) - margin) * scale;
  const quad hi = (1 + (Dp > 0 ? Dp : 0) + margin) * scale;
  *acc = lo > 0 ? (uint64_t)floorf128(lo) : 0;
  *rej = (uint64_t)ceilf128(hi);
}

}  // namespace

int box_shortcuts(int dist, zig_tables_ex* t) {
  for (int j = 0; j <= t->imax; ++j) t->acc52[j] = t->rej52[j] = t->acc23[j] = t->rej23[j] = 0;
  // the always-accept bound of Sec. 2 (exponential): smallest integers at or
  // above tau 2^52 and tau 2^23
  const uint64_t thr52 = dist == ZIG_EXP ? (uint64_t)ceil(ldexp(t->tau, 52)) : 0;
  const uint64_t thr23 = dist == ZIG_EXP ? (uint64_t)ceil(ldexp(t->tau, 23)) : 0;
  for (int j = 1; j <= t->L; ++j) {
    box_bounds(dist, (quad)t->X[j], (quad)t->dX[j], (quad)t->f[j - 1], (quad)t->df[j], 52,
               &t->acc52[j], &t->rej52[j]);
    box_bounds(dist, (quad)t->X32[j], (quad)t->dX32[j], (quad)t->f32[j - 1], (quad)t->df32[j], 23,
               &t->acc23[j], &t->rej23[j]);
    if (t->acc52[j] < thr52) t->acc52[j] = thr52;
    if (t->acc23[j] < thr23) t->acc23[j] = thr23;
  }
  return 0;
}

int build_host_tables_ex(int ibits, zig_tables_ex* exp_tab, zig_tables_ex* nrm_tab) {
  if (ibits != 8 && ibits != 10) return 1;
  if (build_one(ZIG_EXP, ibits, exp_tab) != 0) return 1;
  if (build_one(ZIG_NORMAL, ibits, nrm_tab) != 0) return 1;
  box_shortcuts(ZIG_EXP, exp_tab);
  box_shortcuts(ZIG_NORMAL, nrm_tab);
  return 0;
}

}  // namespace zig
