"""Pins for the oracle's sampler (Table 1, modified column, arXiv:1403.6870).

Three kinds of evidence, none of which re-types the oracle's formulas:
  * scripted word streams with hand-derived outcomes (fast path, exponential
    tail by memorylessness, keep-j on rejection, reflection, normal sign,
    Marsaglia-Tsang tail, loop limits);
  * exact enumeration at reduced width (i_max = 8, 12-bit uniforms): the
    sampler's law for uniform words, composed from exhaustively enumerated
    pieces, must match the exact CDF to within the grid discretisation;
  * full-width distribution tests against closed forms (KS, 1024-bin
    chi-square, raw moments, fast-path exit rate, tail laws).
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import special, stats

SEED = 0x0123456789ABCDEF


def fma(a, b, c):
    """Correctly rounded a*b + c (float(Fraction) rounds to nearest)."""
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def word(i, m, sign=0):
    """Full-width word: layer index in bits 0-7, sign bit 8, U = m 2^-52."""
    return (m << 12) | (sign << 8) | i


def u_word(u):
    m = int(Fraction(u) * 2**52)
    assert Fraction(m, 2**52) == Fraction(u)
    return m << 12


def alias_word(t, j):
    K = 1 << t.abits
    if int(t.T[j]) > 0:
        return j  # column j with threshold 0 < T_j keeps j
    for c in range(t.imax):
        if int(t.alias[c]) == j and int(t.T[c]) < K:
            return c | ((K - 1) << (64 - t.abits))
    raise AssertionError("no column reaches j")


@pytest.fixture(scope="module")
def te(orc):
    return orc.tables(orc.EXP)


@pytest.fixture(scope="module")
def tn(orc):
    return orc.tables(orc.NORMAL)


# --------------------------------------------------------------------------
# scripted word streams
# --------------------------------------------------------------------------
def test_alias_word_helper(orc, te, tn):
    for t in (te, tn):
        for j in range(t.L + 1):
            assert orc.alias_pick(t, alias_word(t, j)) == j


def test_fast_path_is_U_times_X(orc, te, tn):
    rng = np.random.default_rng(1)
    for _ in range(200):
        i = int(rng.integers(0, te.L))
        m = int(rng.integers(0, 2**52))
        x, used, over, err = orc.sample_script(orc.EXP, [word(i, m)])
        assert (used, over, err) == (1, False, False)
        assert x == (m * 2.0**-52) * te.X[i]  # one IEEE rounding
        i = int(rng.integers(0, tn.L))
        s = int(rng.integers(0, 2))
        x, used, over, err = orc.sample_script(orc.NORMAL, [word(i, m, s)])
        assert used == 1 and not over
        assert x == (-1) ** s * ((m * 2.0**-52) * tn.X[i])


def test_fast_path_fp32(orc, te):
    m = 0x8_1234_5678_9ABC
    w = word(17, m)
    x, used, over, err = orc.sample_script(orc.EXP, [w], dtype=orc.F32)
    u32 = np.float32((w >> 41) * 2.0**-23)
    assert used == 1 and x == float(np.float32(u32 * np.float32(te.X32[17])))


def test_exponential_tail_is_X0_plus_exponential(orc, te):
    # i >= L, j = 0, then a fast-path word: X_0 + U X_5 (Sec. 2: the tail of
    # an exponential is itself exponential).
    m2 = 12345678901
    script = [word(253, 5), alias_word(te, 0), word(5, m2)]
    x, used, over, err = orc.sample_script(orc.EXP, script)
    assert used == 3 and not over
    assert x == te.X[0] + (m2 * 2.0**-52) * te.X[5]
    # two tail levels: inner sample first, then X_0 added twice
    script = [word(253, 5), alias_word(te, 0), word(255, 9), alias_word(te, 0), word(5, m2)]
    x, used, over, err = orc.sample_script(orc.EXP, script)
    assert used == 5
    assert x == te.X[0] + (te.X[0] + (m2 * 2.0**-52) * te.X[5])


def test_overhang_keeps_j_on_rejection(orc, te):
    j = 100
    # First attempt: ux = U_1 = 1/2, uy just under the chord: inside the
    # narrow band and above e^-x, so the exact test rejects.
    uy = 0.5 - 2.0**-30
    xx = fma(0.5, te.dX[j], te.X[j])
    assert fma(uy, te.df[j], te.f[j - 1]) > math.exp(-xx)
    # Second attempt (fresh ux, uy) deep under the chord: accepted in box j.
    script = [u_word(0.5) | 252, alias_word(te, j), u_word(uy), u_word(0.25), u_word(0.25)]
    x, used, over, err = orc.sample_script(orc.EXP, script)
    assert (used, over, err) == (5, False, False)
    assert x == fma(0.25, te.dX[j], te.X[j])
    assert te.X[j] <= x <= te.X[j - 1]


def test_overhang_reflection(orc, te):
    j = 37
    # ux + uy = 1.25 > 1: reflected to (1 - uy, 1 - ux) = (0.5, 0.25), whose
    # sum 0.75 lies below tau: accepted without an exact test.
    script = [u_word(0.75) | 254, alias_word(te, j), u_word(0.5)]
    x, used, over, err = orc.sample_script(orc.EXP, script)
    assert used == 3 and not over
    assert x == fma(0.5, te.dX[j], te.X[j])
    ok, xa = orc.overhang_attempt(te, j, 0.75, 0.5)
    assert ok and xa == x


def test_cap_is_reachable(orc, te, tn):
    # j = L is the box [0, X_{L-1}] x [f_{L-1}, P(0)] above the last layer.
    for dist, t in ((orc.EXP, te), (orc.NORMAL, tn)):
        script = [u_word(0.125) | 255, alias_word(t, t.L), u_word(0.0625)]
        x, used, over, err = orc.sample_script(dist, script)
        assert used == 3 and not over
        assert x == fma(0.125, t.dX[t.L], 0.0)
        assert 0 <= x <= t.X[t.L - 1]


def test_normal_overhang_keeps_j(orc, tn):
    j = 120
    xx = fma(0.5, tn.dX[j], tn.X[j])
    uy = 1 - 2.0**-10
    assert fma(uy, tn.df[j], tn.f[j - 1]) > math.exp(-(xx * xx) * 0.5)
    script = [u_word(0.5) | (1 << 8) | 254, alias_word(tn, j), u_word(uy),
              u_word(0.015625), u_word(0.015625)]
    x, used, over, err = orc.sample_script(orc.NORMAL, script)
    assert used == 5 and not over
    assert x == -fma(0.015625, tn.dX[j], tn.X[j])


def test_normal_tail_marsaglia_tsang(orc, te, tn):
    # Accept branch: E_1 = U X_10, E_2 = U' X_20; a = E_1 / X_0 (as E_1 *
    # RN(1/X_0)), accept when 2 E_2 > a^2, return X_0 + a.
    m1, m2 = 2**50, 2**51
    e1 = (m1 * 2.0**-52) * te.X[10]
    e2 = (m2 * 2.0**-52) * te.X[20]
    a = e1 * tn.rinv
    assert e2 + e2 > a * a
    script = [word(254, 3), alias_word(tn, 0), word(10, m1), word(20, m2)]
    x, used, over, err = orc.sample_script(orc.NORMAL, script)
    assert used == 4 and not over
    assert x == tn.X[0] + a
    # Reject branch first: E_2 = 0 cannot exceed a^2 > 0; then accept.
    script = [word(254, 3), alias_word(tn, 0), word(10, m1), word(20, 0),
              word(10, m1), word(20, m2)]
    x, used, over, err = orc.sample_script(orc.NORMAL, script)
    assert used == 6 and not over
    assert x == tn.X[0] + a


def test_loop_limits(orc, te):
    j = 100
    script = [u_word(0.5) | 252, alias_word(te, j), u_word(0.5 - 2.0**-30),
              u_word(0.25), u_word(0.25)]
    try:
        orc.set_limits(1, 16)
        x, used, over, err = orc.sample_script(orc.EXP, script)
        assert err and math.isnan(x) and used == 3
        orc.set_limits(64, 0)
        x, used, over, err = orc.sample_script(orc.EXP, [word(253, 5), alias_word(te, 0), word(5, 7)])
        assert err and math.isnan(x)
    finally:
        orc.set_limits(64, 16)
    x, used, over, err = orc.sample_script(orc.EXP, script)
    assert not err


# --------------------------------------------------------------------------
# exact enumeration at reduced width
# --------------------------------------------------------------------------
UB = 12  # U and alias-threshold bits at reduced width
IB = 3   # i_max = 8


def _composed_cdf(orc, dist, tpts):
    t8 = orc.tables(dist, IB, UB, UB)
    te8 = orc.tables(orc.EXP, IB, UB, UB)
    imax, L = t8.imax, t8.L
    N = 1 << UB
    # fast path through the sampler itself, every first word
    fast = []
    for i in range(imax):
        xs = []
        for m in range(N):
            w0 = (m << (64 - UB)) | i
            x, used, over, err = orc.sample_script(dist, [w0], te=te8, tn=t8)
            if i < L:
                assert used == 1 and not over
                xs.append(abs(x))
            else:
                assert over
        if i < L:
            fast.append(np.sort(np.array(xs)))
    # alias law, every alias word: exactly the integer weights
    counts = np.zeros(imax, dtype=np.int64)
    for c in range(imax):
        for th in range(N):
            counts[orc.alias_pick(t8, c | (th << (64 - UB)))] += 1
    assert [int(v) for v in counts] == [int(v) for v in list(t8.q)[:imax]]
    p = counts / counts.sum()
    # per-overhang accepted grid points
    boxes = {j: np.sort(orc.enum_overhang(t8, j, UB)) for j in range(1, L + 1)}
    X0 = t8.X[0]
    pf = (imax - L) / imax

    def F(t):
        if t < 0:
            return 0.0
        v = sum(np.searchsorted(a, t, side="right") / N for a in fast) / imax
        acc = sum(p[j] * np.searchsorted(boxes[j], t, side="right") / boxes[j].size
                  for j in range(1, L + 1))
        if dist == orc.EXP:
            tail = F(t - X0)
        else:
            # tail law: exact half-normal tail beyond X_0 (the MT step is
            # pinned separately by scripted and statistical tests)
            tail = 0.0 if t <= X0 else 1 - special.erfc(t / math.sqrt(2)) / special.erfc(X0 / math.sqrt(2))
        return v + pf * (acc + p[0] * tail)

    return np.array([F(t) for t in tpts]), t8


@pytest.mark.parametrize("dist", [0, 1])
def test_reduced_width_enumeration_matches_exact_cdf(orc, dist):
    tpts = np.linspace(0.0, 9.0 if dist == 0 else 4.5, 361)
    Fc, t8 = _composed_cdf(orc, dist, tpts)
    exact = 1 - np.exp(-tpts) if dist == 0 else special.erf(tpts / math.sqrt(2))
    dev = np.max(np.abs(Fc - exact))
    # Grid discretisation: at most one grid step (2^-12) of each layer's mass
    # for the fast path and a few steps of each overhang box.
    assert dev < 3.0 / (1 << UB), dev


def test_reduced_width_detects_planted_mistakes(orc):
    """The enumeration bound is tight enough to see plausible mistakes."""
    tpts = np.linspace(0.0, 9.0, 361)
    t8 = orc.tables(orc.EXP, IB, UB, UB)
    exact = 1 - np.exp(-tpts)
    A = np.array([t8.A[j] for j in range(t8.L + 1)])
    # Dropping the cap (j = L) and renormalising the others.
    A2 = A.copy()
    A2[-1] = 0
    A2 *= A.sum() / A2.sum()
    shift = np.max(np.abs(np.cumsum(A2 - A)))
    assert shift > 3.0 / (1 << UB)


# --------------------------------------------------------------------------
# full-width distribution tests
# --------------------------------------------------------------------------
N_STAT = 1 << 22


def _cdf(dist):
    return (lambda x: 1 - np.exp(-x)) if dist == 0 else special.ndtr


def _equiprob_edges(dist, k=1024):
    q = np.arange(1, k) / k
    return -np.log1p(-q) if dist == 0 else special.ndtri(q)


@pytest.mark.parametrize("keying", [0, 1])
@pytest.mark.parametrize("dist,dtype", [(0, 1), (1, 1), (0, 0), (1, 0)])
def test_distribution_full_width(orc, dist, dtype, keying):
    """Per-index keying (0) and packed keying (1) give the same laws."""
    x, errs, words, _ = orc.fill(dist, dtype, SEED, 0, N_STAT, want_words=True, keying=keying)
    assert errs == 0 and np.all(np.isfinite(x))
    x = x.astype(np.float64)
    # KS against the closed-form CDF
    ks = stats.kstest(x, _cdf(dist))
    assert ks.pvalue > 1e-4, ks
    # chi-square over 1024 equiprobable bins (df = 1023)
    cnt = np.bincount(np.searchsorted(_equiprob_edges(dist), x, side="right"), minlength=1024)
    chi2 = float(((cnt - N_STAT / 1024) ** 2 / (N_STAT / 1024)).sum())
    assert abs(chi2 - 1023) < 6 * math.sqrt(2 * 1023), chi2
    # raw moments within 5 standard errors of the closed forms
    if dist == 0:
        mom = [1, 2, 6, 24]
        var = [math.factorial(2 * k) - math.factorial(k) ** 2 for k in (1, 2, 3, 4)]
    else:
        mom = [0, 1, 0, 3]
        var = [1, 2, 15, 96]
    for k in range(4):
        est = float(np.mean(x ** (k + 1)))
        assert abs(est - mom[k]) < 5 * math.sqrt(var[k] / N_STAT), (k, est)
    # fast-path exit rate L/256 ("98.4% probability of exit at step 2")
    L = orc.tables(dist).L
    rate = float(np.mean(words == 1))
    p = L / 256
    assert abs(rate - p) < 5 * math.sqrt(p * (1 - p) / N_STAT)


def test_exponential_tail_law(orc, te):
    x, errs, _, _ = orc.fill(orc.EXP, orc.F64, SEED, 0, 1 << 24)
    tail = x[x > te.X[0]] - te.X[0]
    assert tail.size > 5000
    assert stats.kstest(tail, "expon").pvalue > 1e-4


def test_normal_tail_law(orc, tn):
    x, errs, _, _ = orc.fill(orc.NORMAL, orc.F64, SEED, 0, 1 << 25)
    X0 = tn.X[0]
    t = np.abs(x[np.abs(x) > X0])
    assert t.size > 5000
    den = special.erfc(X0 / math.sqrt(2))
    assert stats.kstest(t, lambda v: 1 - special.erfc(v / math.sqrt(2)) / den).pvalue > 1e-4
    # symmetric sign
    neg = int(np.sum(x < 0))
    assert abs(neg - x.size / 2) < 5 * math.sqrt(x.size / 4)


def test_fp32_tracks_fp64_on_same_counters(orc):
    n = 1 << 20
    for dist in (0, 1):
        x64, _, w64, _ = orc.fill(dist, orc.F64, SEED, 0, n, want_words=True)
        x32, _, w32, _ = orc.fill(dist, orc.F32, SEED, 0, n, want_words=True)
        fast = (w64 == 1) & (w32 == 1)
        assert np.array_equal(w64 == 1, w32 == 1)  # same layer index decision
        # U32 keeps the top 23 of U's 52 bits: |x32 - x64| <= X_i 2^-23 + ulp
        d = np.abs(x32[fast].astype(np.float64) - x64[fast])
        assert d.max() <= 7.6 * 2.0**-23 + 2.0**-21
        flips = float(np.mean(w64 != w32))
        assert flips < 1e-3


@pytest.mark.parametrize("dist,dtype", [(0, 1), (1, 1), (0, 0), (1, 0)])
def test_distribution_ten_bit_index(orc, dist, dtype):
    """i_max = 1024 (Appendix D item 1): i from bits 0-9, the normal's sign
    from bit 10, alias column from bits 0-9 and threshold from bits 10-63;
    the same laws, and step 2 exits at the rate L_max / 1024."""
    te, tn = orc.tables(0, 10, 52, 54), orc.tables(1, 10, 52, 54)
    x, errs, words, _ = orc.fill(dist, dtype, SEED, 0, N_STAT, want_words=True, te=te, tn=tn)
    assert errs == 0 and np.all(np.isfinite(x))
    x = x.astype(np.float64)
    assert stats.kstest(x, _cdf(dist)).pvalue > 1e-4
    cnt = np.bincount(np.searchsorted(_equiprob_edges(dist), x, side="right"), minlength=1024)
    chi2 = float(((cnt - N_STAT / 1024) ** 2 / (N_STAT / 1024)).sum())
    assert abs(chi2 - 1023) < 6 * math.sqrt(2 * 1023), chi2
    L = (te if dist == 0 else tn).L
    p = L / 1024
    rate = float(np.mean(words == 1))
    assert abs(rate - p) < 5 * math.sqrt(p * (1 - p) / N_STAT)
    if dist == 1:
        assert abs(float(np.mean(x > 0)) - 0.5) < 5 * math.sqrt(0.25 / N_STAT)


def test_fast_path_sign_and_zero(orc, te, tn):
    # Step 2 with the normal's sign: a negative draw is the exact negation
    # of the positive one; at U = 0 the value is a zero (reading R16 leaves
    # its sign bit open; the oracle's carries the draw's sign).
    rng = np.random.default_rng(5)
    for dtype, it in ((orc.F64, np.uint64), (orc.F32, np.uint32)):
        for _ in range(100):
            i = int(rng.integers(0, tn.L))
            m = int(rng.integers(1, 2**52))
            if dtype == orc.F32:
                m |= 1 << 29  # U's top 23 bits nonzero
            pos, *_ = orc.sample_script(orc.NORMAL, [word(i, m, 0)], dtype=dtype)
            neg, *_ = orc.sample_script(orc.NORMAL, [word(i, m, 1)], dtype=dtype)
            assert pos > 0 and neg == -pos
        for s in (0, 1):
            for dist, t in ((orc.NORMAL, tn), (orc.EXP, te)):
                x, used, over, err = orc.sample_script(dist, [word(5, 0, s if dist else 0)],
                                                       dtype=dtype)
                ft = np.float64 if dtype == orc.F64 else np.float32
                assert used == 1 and x == 0.0
                sign = (np.array([x], dtype=ft).view(it)[0] >> (63 if dtype == orc.F64 else 31))
                assert int(sign) == (s if dist == orc.NORMAL else 0)
