"""Pins for the oracle's batched-request transforms (exponential with rate
lambda: X / lambda; normal: mu + sigma Z), against exact rational
arithmetic and the distributions they must produce."""
import math
from fractions import Fraction

import numpy as np
from scipy import stats


def test_transform_is_correctly_rounded(orc):
    rng = np.random.default_rng(3)
    for _ in range(500):
        x = float(rng.exponential())
        lam = float(10 ** rng.uniform(-1, 1))
        inv = float(Fraction(1) / Fraction(lam))  # RN(1/lambda)
        assert orc.transform(0, 1, x, lam, 0.0) == float(Fraction(x) * Fraction(inv))
        z, mu, sd = float(rng.normal()), float(rng.uniform(-5, 5)), float(10 ** rng.uniform(-2, 2))
        assert orc.transform(1, 1, z, mu, sd) == float(Fraction(sd) * Fraction(z) + Fraction(mu))
        # FP32: RN32 of the FP64 reciprocal, binary32 product / fma
        xf = np.float32(x)
        inv32 = np.float32(inv)
        assert orc.transform(0, 0, float(xf), lam, 0.0) == float(np.float32(float(Fraction(float(xf)) * Fraction(float(inv32)))))
        zf, muf, sdf = np.float32(z), np.float32(mu), np.float32(sd)
        exact = Fraction(float(sdf)) * Fraction(float(zf)) + Fraction(float(muf))
        assert orc.transform(1, 0, float(zf), mu, sd) == float(np.float32(float(exact)))


def test_request_values_have_the_requested_law(orc):
    n = 1 << 18
    idx = np.arange(n, dtype=np.uint64)
    e = orc.request_values(dict(dist=0, dtype=1, seed=5, offset=0, p0=4.0, p1=0.0), idx)
    assert stats.kstest(e, stats.expon(scale=0.25).cdf).pvalue > 1e-4
    g = orc.request_values(dict(dist=1, dtype=0, seed=6, offset=0, p0=-2.5, p1=3.0), idx)
    assert stats.kstest(g, stats.norm(loc=-2.5, scale=3.0).cdf).pvalue > 1e-4
    assert abs(g.mean() + 2.5) < 5 * 3.0 / math.sqrt(n)


def test_fast_path_requests_fold_the_map_into_one_rounding(orc):
    """A request's fast-path value is RN((1 + U)(+-B_i) + D) with B_i =
    RN(s X_i), D = RN(m -+ B_i) (exact rationals below), and lies within
    the roundings of B_i and D of the exact m + s U X_i."""
    rng = np.random.default_rng(11)
    for dist in (0, 1):
        t = orc.tables(dist)
        for _ in range(400):
            i = int(rng.integers(0, t.L))
            sign = int(rng.integers(0, 2)) if dist == 1 else 0
            m52 = int(rng.integers(0, 2**52))
            w0 = (m52 << 12) | (sign << 8) | i
            if dist == 0:
                lam = float(10 ** rng.uniform(-1, 1))
                p0, p1, s, mm = lam, 0.0, float(Fraction(1) / Fraction(lam)), 0.0
            else:
                p0, p1 = float(rng.uniform(-5, 5)), float(10 ** rng.uniform(-2, 2))
                s, mm = p1, p0
            # FP64
            B = float(Fraction(s) * Fraction(t.X[i]))
            D = float(Fraction(mm) + Fraction(B)) if sign else float(Fraction(mm) - Fraction(B))
            one_u = Fraction(2**52 + m52, 2**52)
            want = float(one_u * Fraction(-B if sign else B) + Fraction(D))
            got = orc.request_fast(dist, 1, w0, p0, p1)
            assert got == want
            exact = Fraction(mm) + (-1 if sign else 1) * Fraction(s) * Fraction(m52, 2**52) * Fraction(t.X[i])
            bound = 2 * (math.ulp(abs(B)) + math.ulp(abs(D)) + math.ulp(abs(got)))
            assert abs(Fraction(got) - exact) <= Fraction(bound)
            # FP32: binary32 B, D and fma from RN32 of the FP64 s and m
            s32, m32 = np.float32(s), np.float32(mm)
            B32 = np.float32(float(Fraction(float(s32)) * Fraction(float(t.X32[i]))))
            D32 = np.float32(float(Fraction(float(m32)) + Fraction(float(B32)) if sign
                                   else Fraction(float(m32)) - Fraction(float(B32))))
            m23 = m52 >> 29
            w32 = (m23 << 41) | (sign << 8) | i
            one_u32 = Fraction(2**23 + m23, 2**23)
            want32 = float(np.float32(float(one_u32 * Fraction(-float(B32) if sign else float(B32))
                                            + Fraction(float(D32)))))
            assert orc.request_fast(dist, 0, w32, p0, p1) == want32


def test_request_values_use_the_fast_path_form(orc):
    """request_values gives the folded form exactly on fast-path draws and
    the transformed variate elsewhere."""
    q = dict(dist=1, dtype=1, seed=21, offset=2**32 - 5000, p0=1.25, p1=0.3)
    n = 20000
    idx = np.arange(n, dtype=np.uint64)
    got = orc.request_values(q, idx)
    x, _, words, _ = orc.fill(1, 1, q["seed"], q["offset"], n, want_words=True)
    fast = words == 1
    assert 0.98 < fast.mean() < 1.0
    w0 = [orc.philox_words(q["seed"], q["offset"] + k, 1)[0] for k in range(n)]
    for k in range(n):
        if fast[k]:
            assert got[k] == orc.request_fast(1, 1, w0[k], q["p0"], q["p1"])
        else:
            assert got[k] == orc.transform(1, 1, float(x[k]), q["p0"], q["p1"])
