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
