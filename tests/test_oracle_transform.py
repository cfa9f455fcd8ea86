"""Pins for the oracle's batched-request transforms (exponential with rate
lambda: X RN(1/lambda); normal: fma(sigma, Z, mu)), against exact rational
arithmetic and the distributions they must produce; the transform applies
to every draw of a request."""
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


def test_request_values_map_every_draw_plainly(orc):
    """request_values is the plain map of the oracle's standard variate for
    every draw, fast path or fringe, in both precisions."""
    n = 20000
    idx = np.arange(n, dtype=np.uint64)
    for dist, p0, p1 in ((0, 3.7, 0.0), (1, 1.25, 0.3)):
        for dtype in (1, 0):
            q = dict(dist=dist, dtype=dtype, seed=21, offset=2**32 - 5000, p0=p0, p1=p1)
            got = orc.request_values(q, idx)
            x, _, words, _ = orc.fill(dist, dtype, q["seed"], q["offset"], n, want_words=True)
            assert 0.98 < float(np.mean(words == 1)) < 1.0
            want = np.array([orc.transform(dist, dtype, float(v), p0, p1) for v in x])
            assert np.array_equal(got, want)


def test_first_words_are_the_stream_heads(orc):
    idx = np.array([0, 1, 7, 2**32 - 3, 12345], dtype=np.uint64)
    w = orc.first_words(99, 2**32 - 2, idx)
    for k, g in enumerate(idx):
        assert int(w[k]) == orc.philox_words(99, (2**32 - 2 + int(g)) % 2**64, 1)[0]
