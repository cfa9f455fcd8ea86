"""Pins for the oracle's fused-reduction reference (power sums + histogram).

The sums are checked against exact rational arithmetic over the oracle's own
samples (Fraction), the histogram against an independent numpy binning of the
same samples: bin = floor(256 x) + 2048 on [-8, 8), 4096 below, 4097 above.
"""
from fractions import Fraction

import numpy as np


import pytest


@pytest.mark.parametrize("keying", [0, 1])
def test_moments_and_histogram_match_plain_definitions(orc, keying):
    seed, off, n = 0x0123456789ABCDEF, 1001, 1 << 14
    for dist, dtype in ((1, 0), (0, 1), (1, 1)):
        x, errs, _, _ = orc.fill(dist, dtype, seed, off, n, keying=keying)
        sums, abss, hist, e2 = orc.moments(dist, dtype, seed, off, n, keying=keying)
        assert errs == 0 and e2 == 0
        xs = [Fraction(float(v)) for v in x]
        for k in range(4):
            exact = sum(v ** (k + 1) for v in xs)
            exact_abs = sum(abs(v) ** (k + 1) for v in xs)
            assert abs(Fraction(float(sums[k])) - exact) <= abs(exact) * Fraction(1, 2**52) + Fraction(1, 2**100)
            assert abs(Fraction(float(abss[k])) - exact_abs) <= exact_abs * Fraction(1, 2**52)
        xd = x.astype(np.float64)
        b = np.where(xd < -8, 4096, np.where(xd >= 8, 4097, np.floor(256 * xd) + 2048)).astype(np.int64)
        ref = np.bincount(b, minlength=4098)
        assert np.array_equal(hist.astype(np.int64), ref)
        assert int(hist.sum()) == n


def test_histogram_edges(orc):
    """Values on bin edges go to the bin they open."""
    xs = np.array([-8.0, -8.0 + 1 / 256, -1 / 512, 0.0, 7.99609375, 8.0, -8.000001])
    b = np.where(xs < -8, 4096, np.where(xs >= 8, 4097, np.floor(256 * xs) + 2048))
    assert list(b.astype(int)) == [0, 1, 2047, 2048, 4095, 4097, 4096]
