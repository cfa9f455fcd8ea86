"""The tolerance of batched fast-path draws (tests/parity.py fold_bound)
holds for the folded arithmetic the library uses.

The oracle defines a batched request's value as the plain map of the
standard variate (exponential z * RN(1/lambda), normal fma(sigma, z, mu)).
The library rounds a fast-path draw once as RN((1 + U)(+-B_i) + D) with
B_i = RN(s X_i) and D = RN(m -+ B_i).  Here that folded value is formed in
exact rational arithmetic with one correct rounding per step, on random
and adversarial draws (cancellation of mu against sigma z, tiny sigma
beside a large mu, m = 0, U = 0, the largest and smallest X_i), and
compared with the oracle's plain value under the bound the GPU test uses.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from parity import fold_bound


def rn(q: Fraction, bits: int) -> float:
    """q rounded to nearest-even with a `bits`-bit significand (normal range)."""
    if q == 0:
        return 0.0
    neg = q < 0
    a = -q if neg else q
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    # a in [2^e, 2^(e+1)): scale to [2^(bits-1), 2^bits)
    sc = a / Fraction(2) ** (e - bits + 1)
    n, r = divmod(sc.numerator, sc.denominator)
    if 2 * r > sc.denominator or (2 * r == sc.denominator and n & 1):
        n += 1
    v = math.ldexp(float(n), e - bits + 1)
    return -v if neg else v


def fold(dist, dtype, m52, i, neg, X, p0, p1):
    """The library's folded fast-path value, exactly rounded per step."""
    bits = 53 if dtype == 1 else 24
    ubits = 52 if dtype == 1 else 23
    m = m52 if dtype == 1 else m52 >> 29
    if dist == 0:
        s = float(Fraction(1) / Fraction(p0))  # RN64(1/lambda), then RN32 for FP32
        s = s if dtype == 1 else rn(Fraction(s), 24)
        mu = 0.0
    else:
        s = p1 if dtype == 1 else rn(Fraction(p1), 24)
        mu = p0 if dtype == 1 else rn(Fraction(p0), 24)
    B = rn(Fraction(s) * Fraction(X[i]), bits)
    sB = -B if neg else B
    D = rn(Fraction(mu) - Fraction(sB), bits)
    one_u = Fraction(2**ubits + m, 2**ubits)
    return rn(one_u * Fraction(sB) + Fraction(D), bits)


def plain(orc, dist, dtype, m52, i, neg, X, p0, p1):
    """The oracle's value: its transform of the standard fast-path variate."""
    bits = 53 if dtype == 1 else 24
    ubits = 52 if dtype == 1 else 23
    m = m52 if dtype == 1 else m52 >> 29
    z = rn(Fraction(m, 2**ubits) * Fraction(X[i]), bits)
    z = -z if neg else z
    return orc.transform(dist, dtype, z, p0, p1)


@pytest.mark.parametrize("dtype", [1, 0])
@pytest.mark.parametrize("dist", [0, 1])
def test_fold_within_bound(orc, dist, dtype):
    t = orc.tables(dist)
    X = np.ctypeslib.as_array(t.X if dtype == 1 else t.X32).astype(np.float64)
    rng = np.random.default_rng(1000 + 2 * dist + dtype)
    worst = 0.0
    cases = 0
    for k in range(3000):
        i = int(rng.integers(0, t.L)) if k % 7 else int(rng.choice([0, 1, t.L - 1]))
        neg = bool(rng.integers(0, 2)) if dist == 1 else False
        m52 = int(rng.integers(0, 2**52)) if k % 11 else int(rng.choice([0, 1, 2**52 - 1]))
        if dist == 0:
            p0, p1 = float(10 ** rng.uniform(-1, 1)), 0.0
        else:
            p1 = float(10 ** rng.uniform(-2, 2))
            kind = k % 4
            if kind == 0:
                p0 = float(rng.uniform(-5, 5))
            elif kind == 1:  # mu cancels sigma z
                z = (m52 / 2**52) * X[i] * (-1 if neg else 1)
                p0 = float(-p1 * z * (1 + rng.uniform(-1e-6, 1e-6)))
            elif kind == 2:  # large mu, tiny sigma
                p0, p1 = float(rng.uniform(-5, 5)), float(10 ** rng.uniform(-2, -1))
            else:
                p0 = 0.0
        y_lib = fold(dist, dtype, m52, i, neg, X, p0, p1)
        y_orc = plain(orc, dist, dtype, m52, i, neg, X, p0, p1)
        w0 = np.array([(m52 << 12) | (int(neg) << 8) | i], dtype=np.uint64)
        b = float(fold_bound(dist, dtype, np.array([y_orc]), w0, X, p0, p1)[0])
        err = abs(y_lib - y_orc)
        assert err <= b, (dist, dtype, i, neg, m52, p0, p1, y_lib, y_orc, b)
        if b > 0:
            worst = max(worst, err / b)
        cases += 1
    assert cases == 3000 and worst <= 1.0


def test_bound_is_a_few_ulps_without_cancellation(orc):
    """Away from cancellation the bound is a few ulps of the output."""
    t = orc.tables(1)
    X = np.ctypeslib.as_array(t.X).astype(np.float64)
    rng = np.random.default_rng(7)
    for _ in range(500):
        i = int(rng.integers(0, t.L))
        m52 = int(rng.integers(2**50, 2**52))
        p0, p1 = 0.5, 2.0
        y = 0.5 + 2.0 * (m52 / 2**52) * X[i]
        w0 = np.array([(m52 << 12) | i], dtype=np.uint64)
        b = float(fold_bound(1, 1, np.array([y]), w0, X, p0, p1)[0])
        assert b <= 16 * math.ulp(max(abs(y), abs(p0) + p1 * X[i]))
    # the exponential's bound is 4 units of roundoff of the output
    assert fold_bound(0, 1, np.array([1.5]), np.array([0], dtype=np.uint64), X, 2.0, 0.0)[0] \
        <= 4 * 2.0**-53 * 1.5 * (1 + 2.0**-19)
