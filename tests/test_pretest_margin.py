"""The fringe's FP32 pre-test never changes an accept/reject decision.

On the device, the exact test y < exp(-a) of an overhang attempt is first
made in FP32 on approximations xa, ya of x and y (from the top 24 bits of
the uniforms and the binary32 tables) and answers only outside a relative
margin of 2^-14 around the curve.  This checks, with numpy's float32
arithmetic standing in for the device's, that the combined error of those
approximations and of a 2-ulp expf stays below 2^-17 relative, for every
overhang box of both distributions, at random and extreme uniforms.
"""
import numpy as np
import pytest

MARGIN = 2.0**-14
CLAIM = 2.0**-17


def _f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32)


@pytest.mark.parametrize("dist", [0, 1])
def test_fp32_pretest_error_below_margin(orc, dist):
    t = orc.tables(dist)
    rng = np.random.default_rng(17 + dist)
    m = 4096
    worst = 0.0
    for j in range(1, t.L + 1):
        mx = np.concatenate([rng.integers(0, 2**52, size=m, dtype=np.uint64),
                             np.array([0, 2**52 - 1, 2**51, 2**52 - 2**28], dtype=np.uint64)])
        my = np.concatenate([rng.integers(0, 2**52, size=m, dtype=np.uint64),
                             np.array([2**52 - 1, 0, 2**51, 2**28], dtype=np.uint64)])
        ux = mx.astype(np.float64) * 2.0**-52
        uy = my.astype(np.float64) * 2.0**-52
        # exact FP64 quantities of the oracle (a*b+c with one rounding is
        # emulated closely enough by float64 arithmetic for an error bound)
        x = ux * t.dX[j] + t.X[j]
        y = uy * t.df[j] + t.f[j - 1]
        a = x if dist == 0 else 0.5 * x * x
        exact = y / np.exp(-a)
        # device FP32 approximations
        ua = _f32((mx >> np.uint64(28)).astype(np.float64) * 2.0**-24)
        va = _f32((my >> np.uint64(28)).astype(np.float64) * 2.0**-24)
        xa = _f32(ua.astype(np.float64) * float(t.dX32[j]) + float(t.X32[j]))
        ya = _f32(va.astype(np.float64) * float(t.df32[j]) + float(t.f32[j - 1]))
        aa = xa if dist == 0 else (np.float32(0.5) * xa) * xa
        e = np.exp(-aa.astype(np.float64))
        for ulps in (-2, 2):  # expf within 2 ulp
            e2 = _f32(e) + ulps * np.spacing(_f32(e))
            approx = ya.astype(np.float64) / e2.astype(np.float64)
            worst = max(worst, float(np.max(np.abs(approx / exact - 1))))
    print(f"worst relative error {worst:.3e}")
    assert worst < CLAIM, worst
    assert CLAIM * 4 <= MARGIN
