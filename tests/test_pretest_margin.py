"""The fringe's FP32 pre-test never changes an accept/reject decision.

On the device, the exact test y < exp(-a) of an overhang attempt is first
made in FP32 on approximations xa, ya of x and y (from the top 24 bits of
the uniforms and the binary32 tables) and answers only outside a relative
margin of 2^-17 around the curve.  Two checks that the approximation error
stays well inside that margin, for every overhang box of both distributions
at both table widths (i_max 256 and 1024) and both output precisions:

* an a-priori bound, from the error of each approximation step (24-bit
  uniforms, binary32 tables, one rounding per FP32 operation, expf within
  2 ulp), is at most 2^-18 and leaves the margin decisive;
* numpy's float32 arithmetic, standing in for the device's, at random and
  extreme uniforms, stays below 2^-19 (measured worst 1.1e-6).
"""
import math

import numpy as np
import pytest

MARGIN = 2.0**-17
BOUND = 2.0**-18   # a-priori bound on the relative error of ya / expf(-aa)
SAMPLED = 2.0**-19  # sampled worst case must stay below this
U32 = 2.0**-24      # binary32 unit roundoff
EXPF_REL = 2.0 * 2.0**-23  # 2 ulp of expf, relative

TABLES = [(8, 56), (10, 54)]  # (index bits, alias bits) of the two table widths


def _f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def _tab(orc, dist, ib, ab):
    return orc.tables(dist, ib, 52, ab)


def apriori_bound(t, dist, j, fp64):
    """Upper bound on |(ya / e) / (y / exp(-a)) - 1| over box j.

    FP64 outputs: x = X_j + U_x dX_j and y = f_{j-1} + U_y df_j in FP64;
    xa = RN32(ua dX32_j + X32_j) with ua the top 24 bits of U_x
    (0 <= U_x - ua < 2^-24), so |xa - x| <= u (2 |dX| + |X_j| + x_max);
    likewise ya.  FP32 outputs: x and y are themselves those FP32 values,
    so xa = x and ya = y exactly.  Normal: aa = RN32(RN32(xa / 2) xa) adds
    one rounding; a = x^2 / 2 moves by at most |xa - x| (x_max + |xa - x| / 2).
    expf adds 2 ulp."""
    X, dX, f, df = t.X[j], t.dX[j], t.f[j - 1], t.df[j]
    xmax = max(X, X + dX)
    ymin, ymax = min(f, f + df), max(f, f + df)
    if fp64:
        dx = U32 * (2 * abs(dX) + abs(X) + xmax) * (1 + 4 * U32)
        dy = U32 * (2 * abs(df) + f + ymax) * (1 + 4 * U32)
    else:
        dx = dy = 0.0
    if dist == 0:
        da = dx
    else:
        da = dx * (xmax + dx / 2) + U32 * 0.5 * (xmax + dx) ** 2
    re = math.expm1(da) + EXPF_REL
    ry = dy / ymin
    return (1 + ry) / (1 - re) - 1


@pytest.mark.parametrize("ib,ab", TABLES)
@pytest.mark.parametrize("dist", [0, 1])
def test_apriori_bound_below_margin(orc, dist, ib, ab):
    t = _tab(orc, dist, ib, ab)
    worst = max(apriori_bound(t, dist, j, fp64) for j in range(1, t.L + 1)
                for fp64 in (True, False))
    print(f"a-priori bound {worst:.3e} (2^{math.log2(worst):.2f})")
    assert worst <= BOUND
    # reject (ya > RN32(e (1 + m))) implies y / exp(-a) >= 1; accept
    # (ya < RN32(e (1 - m))) implies y / exp(-a) < 1; 1 +- m is exact in FP32
    assert (1 + MARGIN) * (1 - U32) >= 1 + BOUND
    assert (1 - MARGIN) * (1 + U32) < 1 - BOUND


def _uniforms(rng, m, bits):
    top = 2**bits
    mx = np.concatenate([rng.integers(0, top, size=m, dtype=np.uint64),
                         np.array([0, top - 1, top // 2, top - 2**(bits - 24)], dtype=np.uint64)])
    my = np.concatenate([rng.integers(0, top, size=m, dtype=np.uint64),
                         np.array([top - 1, 0, top // 2, 2**(bits - 24)], dtype=np.uint64)])
    return mx, my


@pytest.mark.parametrize("ib,ab", TABLES)
@pytest.mark.parametrize("dist", [0, 1])
def test_fp32_pretest_error_fp64_outputs(orc, dist, ib, ab):
    t = _tab(orc, dist, ib, ab)
    rng = np.random.default_rng(17 + dist + ib)
    worst = 0.0
    for j in range(1, t.L + 1):
        mx, my = _uniforms(rng, 2048, 52)
        ux = mx.astype(np.float64) * 2.0**-52
        uy = my.astype(np.float64) * 2.0**-52
        # FP64 quantities of the exact test (float64 a*b+c stands in for
        # the FMA closely enough for an error bound)
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
    assert worst < SAMPLED, worst


@pytest.mark.parametrize("ib,ab", TABLES)
@pytest.mark.parametrize("dist", [0, 1])
def test_fp32_pretest_error_fp32_outputs(orc, dist, ib, ab):
    """FP32 outputs: x, y are the FP32 values the pre-test also uses; only
    the product a (normal) and expf differ from the FP64 test of them."""
    t = _tab(orc, dist, ib, ab)
    rng = np.random.default_rng(29 + dist + ib)
    worst = 0.0
    for j in range(1, t.L + 1):
        mx, my = _uniforms(rng, 2048, 23)
        ua = _f32(mx.astype(np.float64) * 2.0**-23)
        va = _f32(my.astype(np.float64) * 2.0**-23)
        xa = _f32(ua.astype(np.float64) * float(t.dX32[j]) + float(t.X32[j]))
        ya = _f32(va.astype(np.float64) * float(t.df32[j]) + float(t.f32[j - 1]))
        xd = xa.astype(np.float64)
        a = xd if dist == 0 else 0.5 * xd * xd
        exact = ya.astype(np.float64) / np.exp(-a)
        aa = xa if dist == 0 else (np.float32(0.5) * xa) * xa
        e = np.exp(-aa.astype(np.float64))
        for ulps in (-2, 2):
            e2 = _f32(e) + ulps * np.spacing(_f32(e))
            approx = ya.astype(np.float64) / e2.astype(np.float64)
            worst = max(worst, float(np.max(np.abs(approx / exact - 1))))
    print(f"worst relative error {worst:.3e}")
    assert worst < SAMPLED, worst


def test_margin_matches_the_kernel():
    """The margin the kernel source uses is the one proved here."""
    import pathlib
    import re
    src = (pathlib.Path(__file__).resolve().parents[1] / "paper_1403_6870_gb300" / "csrc"
           / "zig_device.cuh").read_text()
    m = re.search(r"constexpr float kPreTestMargin = 1\.0f / (\d+)\.0f;", src)
    assert m is not None
    assert 1.0 / int(m.group(1)) == MARGIN
