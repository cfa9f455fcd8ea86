"""Parity rule between the CUDA path and the CPU oracle.

Stated tolerance (FP64; applied to FP32 against the FP32 oracle as well):
  * uniform words and layer indices are bit-exact, so the fast-path
    outputs (one word consumed) must be bit-identical (a zero by value:
    the sign bit of a zero is not fixed, reading R16);
  * every other output must be identical too unless an accept/reject
    decision could have flipped: the oracle records, per output, the
    smallest gap |y - P(x)| of its exact rejection tests in FP64 ulps of
    P(x).  A mismatch is accepted as a flip only where that gap is <= 4 ulp
    (the device exp and the host libm exp may differ by an ulp), and flips
    may affect at most ceil(1e-9 n) outputs;
  * where no flip is possible the outputs may differ by at most 2 ulp (the
    rounding order of the fringe arithmetic is fixed, so in practice they
    are identical and the count of non-identical values is reported).
"""
import math

import numpy as np


def ulp_distance(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Distance in units in the last place between same-dtype arrays."""
    it = np.int64 if a.dtype == np.float64 else np.int32
    mag = np.int64((1 << 63) - 1) if a.dtype == np.float64 else np.int64((1 << 31) - 1)

    def line(x):
        i = x.view(it).astype(np.int64)
        return np.where(i < 0, -(i & mag), i)

    return np.abs(line(a) - line(b))


def check(gpu: np.ndarray, ref: np.ndarray, words: np.ndarray, margin: np.ndarray) -> dict:
    assert gpu.shape == ref.shape and gpu.dtype == ref.dtype
    n = gpu.size
    gnan, rnan = np.isnan(gpu), np.isnan(ref)
    assert np.array_equal(gnan, rnan), f"NaN positions differ at {np.nonzero(gnan != rnan)[0][:10]}"
    ok = ~gnan
    it = np.uint64 if gpu.dtype == np.float64 else np.uint32
    # a zero compares by value: the library's is +0 for either sign, the
    # oracle's carries the normal's sign bit (reading R16)
    same = (gpu.view(it) == ref.view(it)) | (gpu == ref)
    same |= gnan
    fast = words == 1
    bad_fast = np.nonzero(fast & ~same)[0]
    assert bad_fast.size == 0, f"fast-path mismatch at {bad_fast[:10]}: {gpu[bad_fast[:5]]} vs {ref[bad_fast[:5]]}"
    diff = np.nonzero(~same & ok)[0]
    flips = diff[margin[diff] <= 4.0]
    other = diff[margin[diff] > 4.0]
    if other.size:
        d = ulp_distance(gpu[other], ref[other])
        assert d.max() <= 2, f"fringe mismatch beyond 2 ulp at {other[:10]}: {gpu[other[:5]]} vs {ref[other[:5]]}"
    assert flips.size <= max(1, math.ceil(1e-9 * n)), f"{flips.size} flipped decisions"
    return dict(n=n, fringe=int((~fast).sum()), flips=int(flips.size), ulp_diff=int(other.size))


# ---------------------------------------------------------------------------
# Batched requests
# ---------------------------------------------------------------------------
# The oracle's value of element t of a request is the plain map of its
# standard variate z (a draw of the rules above): exponential with rate
# lambda RN(z * s), s = RN(1/lambda); normal RN(sigma z + mu) (one fma).
# The library computes exactly that for every draw that leaves the fast
# path.  For a fast-path draw (step 2 of Table 1, z = +-RN(U X_i)) it folds
# the map into the step's one rounding:
#     y_lib = RN((1 + U)(+-B_i) + D),  B_i = RN(s X_i),  D = RN(m -+ B_i)
# (s = RN(1/lambda), m = 0 for the exponential; s = sigma, m = mu for the
# normal; FP32 requests in binary32 with RN32 of s and m).  With unit
# roundoff u (2^-53, 2^-24) and T = m +- s U X_i the exact map of the exact
# fast-path value:
#     |y_lib - T| <= u|T| + u s U X_i + u|m -+ s X_i|   (the last term is 0
#                                                          when m = 0: D = -+B_i exactly)
#     |y_orc - T| <= u|T| + u s U X_i
# to first order, and s U X_i <= |T| + |m|, so
#     |y_lib - y_orc| <= 4u|y_orc| + 2u|m| + u|m -+ s X_i|   (normal)
#     |y_lib - y_orc| <= 4u|y_orc|                           (exponential),
# applied below with a factor 1 + 2^-20 for the second-order terms.
FOLD_SLACK = 1.0 + 2.0**-20


def fold_bound(dist: int, dtype: int, y_orc: np.ndarray, w0: np.ndarray, X: np.ndarray,
               p0: float, p1: float) -> np.ndarray:
    """Largest |y_lib - y_orc| allowed for fast-path draws with first words
    w0 (layer index in bits 0-7, the normal's sign in bit 8), table X (the
    dtype's X_i) and the request parameters (p0, p1)."""
    u = 2.0**-53 if dtype == 1 else 2.0**-24
    y = np.abs(np.asarray(y_orc, dtype=np.float64))
    if dist == 0:
        return 4 * u * y * FOLD_SLACK
    cast = (lambda v: float(v)) if dtype == 1 else (lambda v: float(np.float32(v)))
    m, s = cast(p0), cast(p1)
    i = (w0 & np.uint64(0xFF)).astype(np.int64)
    neg = ((w0 >> np.uint64(8)) & np.uint64(1)).astype(bool)
    sx = s * np.asarray(X, dtype=np.float64)[i]
    d = np.abs(np.where(neg, m + sx, m - sx))
    return (4 * u * y + 2 * u * abs(m) + u * d) * FOLD_SLACK


def check_batch(orc, q: dict, got: np.ndarray, idx: np.ndarray) -> dict:
    """Compare a batched request's outputs at positions idx with the
    oracle's plain map: draws outside the fast path by check() (bit-exact
    up to flipped decisions), fast-path draws within fold_bound()."""
    idx = np.ascontiguousarray(idx, dtype=np.uint64)
    ft = np.float64 if q["dtype"] == 1 else np.float32
    got = np.asarray(got, dtype=ft)
    ref = orc.request_values(q, idx).astype(ft)
    _, _, words, margin = orc.fill(q["dist"], q["dtype"], q["seed"], q["offset"], 0, idx=idx,
                                   want_words=True, want_margin=True)
    fast = words == 1
    out = check(got[~fast], ref[~fast], words[~fast], margin[~fast]) if (~fast).any() else {}
    if fast.any():
        assert not np.isnan(got[fast]).any()
        w0 = orc.first_words(q["seed"], q["offset"], idx[fast])
        t = orc.tables(q["dist"])
        X = np.ctypeslib.as_array(t.X) if q["dtype"] == 1 else np.ctypeslib.as_array(t.X32)
        bound = fold_bound(q["dist"], q["dtype"], ref[fast], w0, X, q["p0"], q["p1"])
        err = np.abs(got[fast].astype(np.float64) - ref[fast].astype(np.float64))
        worst = int(np.argmax(err - bound))
        assert np.all(err <= bound), (
            f"fast-path fold beyond its bound at {idx[fast][worst]}: "
            f"{got[fast][worst]!r} vs {ref[fast][worst]!r} (bound {bound[worst]:.3g})")
        out["fast"] = int(fast.sum())
        out["fast_exact"] = int((got[fast] == ref[fast]).sum())
        out["fast_max_over_bound"] = float(np.max(np.where(bound > 0, err / np.where(bound > 0, bound, 1), 0)))
    return out
