"""Parity rule between the CUDA path and the CPU oracle.

Stated tolerance (FP64; applied to FP32 against the FP32 oracle as well):
  * uniform words and layer indices are bit-exact, so the fast-path
    outputs (one word consumed) must be bit-identical;
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
    same = gpu.view(it) == ref.view(it)
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
