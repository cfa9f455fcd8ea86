"""The integer-built uniform of the packed-keying fringe stages.

Prec<double>::val_int forms U = m 2^-52 (m an integer, 0 <= m <= 2^52)
without the FP64 pipe: m's leading one is shifted to bit 52 and the biased
exponent 1033 - clz64(m) is added beneath it (the leading one carries into
the exponent field), m = 0 giving +0.  This checks that construction
against exact arithmetic for every leading-zero count, the ends of the
range and random m, and that the kernel source uses the same constants.
"""
import pathlib
import re
from fractions import Fraction

import numpy as np

SRC = pathlib.Path(__file__).resolve().parents[1] / "paper_1403_6870_gb300" / "csrc" / "zig_device.cuh"


def val_int(m: int) -> float:
    lz = 64 - m.bit_length()
    bits = ((m << ((lz - 11) & 63)) + ((1033 - lz) << 52)) & (2**64 - 1)
    return 0.0 if m == 0 else float(np.array([bits], dtype=np.uint64).view(np.float64)[0])


def test_every_leading_zero_count_and_the_ends():
    ms = [0, 1, 2, 3, 2**52 - 1, 2**52, 2**51, 2**51 + 1]
    for k in range(53):
        ms += [2**k, 2**k + 1 if k else 1, 2**(k + 1) - 1]
    for m in ms:
        assert Fraction(val_int(m)) == Fraction(m, 2**52), m
    assert np.signbit(val_int(0)) == False  # noqa: E712


def test_random_significands():
    rng = np.random.default_rng(52)
    for m in rng.integers(0, 2**52, size=200000, dtype=np.uint64).tolist():
        assert val_int(m) == m * 2.0**-52  # exact: m has at most 52 bits


def test_kernel_uses_these_constants():
    src = SRC.read_text()
    body = src[src.index("double val_int(UInt m)"):]
    body = body[:body.index("}")]
    assert "__clzll" in body
    assert re.search(r"m << \(\(lz - 11\) & 63\)", body)
    assert re.search(r"\(1033 - lz\) << 52", body)
    assert "m == 0 ? 0.0" in body
