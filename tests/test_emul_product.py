"""The library's integer-emulated fast-path product (csrc/zig_emul.h)
equals the IEEE product RN(U X_i) bit for bit.

Table 1 step 2 returns U X_i rounded once; the library can form that
rounding from integers instead of a binary64 fused multiply-add.  The host
build of the same function is compared with numpy's binary64
multiplication (correctly rounded, with U = m 2^-52 exact) on 2^24 random
(m, X_i) pairs over both distributions' tables and random significands,
every power-of-two m, exact rounding ties, rounding carries into the
exponent, negative X (the normal's sign) and m = 0.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1403_6870_gb300", "csrc")


@pytest.fixture(scope="module")
def emul(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("emul") / "libemul.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", f"-I{CSRC}",
                    os.path.join(HERE, "emul_check.cpp"), "-o", so], check=True)
    lib = ctypes.CDLL(so)
    lib.emul_batch.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_uint64]

    def run(m, x):
        m = np.ascontiguousarray(m, dtype=np.uint64)
        xb = np.ascontiguousarray(np.asarray(x, dtype=np.float64)).view(np.uint64)
        out = np.empty(m.size, dtype=np.uint64)
        lib.emul_batch(m.ctypes.data, xb.ctypes.data, out.ctypes.data, m.size)
        return out

    return run


def ieee(m, x):
    """RN(m 2^-52 x): m 2^-52 is exact in binary64, the product rounds once."""
    u = np.ldexp(np.asarray(m, dtype=np.uint64).astype(np.float64), -52)
    r = u * np.asarray(x, dtype=np.float64)
    return np.where(np.asarray(m) == 0, 0.0, r).view(np.uint64)  # U = 0 gives +0


def test_random_pairs_over_the_tables(emul, orc):
    rng = np.random.default_rng(52)
    xs = []
    for dist in (0, 1):
        t = orc.tables(dist)
        xs.append(np.ctypeslib.as_array(t.X)[:t.L].astype(np.float64))
    X = np.concatenate(xs)
    n = 1 << 24
    for chunk in range(4):
        m = rng.integers(0, 2**52, size=n // 4, dtype=np.uint64)
        x = X[rng.integers(0, X.size, size=n // 4)]
        x = np.where(rng.integers(0, 2, size=x.size) == 1, -x, x)  # the normal's sign
        assert np.array_equal(emul(m, x), ieee(m, x))


def test_random_significands_and_small_m(emul):
    rng = np.random.default_rng(53)
    n = 1 << 20
    x = np.ldexp(1.0 + rng.random(n), rng.integers(-40, 40, size=n))
    shift = rng.integers(0, 52, size=n).astype(np.uint64)
    m = rng.integers(1, 2**52, size=n, dtype=np.uint64) >> shift  # every leading-zero count
    m = np.maximum(m, 1)
    assert np.array_equal(emul(m, x), ieee(m, x))
    p = np.uint64(1) << np.arange(52, dtype=np.uint64)
    xx = np.full(p.size, 3.7)
    assert np.array_equal(emul(p, xx), ieee(p, xx))


def test_ties_and_carries(emul):
    rng = np.random.default_rng(54)
    # ties: U = 3/4 (or 3/8, ...) times an odd significand leaves exactly
    # half an ulp, both below and above the binade change of the product
    sig = (rng.integers(2**52, 2**53, size=4096, dtype=np.uint64) | np.uint64(1))
    x = np.ldexp(sig.astype(np.float64), -52)
    for mm in (3 << 50, 3 << 49, 3 << 40, 5 << 49, 7 << 48):
        m = np.full(sig.size, mm, dtype=np.uint64)
        assert np.array_equal(emul(m, x), ieee(m, x))
    # carries: the largest significands and m, rounding up to the next binade
    x = np.nextafter(np.ldexp(np.ones(64), np.arange(-32, 32)), 0.0)
    m = np.full(x.size, 2**52 - 1, dtype=np.uint64)
    assert np.array_equal(emul(m, x), ieee(m, x))
    # U = 0: +0 for either sign
    z = emul(np.zeros(2, dtype=np.uint64), np.array([2.5, -2.5]))
    assert np.array_equal(z, np.zeros(2, dtype=np.uint64))
