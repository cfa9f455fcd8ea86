"""Pins for the oracle's Philox4x32-10 uniform source.

The oracle's Philox is checked against an independent implementation that
is present on this machine: PyTorch's host Philox engine
(ATen/core/PhiloxRNGEngine.h), compiled into a tiny checker program.  The
word-stream layout (counter = (g_lo, g_hi, 0, attempt), key = (seed_lo,
seed_hi), words r0|r1<<32 then r2|r3<<32 per block) is then checked against
the raw blocks.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _aten_checker(tmp_path_factory):
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    hdr = os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")
    if not os.path.exists(hdr) or shutil.which("g++") is None:
        pytest.skip("ATen Philox header or g++ not available")
    exe = str(tmp_path_factory.mktemp("aten") / "philox_aten_check")
    r = subprocess.run(["g++", "-std=c++17", "-O1", f"-I{inc}",
                        os.path.join(HERE, "philox_aten_check.cpp"), "-o", exe],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("ATen Philox checker does not compile here: " + r.stderr[-300:])
    return exe


@pytest.fixture(scope="module")
def aten(tmp_path_factory):
    return _aten_checker(tmp_path_factory)


def _cases():
    rng = np.random.default_rng(1403_6870)
    cases = []
    # Carry cases around the 2^32 boundary of the counter's low word, the
    # seed of the workloads, zero key, all-ones key, attempts > 0.
    for g in (0, 1, 2**32 - 1, 2**32, 2**32 + 1, 2**32 - 2**19, 2**64 - 1, 2**63):
        for seed in (0, 0x0123456789ABCDEF, 2**64 - 1):
            for a in (0, 1, 7, 2**31 + 5):
                cases.append((seed, g, a))
    for _ in range(2000):
        cases.append((int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2)),
                      int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2)),
                      int(rng.integers(0, 64))))
    return cases


def test_philox_matches_aten_engine(orc, aten):
    cases = _cases()
    inp = "\n".join(f"{s} {g} {a} 0" for s, g, a in cases) + "\n"
    out = subprocess.run([aten], input=inp, capture_output=True, text=True, check=True).stdout
    ref = [tuple(int(v) for v in line.split()) for line in out.strip().splitlines()]
    assert len(ref) == len(cases)
    for (s, g, a), r in zip(cases, ref):
        mine = orc.philox([g & 0xFFFFFFFF, g >> 32, 0, a], [s & 0xFFFFFFFF, s >> 32])
        assert mine == r, (s, g, a)


def test_word_stream_layout(orc):
    seed, g = 0x0123456789ABCDEF, 2**32 + 12345
    words = orc.philox_words(seed, g, 6)
    for a in range(3):
        r = orc.philox([g & 0xFFFFFFFF, g >> 32, 0, a], [seed & 0xFFFFFFFF, seed >> 32])
        assert words[2 * a] == r[0] | (r[1] << 32)
        assert words[2 * a + 1] == r[2] | (r[3] << 32)


def test_philox_bits_uniform(orc):
    """Each of the 64 bits of the first word is a fair coin (5 SE)."""
    seed = 0x0123456789ABCDEF
    n = 4096
    w = np.array([orc.philox_words(seed, g, 1)[0] for g in range(n)], dtype=np.uint64)
    for b in range(64):
        ones = int(((w >> np.uint64(b)) & np.uint64(1)).sum())
        assert abs(ones - n / 2) < 5 * np.sqrt(n / 4), b


def _aten_blocks(aten, rows):
    """ATen's blocks for (seed, g, attempt, domain) rows."""
    inp = "\n".join(f"{s} {g} {a} {d}" for s, g, a, d in rows) + "\n"
    out = subprocess.run([aten], input=inp, capture_output=True, text=True, check=True).stdout
    return [tuple(int(v) for v in line.split()) for line in out.strip().splitlines()]


@pytest.mark.parametrize("dtype", [0, 1])
def test_packed_word_stream_matches_aten(orc, aten, dtype):
    """Packed keying: the first word of counter g is taken from the block of
    g >> 1 (FP64: half g & 1) or g >> 2 (FP32: 32-bit output g & 3, its low
    9 bits kept and its top 23 bits moved to bits 41-63); later words are
    counter g's private stream, blocks (g_lo, g_hi, 1, a).  Raw blocks come
    from the independent ATen engine."""
    rng = np.random.default_rng(20260 + dtype)
    gs = [0, 1, 2, 3, 4, 5, 2**32 - 1, 2**32, 2**32 + 2, 2**64 - 1, 2**64 - 4]
    gs += [int(v) for v in rng.integers(0, 2**63, size=200)]
    seeds = [0x0123456789ABCDEF, 0, 2**64 - 1]
    for seed in seeds:
        shift = 1 if dtype == 1 else 2
        rows = []
        for g in gs:
            rows.append((seed, g >> shift, 0, 0))
            rows += [(seed, g, a, 1) for a in range(2)]
        ref = _aten_blocks(aten, rows)
        for k, g in enumerate(gs):
            fast, p0, p1 = ref[3 * k], ref[3 * k + 1], ref[3 * k + 2]
            words = orc.packed_words(seed, g, dtype, 5)
            if dtype == 1:
                h = g & 1
                assert words[0] == fast[2 * h] | (fast[2 * h + 1] << 32), (seed, g)
            else:
                lane = fast[g & 3]
                assert words[0] == (lane & 0x1FF) | ((lane >> 9) << 41), (seed, g)
            assert words[1:] == [p0[0] | (p0[1] << 32), p0[2] | (p0[3] << 32),
                                 p1[0] | (p1[1] << 32), p1[2] | (p1[3] << 32)], (seed, g)
