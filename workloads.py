"""Seeded synthetic workloads: the only inputs shared by the CUDA path's
tests/bench and the CPU oracle.  Holds none of the sampler's arithmetic.

The generator's inputs are (seed, counter offset, n, distribution, dtype);
the batched-serving mix is a list of such requests with parameters.  The
paper's own workload is "generate and aggregate 10^9 PRNs" (Sec. 4,
Timings); no dataset is involved.
"""
from __future__ import annotations

import numpy as np

SEED = 0x0123456789ABCDEF  # Philox key of the single-request workloads
EXP, NORMAL = 0, 1
F32, F64 = 0, 1

MASK64 = (1 << 64) - 1

# Single-request workloads (name -> parameters).
WORKLOADS = {
    # standard exponential, FP64, small enough for the oracle in full
    "exp_f64_2p20": dict(dist=EXP, dtype=F64, n=1 << 20, offset=0),
    # the same, with the counter crossing the 2^32 carry into the high word
    "exp_f64_2p20_carry": dict(dist=EXP, dtype=F64, n=1 << 20, offset=(1 << 32) - (1 << 19)),
    # standard normal, FP64, 2 GiB materialised
    "normal_f64_2p28": dict(dist=NORMAL, dtype=F64, n=1 << 28, offset=0),
    # precision variant: FP32 arithmetic and outputs, 4 GiB each
    "exp_f32_2p30": dict(dist=EXP, dtype=F32, n=1 << 30, offset=0),
    "normal_f32_2p30": dict(dist=NORMAL, dtype=F32, n=1 << 30, offset=0),
    # fused in-register reduction: 2^34 FP32 normals never stored
    "normal_f32_fused_2p34": dict(dist=NORMAL, dtype=F32, n=1 << 34, offset=0),
}


def splitmix64(x: int) -> int:
    """SplitMix64 output function (Steele, Lea, Flood 2014), used only to
    derive per-request seeds and offsets of the batched mix."""
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def batch_requests(count: int = 4096, rng_seed: int = 20140327, max_size: float = 1e7,
                   min_size: float = 1e2) -> list[dict]:
    """Batched serving mix: sizes log-uniform in [1e2, 1e7], half exponential
    (rate log-uniform in [0.1, 10]) and half normal (mean uniform in [-5, 5],
    sd log-uniform in [0.01, 100]), dtype FP32 or FP64 at random, each
    request with its own Philox seed and 40-bit counter offset."""
    rng = np.random.default_rng(rng_seed)
    lo, hi = np.log10(min_size), np.log10(max_size)
    reqs = []
    for r in range(count):
        size = int(np.floor(10.0 ** rng.uniform(lo, hi)))
        dist = int(rng.integers(0, 2))
        rate = float(10.0 ** rng.uniform(-1, 1))
        mean = float(rng.uniform(-5, 5))
        sd = float(10.0 ** rng.uniform(-2, 2))
        dtype = int(rng.integers(0, 2))
        reqs.append(dict(
            n=size, dist=dist, dtype=dtype,
            p0=rate if dist == EXP else mean,
            p1=0.0 if dist == EXP else sd,
            seed=splitmix64(r),
            offset=splitmix64(r + (1 << 32)) & ((1 << 40) - 1),
        ))
    return reqs


def sample_positions(n: int, m: int, rng_seed: int = 1403) -> np.ndarray:
    """Up to m distinct positions in [0, n): both ends, a run at the start
    and end of every 2^20 stride, and uniform picks -- for checking large
    outputs against the oracle one sample at a time."""
    rng = np.random.default_rng(rng_seed)
    pos = {0, n - 1}
    for s in range(0, n, max(1, n // 64)):
        pos.update(range(s, min(n, s + 64)))
    pos.update(range(max(0, n - 256), n))
    k = max(0, m - len(pos))
    if k:
        pos.update(int(v) for v in rng.integers(0, n, size=k))
    out = np.array(sorted(p for p in pos if 0 <= p < n), dtype=np.uint64)
    return out[:m] if out.size > m else out
