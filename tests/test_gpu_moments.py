"""GPU parity of the fused generate-and-reduce path (zig_moments).

The variates are those of zig_normal/zig_exponential on the same counters
(themselves checked element by element), so the oracle's plain definitions
apply: the histogram must equal the oracle's exactly; each power sum must
be within the rounding bound of its accumulation scheme (FP32 partials of
at most m terms, m = 32 at the default FP32 shape and 64 with packed
keying, then summed in double-FP32 by an error-free two-sum, whose error is
far below the bound):
|S_gpu - S| <= (m + 4) 2^-24 sum |x|^k (FP32) or 1e-12 sum |x|^k (FP64);
FP32 sums are also held to the error actually achieved, within one unit of
2^-24 sum |x|^k (measured: at most 0.17).
Packed keying (zig_moments_keyed) is checked against the oracle's packed
word source the same way.
At the full 2^34 size: moments within 5 standard errors of the closed
forms and the histogram against the exact bin probabilities.
"""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def zig():
    assert torch.cuda.is_available()
    from paper_1403_6870_gb300 import build

    build.build()
    import paper_1403_6870_gb300 as z

    z.zig_build_tables()
    return z


def _run(z, dist, dtype, n, seed, offset, keying=0):
    sums = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    hist = torch.full((4098,), -1, dtype=torch.int64, device="cuda")
    ws = torch.empty(z.zig_moments_workspace_bytes(dist, dtype), dtype=torch.uint8, device="cuda")
    if keying:
        z.zig_moments_keyed(dist, dtype, keying, n, seed, offset, sums, hist, ws)
    else:
        z.zig_moments(dist, dtype, n, seed, offset, sums, hist, ws)
    return sums.cpu().numpy(), hist.cpu().numpy().astype(np.uint64)


def _tol(dtype, keying, abss):
    m = 64 if keying else 32  # FP32 terms per partial sum
    return ((m + 4) * 2.0**-24 if dtype == 0 else 1e-12) * abss + 1e-300


@pytest.mark.parametrize("keying", [0, 1])
@pytest.mark.parametrize("dist,dtype", [(1, 0), (0, 0), (1, 1), (0, 1)])
def test_moments_match_oracle(zig, orc, dist, dtype, keying):
    n, seed, off = (1 << 22) + 333, 0x9E3779B97F4A7C15, 4321
    for rep in range(2):  # twice: the workspace ticket must reset
        sums, hist = _run(zig, dist, dtype, n, seed, off, keying)
        assert zig.zig_status_poll() == zig.ZIG_OK
        ref, abss, rhist, errs = orc.moments(dist, dtype, seed, off, n, keying=keying)
        assert errs == 0
        assert np.array_equal(hist, rhist)
        assert int(hist.sum()) == n
        tol = _tol(dtype, keying, abss)
        assert np.all(np.abs(sums - ref) <= tol), (sums, ref, tol)
        if dtype == 0:
            # the achieved error (fixed inputs, so the sums repeat bit for
            # bit) is far inside the worst case: measured on GB300 at most
            # 0.17 units of 2^-24 sum |x|^k at 2^22 and 2^26 values; one
            # unit flags a systematic accumulation error
            assert np.all(np.abs(sums - ref) <= 2.0**-24 * abss), (sums, ref, abss)


@pytest.mark.parametrize("keying", [0, 1])
def test_moments_across_the_counter_carry(zig, orc, keying):
    """Counters crossing 2^32 (the high counter word changes mid-tile):
    histogram exact, sums within the bound, FP32 normals."""
    n, seed, off = (1 << 20) + 7, 0x0123456789ABCDEF, 2**32 - 5001
    sums, hist = _run(zig, 1, 0, n, seed, off, keying)
    assert zig.zig_status_poll() == zig.ZIG_OK
    ref, abss, rhist, errs = orc.moments(1, 0, seed, off, n, keying=keying)
    assert errs == 0 and np.array_equal(hist, rhist)
    assert np.all(np.abs(sums - ref) <= _tol(0, keying, abss)), (sums, ref)


def test_moments_small_and_edge_sizes(zig, orc):
    for n in (1, 7, 1000, 3584 * 7 + 5):
        sums, hist = _run(zig, 1, 0, n, W.SEED, 17)
        ref, abss, rhist, _ = orc.moments(1, 0, W.SEED, 17, n)
        assert np.array_equal(hist, rhist)
        assert np.all(np.abs(sums - ref) <= _tol(0, 0, abss))


def test_workspace_too_small(zig):
    sums = torch.zeros(4, dtype=torch.float64, device="cuda")
    hist = torch.zeros(4098, dtype=torch.int64, device="cuda")
    ws = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(zig.ZigError) as e:
        zig.zig_moments(1, 0, 1 << 24, 1, 0, sums, hist, ws)
    assert e.value.status == zig.ZIG_E_NOMEM


@pytest.mark.parametrize("keying", [0, 1])
def test_fused_2p34_normal_f32(zig, keying):
    # the bench's fused launches (per-index and packed keying): 2^34 values,
    # their moments and histogram against the normal law
    c = W.WORKLOADS["normal_f32_fused_2p34"]
    n = c["n"]
    sums, hist = _run(zig, c["dist"], c["dtype"], n, W.SEED, c["offset"], keying=keying)
    assert zig.zig_status_poll() == zig.ZIG_OK
    assert int(hist.sum()) == n
    m = sums / n
    for k, (mu, var) in enumerate(zip((0, 1, 0, 3), (1, 2, 15, 96))):
        assert abs(m[k] - mu) < 5 * math.sqrt(var / n), (k, m[k])
    from scipy import special

    edges = (np.arange(4097) - 2048) / 256.0
    p = np.diff(special.ndtr(edges))
    p = np.concatenate([p, [special.ndtr(-8.0), special.ndtr(-8.0)]])
    e = n * p
    ok = e > 50
    chi2 = float(((hist[ok].astype(np.float64) - e[ok]) ** 2 / e[ok]).sum())
    df = int(ok.sum()) - 1
    assert abs(chi2 - df) < 6 * math.sqrt(2 * df), (chi2, df)
