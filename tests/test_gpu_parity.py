"""GPU parity: the CUDA path (called through the C ABI) against the CPU oracle.

Element-by-element on the same seeded counters (rule in tests/parity.py):
sizes the oracle finishes in seconds that span many tiles and a ragged
tail, misaligned output pointers, tiny sizes, the 2^32 and 2^64 counter
boundaries, split invariance, the loop-limit error path, and the full
workloads (2^28 FP64 normals, 2^30 FP32 variates) on sampled positions
plus distribution tests of the whole device output.
"""
import math

import numpy as np
import pytest

import workloads as W
from parity import check

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def zig():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_1403_6870_gb300 import build

    build.build()
    import paper_1403_6870_gb300 as z

    z.zig_build_tables()
    return z


def _tdt(dtype):
    return torch.float64 if dtype == W.F64 else torch.float32


def gpu_gen(z, dist, dtype, n, seed, offset, pad=0):
    """Generate into a view starting `pad` elements into a fresh buffer."""
    buf = torch.full((n + pad + 8,), float("nan"), dtype=_tdt(dtype), device="cuda")
    out = buf[pad:pad + n]
    fn = z.zig_exponential if dist == W.EXP else z.zig_normal
    fn(out, n, seed, offset)
    return out, buf


def oracle_ref(orc, dist, dtype, seed, offset, n=None, idx=None):
    v, errs, words, margin = orc.fill(dist, dtype, seed, offset, n or 0, idx=idx,
                                      want_words=True, want_margin=True)
    return v, words, margin


@pytest.mark.parametrize("name", ["exp_f64_2p20", "exp_f64_2p20_carry"])
def test_exponential_f64_full(zig, orc, name):
    c = W.WORKLOADS[name]
    out, _ = gpu_gen(zig, c["dist"], c["dtype"], c["n"], W.SEED, c["offset"])
    assert zig.zig_status_poll() == zig.ZIG_OK
    ref, words, margin = oracle_ref(orc, c["dist"], c["dtype"], W.SEED, c["offset"], c["n"])
    rep = check(out.cpu().numpy(), ref, words, margin)
    assert rep["fringe"] > 10000


@pytest.mark.parametrize("dist", [W.EXP, W.NORMAL])
@pytest.mark.parametrize("dtype", [W.F64, W.F32])
@pytest.mark.parametrize("pad", [0, 1, 3])
def test_ragged_and_misaligned(zig, orc, dist, dtype, pad):
    n = (1 << 20) + 12345
    seed, off = 0xDEADBEEFCAFEF00D, 777
    out, buf = gpu_gen(zig, dist, dtype, n, seed, off, pad=pad)
    assert zig.zig_status_poll() == zig.ZIG_OK
    ref, words, margin = oracle_ref(orc, dist, dtype, seed, off, n)
    check(out.cpu().numpy(), ref, words, margin)
    # nothing outside [pad, pad + n) was written
    b = buf.cpu().numpy()
    assert np.all(np.isnan(b[:pad])) and np.all(np.isnan(b[pad + n:]))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 31, 33, 255, 256, 257, 1023, 4097, 65537])
def test_small_sizes(zig, orc, n):
    for dist in (W.EXP, W.NORMAL):
        for dtype in (W.F64, W.F32):
            for pad in (0, 1, 2):
                out, buf = gpu_gen(zig, dist, dtype, n, W.SEED, 5 * n, pad=pad)
                ref, words, margin = oracle_ref(orc, dist, dtype, W.SEED, 5 * n, n)
                check(out.cpu().numpy(), ref, words, margin)
                b = buf.cpu().numpy()
                assert np.all(np.isnan(b[:pad])) and np.all(np.isnan(b[pad + n:]))
    assert zig.zig_status_poll() == zig.ZIG_OK


def test_zero_length_is_noop(zig):
    buf = torch.full((4,), 7.0, dtype=torch.float64, device="cuda")
    zig.zig_normal(buf, 0, 1, 0)
    assert torch.all(buf == 7.0)


def test_counter_at_top_of_range(zig, orc):
    n = 3000
    off = 2**64 - n  # last counter is 2^64 - 1
    for dist in (W.EXP, W.NORMAL):
        out, _ = gpu_gen(zig, dist, W.F64, n, W.SEED, off)
        ref, words, margin = oracle_ref(orc, dist, W.F64, W.SEED, off, n)
        check(out.cpu().numpy(), ref, words, margin)
    with pytest.raises(zig.ZigError):
        gpu_gen(zig, W.EXP, W.F64, n + 1, W.SEED, off)


def test_split_invariance(zig):
    n, a = 1 << 20, 333331
    for dist in (W.EXP, W.NORMAL):
        for dtype in (W.F64, W.F32):
            whole, _ = gpu_gen(zig, dist, dtype, n, 99, 12345)
            part = torch.empty(n, dtype=_tdt(dtype), device="cuda")
            fn = zig.zig_exponential if dist == W.EXP else zig.zig_normal
            fn(part[:a], a, 99, 12345)
            fn(part[a:], n - a, 99, 12345 + a)
            assert torch.equal(whole.view(torch.int32 if dtype == W.F32 else torch.int64),
                               part.view(torch.int32 if dtype == W.F32 else torch.int64))


def test_loop_limit_reports_and_matches_oracle(zig, orc):
    n = 1 << 20
    try:
        zig.zig_set_fringe_limits(1, 16)
        orc.set_limits(1, 16)
        out, _ = gpu_gen(zig, W.EXP, W.F64, n, W.SEED, 0)
        assert zig.zig_status_poll() == zig.ZIG_E_LOOP_LIMIT
        assert zig.zig_status_poll() == zig.ZIG_OK  # poll clears the word
        v, errs, words, margin = orc.fill(W.EXP, W.F64, W.SEED, 0, n, want_words=True,
                                          want_margin=True)
        assert errs > 0
        got = out.cpu().numpy()
        assert int(np.isnan(got).sum()) == errs
        check(got, v, words, margin)
    finally:
        zig.zig_set_fringe_limits(64, 16)
        orc.set_limits(64, 16)


def _gpu_distribution_stats(x: "torch.Tensor", dist: int):
    """KS distance, 1024-bin equiprobable chi-square and raw moments of a
    device array, all computed on the device in FP64."""
    from scipy import special

    n = x.numel()
    xd = x.double()
    q = np.arange(1, 1024) / 1024
    edges = -np.log1p(-q) if dist == W.EXP else special.ndtri(q)
    e = torch.tensor(edges, dtype=torch.float64, device=x.device)
    cnt = torch.bincount(torch.bucketize(xd, e, right=True), minlength=1024).double()
    chi2 = float(((cnt - n / 1024) ** 2 / (n / 1024)).sum())
    s, _ = torch.sort(xd)
    F = (1 - torch.exp(-s)) if dist == W.EXP else torch.special.ndtr(s)
    i = torch.arange(1, n + 1, device=x.device, dtype=torch.float64)
    D = float(torch.maximum(i / n - F, F - (i - 1) / n).max())
    del s, F, i
    moms = [float((xd ** k).mean()) for k in (1, 2, 3, 4)]
    return D, chi2, moms


def test_normal_f64_2p28_full_size(zig, orc):
    c = W.WORKLOADS["normal_f64_2p28"]
    n = c["n"]
    out, _ = gpu_gen(zig, c["dist"], c["dtype"], n, W.SEED, c["offset"])
    assert zig.zig_status_poll() == zig.ZIG_OK
    idx = W.sample_positions(n, 1 << 20)
    got = out[torch.from_numpy(idx.astype(np.int64)).cuda()].cpu().numpy()
    ref, words, margin = oracle_ref(orc, c["dist"], c["dtype"], W.SEED, c["offset"], idx=idx)
    check(got, ref, words, margin)
    D, chi2, moms = _gpu_distribution_stats(out, W.NORMAL)
    assert D < 1.63 / math.sqrt(n) * 1.5  # KS 1% critical value, with slack
    assert abs(chi2 - 1023) < 6 * math.sqrt(2 * 1023)
    for m, mu, var in zip(moms, (0, 1, 0, 3), (1, 2, 15, 96)):
        assert abs(m - mu) < 5 * math.sqrt(var / n)


@pytest.mark.parametrize("name", ["exp_f32_2p30", "normal_f32_2p30"])
def test_f32_2p30_full_size(zig, orc, name):
    c = W.WORKLOADS[name]
    n = c["n"]
    out, _ = gpu_gen(zig, c["dist"], c["dtype"], n, W.SEED, c["offset"])
    assert zig.zig_status_poll() == zig.ZIG_OK
    idx = W.sample_positions(n, 1 << 20)
    tidx = torch.from_numpy(idx.astype(np.int64)).cuda()
    got = out[tidx].cpu().numpy()
    ref, words, margin = oracle_ref(orc, c["dist"], c["dtype"], W.SEED, c["offset"], idx=idx)
    check(got, ref, words, margin)
    # against FP64 on the same counters: |x32 - x64| and decision flips
    r64, w64, _ = oracle_ref(orc, c["dist"], W.F64, W.SEED, c["offset"], idx=idx)
    fast = (words == 1) & (w64 == 1)
    d = np.abs(got[fast].astype(np.float64) - r64[fast])
    assert d.max() <= 7.6 * 2.0**-23 + 2.0**-21
    # decisions that flip between FP32 and FP64 (different word counts):
    # measured 4.2e-8 of the 2^30 counters, so at most one in these 2^20
    assert float(np.mean(words != w64)) < 1e-6
    # the whole 2^30 outputs: KS, 1024-bin chi-square and four moments
    D, chi2, moms = _gpu_distribution_stats(out, c["dist"])
    del out
    torch.cuda.empty_cache()
    assert D < 1.63 / math.sqrt(n) * 1.5
    assert abs(chi2 - 1023) < 6 * math.sqrt(2 * 1023)
    if c["dist"] == W.EXP:
        want = zip(moms, (1, 2, 6, 24), (1, 20, 684, 40320 - 576))
    else:
        want = zip(moms, (0, 1, 0, 3), (1, 2, 15, 96))
    for m, mu, var in want:
        assert abs(m - mu) < 5 * math.sqrt(var / n)


def test_f32_zeros_are_positive_and_match_oracle(zig, orc):
    # FP32 keeps 23 bits of U, so U = 0 comes up about once in 2^23 draws:
    # every such fast-path value is +0 on the GPU whatever the normal's sign
    # (reading R16), and a zero of step 2 in the oracle (whose sign bit
    # follows the draw's).
    n = 1 << 27
    for dist in (W.NORMAL, W.EXP):
        out, _ = gpu_gen(zig, dist, W.F32, n, W.SEED, 12345)
        bits = out.view(torch.int32)
        zpos = torch.nonzero((bits & 0x7FFFFFFF) == 0).flatten()
        assert zpos.numel() >= 4  # ~16 expected
        assert int((bits[zpos] != 0).sum()) == 0
        idx = zpos.cpu().numpy().astype(np.uint64)
        ref, words, margin = oracle_ref(orc, dist, W.F32, W.SEED, 12345, idx=idx)
        assert np.all(ref == 0.0) and np.all(words == 1)  # zeros of step 2 there too
    assert zig.zig_status_poll() == zig.ZIG_OK


def test_status_word_is_taken_once_from_any_stream(zig):
    """zig_status_poll reads and clears the device's status word with one
    atomic exchange ordered on the stream it is given, and synchronises
    only that stream: a loop-limit condition recorded by work on one
    stream is reported by a poll on another stream once that work is
    done, and the next poll finds the word clear."""
    n = 1 << 20
    a, b = torch.cuda.Stream(), torch.cuda.Stream()
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    try:
        zig.zig_set_fringe_limits(1, 16)
        zig.zig_exponential(out, n, W.SEED, 0, stream=a)
        a.synchronize()
        zig.zig_set_fringe_limits(64, 16)
        assert zig.zig_status_poll(b) == zig.ZIG_E_LOOP_LIMIT
        assert zig.zig_status_poll(a) == zig.ZIG_OK
        zig.zig_normal(out, n, W.SEED, n, stream=b)
        assert zig.zig_status_poll(b) == zig.ZIG_OK
    finally:
        zig.zig_set_fringe_limits(64, 16)


def test_concurrent_polls_report_a_condition_once(zig):
    """Two threads poll at the same moment, each on its own stream, after a
    launch recorded a loop-limit condition: exactly one of them reports it
    and the other finds the word clear, every time (each poll reads the
    take of its own exchange)."""
    import threading

    n = 1 << 16
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    gen = torch.cuda.Stream()
    try:
        zig.zig_set_fringe_limits(1, 16)
        for it in range(100):
            zig.zig_exponential(out, n, W.SEED, it * n, stream=gen)
            gen.synchronize()
            got = [None, None]
            start = threading.Barrier(2)

            def poll(k):
                start.wait()
                got[k] = zig.zig_status_poll(streams[k])

            th = [threading.Thread(target=poll, args=(k,)) for k in range(2)]
            for t in th:
                t.start()
            for t in th:
                t.join()
            assert sorted(got) == sorted([zig.ZIG_OK, zig.ZIG_E_LOOP_LIMIT]), (it, got)
    finally:
        zig.zig_set_fringe_limits(64, 16)
        assert zig.zig_status_poll() == zig.ZIG_OK


@pytest.mark.parametrize("dist", [W.EXP, W.NORMAL])
@pytest.mark.parametrize("dtype", [W.F64, W.F32])
def test_tile_and_wave_boundaries(zig, orc, dist, dtype):
    """Sizes at the default shapes' tile boundary (256 threads x 32 outputs
    = 8192 per CTA tile for FP64 V4 R8 and FP32 V8 R4) and at one full wave
    of the persistent grid (152 SMs x 3 CTAs x 8192) plus a ragged rest,
    element by element against the oracle."""
    for n, off in ((8191, 3), (8192, 0), (8193, 2**32 - 4096), (456 * 8192 + 5, 77)):
        out, buf = gpu_gen(zig, dist, dtype, n, W.SEED, off, pad=1)
        got = out.cpu().numpy()
        ref, words, margin = oracle_ref(orc, dist, dtype, W.SEED, off, n=n)
        check(got, ref, words, margin)
        tail = buf[1 + n:].cpu().numpy()
        assert np.all(np.isnan(tail))  # nothing written past the end
    assert zig.zig_status_poll() == zig.ZIG_OK
