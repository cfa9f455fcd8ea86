"""GPU parity of the i_max = 1024 tables (zig_generate with index_bits 10,
Appendix D item 1) against the oracle run on its own 10-bit tables,
element by element (rule in tests/parity.py): per-index keying for all
four dist/dtype pairs and packed keying for FP64, ragged sizes spanning
many tiles, misaligned output pointers, the 2^32 counter carry, tiny sizes,
and the rejected combination (packed FP32 has no room for 10 index bits).
"""
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


def _gen(z, dist, dtype, keying, n, seed, offset, pad=0):
    buf = torch.full((n + pad + 8,), float("nan"), device="cuda",
                     dtype=torch.float64 if dtype == W.F64 else torch.float32)
    out = buf[pad:pad + n]
    z.zig_generate(dist, keying, out, n, seed, offset, index_bits=10)
    return out, buf


def _ref(orc, dist, dtype, keying, seed, offset, n):
    te, tn = orc.tables(0, 10, 52, 54), orc.tables(1, 10, 52, 54)
    v, errs, words, margin = orc.fill(dist, dtype, seed, offset, n, want_words=True,
                                      want_margin=True, te=te, tn=tn, keying=keying)
    return v, words, margin


CASES = [(W.EXP, W.F64, 0), (W.NORMAL, W.F64, 0), (W.EXP, W.F32, 0), (W.NORMAL, W.F32, 0),
         (W.EXP, W.F64, 1), (W.NORMAL, W.F64, 1)]


@pytest.mark.parametrize("dist,dtype,keying", CASES)
@pytest.mark.parametrize("offset,pad", [(0, 0), (777, 1), (2**32 - 2**19 - 3, 3)])
def test_ten_bit_against_oracle(zig, orc, dist, dtype, keying, offset, pad):
    n = (1 << 21) + 12345
    seed = 0xDEADBEEFCAFEF00D
    out, buf = _gen(zig, dist, dtype, keying, n, seed, offset, pad)
    assert zig.zig_status_poll() == zig.ZIG_OK
    v, words, margin = _ref(orc, dist, dtype, keying, seed, offset, n)
    rep = check(out.cpu().numpy(), v, words, margin)
    assert rep["fringe"] > 2000
    b = buf.cpu().numpy()
    assert np.all(np.isnan(b[:pad])) and np.all(np.isnan(b[pad + n:]))


@pytest.mark.parametrize("n", [1, 3, 7, 33, 257, 4097])
def test_ten_bit_small_sizes(zig, orc, n):
    for dist, dtype, keying in CASES:
        for pad in (0, 1):
            out, buf = _gen(zig, dist, dtype, keying, n, W.SEED, 3 * n + 1, pad)
            v, words, margin = _ref(orc, dist, dtype, keying, W.SEED, 3 * n + 1, n)
            check(out.cpu().numpy(), v, words, margin)
    assert zig.zig_status_poll() == zig.ZIG_OK


def test_ten_bit_packed_fp32_is_rejected(zig):
    b = torch.empty(64, dtype=torch.float32, device="cuda")
    with pytest.raises(zig.ZigError):
        zig.zig_generate(W.NORMAL, 1, b, 64, 1, 0, index_bits=10)
    with pytest.raises(zig.ZigError):
        zig.zig_generate(W.NORMAL, 0, b, 64, 1, 0, index_bits=9)


@pytest.mark.parametrize("dist,keying", [(W.NORMAL, 0), (W.EXP, 0), (W.NORMAL, 1), (W.EXP, 1)])
def test_ten_bit_2p28_full_size_sampled(zig, orc, dist, keying):
    """The launch the bench times for the 1024-slot tables (2^28 FP64
    outputs in one call, counters from 5 * 2^28): 2^20 sampled positions
    against the oracle one by one, a few thousand of them fringe draws."""
    n = 1 << 28
    offset = 5 * n
    out, _ = _gen(zig, dist, W.F64, keying, n, W.SEED, offset)
    assert zig.zig_status_poll() == zig.ZIG_OK
    idx = W.sample_positions(n, 1 << 20)
    got = out[torch.from_numpy(idx.astype(np.int64)).cuda()].cpu().numpy()
    del out
    torch.cuda.empty_cache()
    te, tn = orc.tables(0, 10, 52, 54), orc.tables(1, 10, 52, 54)
    v, errs, words, margin = orc.fill(dist, W.F64, W.SEED, offset, 0, idx=idx, want_words=True,
                                      want_margin=True, te=te, tn=tn, keying=keying)
    assert errs == 0
    rep = check(got, v, words, margin)
    assert rep["fringe"] > 1000
