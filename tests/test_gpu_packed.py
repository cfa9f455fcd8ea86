"""GPU parity of packed keying (zig_generate with ZIG_KEY_PACKED) against
the oracle's packed word source, element by element (rule in
tests/parity.py): all four dist/dtype pairs, ragged sizes spanning many
tiles, counters whose first vector is and is not a multiple of the block
width, misaligned output pointers, tiny sizes, the 2^32 carry of the block
counters and of the private counters, the top of the counter range, split
invariance, and ZIG_KEY_INDEX through the same entry point matching
zig_exponential / zig_normal bit for bit.  Packed and per-index outputs
are never compared with each other.
"""
import numpy as np
import pytest

import workloads as W
from parity import check

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PACKED = 1


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


def gen(z, dist, dtype, n, seed, offset, pad=0, keying=PACKED):
    buf = torch.full((n + pad + 8,), float("nan"), dtype=_tdt(dtype), device="cuda")
    out = buf[pad:pad + n]
    z.zig_generate(dist, keying, out, n, seed, offset)
    return out, buf


def ref(orc, dist, dtype, seed, offset, n):
    v, errs, words, margin = orc.fill(dist, dtype, seed, offset, n, want_words=True,
                                      want_margin=True, keying=PACKED)
    return v, words, margin


@pytest.mark.parametrize("dist", [W.EXP, W.NORMAL])
@pytest.mark.parametrize("dtype", [W.F64, W.F32])
@pytest.mark.parametrize("offset,pad", [(0, 0), (777, 1), (2**32 - 2**19 - 2, 0), (6, 3),
                                        (2**34 - 9, 2)])
def test_packed_ragged_against_oracle(zig, orc, dist, dtype, offset, pad):
    n = (1 << 20) + 12345
    seed = 0xDEADBEEFCAFEF00D
    out, buf = gen(zig, dist, dtype, n, seed, offset, pad=pad)
    assert zig.zig_status_poll() == zig.ZIG_OK
    v, words, margin = ref(orc, dist, dtype, seed, offset, n)
    rep = check(out.cpu().numpy(), v, words, margin)
    assert rep["fringe"] > 5000
    b = buf.cpu().numpy()
    assert np.all(np.isnan(b[:pad])) and np.all(np.isnan(b[pad + n:]))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 9, 31, 33, 257, 4097, 65537])
def test_packed_small_sizes(zig, orc, n):
    for dist in (W.EXP, W.NORMAL):
        for dtype in (W.F64, W.F32):
            for pad in (0, 1, 2):
                for off in (4 * n, 4 * n + 1, 4 * n + 3):
                    out, buf = gen(zig, dist, dtype, n, W.SEED, off, pad=pad)
                    v, words, margin = ref(orc, dist, dtype, W.SEED, off, n)
                    check(out.cpu().numpy(), v, words, margin)
                    b = buf.cpu().numpy()
                    assert np.all(np.isnan(b[:pad])) and np.all(np.isnan(b[pad + n:]))
    assert zig.zig_status_poll() == zig.ZIG_OK


def test_packed_top_of_counter_range(zig, orc):
    n = 5000
    off = 2**64 - n
    for dist in (W.EXP, W.NORMAL):
        for dtype in (W.F64, W.F32):
            out, _ = gen(zig, dist, dtype, n, W.SEED, off)
            v, words, margin = ref(orc, dist, dtype, W.SEED, off, n)
            check(out.cpu().numpy(), v, words, margin)


def test_packed_split_invariance(zig):
    n, a = 1 << 20, 333331  # the second call starts on an odd counter
    for dist in (W.EXP, W.NORMAL):
        for dtype in (W.F64, W.F32):
            whole, _ = gen(zig, dist, dtype, n, 99, 12344)
            part = torch.empty(n, dtype=_tdt(dtype), device="cuda")
            zig.zig_generate(dist, PACKED, part[:a], a, 99, 12344)
            zig.zig_generate(dist, PACKED, part[a:], n - a, 99, 12344 + a)
            it = torch.int32 if dtype == W.F32 else torch.int64
            assert torch.equal(whole.view(it), part.view(it))


def test_index_keying_equals_the_plain_calls(zig):
    n = 300007
    for dist in (W.EXP, W.NORMAL):
        for dtype in (W.F64, W.F32):
            a, _ = gen(zig, dist, dtype, n, 5, 1234, keying=0)
            b = torch.empty(n, dtype=_tdt(dtype), device="cuda")
            (zig.zig_exponential if dist == W.EXP else zig.zig_normal)(b, n, 5, 1234)
            it = torch.int32 if dtype == W.F32 else torch.int64
            assert torch.equal(a.view(it), b.view(it))


def test_generate_rejects_unknown_keying(zig):
    b = torch.empty(16, dtype=torch.float64, device="cuda")
    with pytest.raises(zig.ZigError):
        zig.zig_generate(W.NORMAL, 2, b, 16, 1, 0)
    with pytest.raises(zig.ZigError):
        zig.zig_generate(7, 0, b, 16, 1, 0)


def _zero_fringe():
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden",
                           "packed_f32_zero_fringe.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("dist", [W.EXP, W.NORMAL])
@pytest.mark.parametrize("shift", [1000, 1001, 4096])
def test_packed_f32_fringe_draw_with_zero_u(zig, orc, dist, shift):
    """A fringe draw whose U is zero: its first overhang attempt starts at
    u_x = 0 (the box's right edge X_j), and for the normal the sign comes
    from a first word whose U bits are all zero (counters from
    tests/golden/packed_f32_zero_fringe.json; the normal's has its sign bit
    set).  Offsets put it in the vector body at both block alignments."""
    fx = _zero_fringe()
    g = fx["exp" if dist == W.EXP else "normal"]
    n = 8192
    off = g - shift
    out, _ = gen(zig, dist, W.F32, n, fx["seed"], off)
    v, words, margin = ref(orc, dist, W.F32, fx["seed"], off, n)
    got = out.cpu().numpy()
    check(got, v, words, margin)
    assert words[shift] > 1  # the draw left step 2
    assert zig.zig_status_poll() == zig.ZIG_OK


@pytest.mark.parametrize("dist,dtype", [(W.NORMAL, W.F64), (W.EXP, W.F64), (W.NORMAL, W.F32),
                                        (W.EXP, W.F32)])
def test_packed_2p28_full_size_sampled(zig, orc, dist, dtype):
    """The launch the bench times for packed keying (2^28 outputs in one
    call, counters from 5 * 2^28): 2^20 sampled positions against the
    oracle one by one, about 12 K of them fringe draws."""
    n = 1 << 28
    offset = 5 * n
    out, _ = gen(zig, dist, dtype, n, W.SEED, offset)
    assert zig.zig_status_poll() == zig.ZIG_OK
    idx = W.sample_positions(n, 1 << 20)
    got = out[torch.from_numpy(idx.astype(np.int64)).cuda()].cpu().numpy()
    del out
    torch.cuda.empty_cache()
    v, errs, words, margin = orc.fill(dist, dtype, W.SEED, offset, 0, idx=idx, want_words=True,
                                      want_margin=True, keying=PACKED)
    assert errs == 0
    rep = check(got, v, words, margin)
    assert rep["fringe"] > 5000
