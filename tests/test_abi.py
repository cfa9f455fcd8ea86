"""CPU-side checks of the C ABI (no kernel launches).

- libzig.so loads and exports every function declared in include/zig.h;
- the library's host tables (built independently of the oracle) agree with
  the oracle's: L_max equal, every binary64/binary32 entry and the alias
  table identical;
- argument checks that return before touching the device.
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def zig():
    from paper_1403_6870_gb300 import build

    build.build()
    import paper_1403_6870_gb300 as z

    return z


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(zig_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(zig):
    lib = ctypes.CDLL(zig.LIB_PATH)
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            names += _declared(h)
    assert "zig_normal" in names and "zig_build_tables" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_covers_all_codes(zig):
    seen = set()
    for s in range(10):
        msg = zig.zig_strerror(s)
        assert msg and msg != "unknown status"
        seen.add(msg)
    assert len(seen) == 10
    assert zig.zig_strerror(99) == "unknown status"


@pytest.mark.parametrize("dist", [0, 1])
def test_library_tables_equal_oracle_tables(zig, orc, dist):
    t = zig.zig_export_tables(dist)
    r = orc.tables(dist)
    assert t.L == r.L and t.imax == 256
    L = t.L
    for name in ("X", "f", "dX", "df", "X32", "f32", "dX32", "df32"):
        a = np.ctypeslib.as_array(getattr(t, name))[: L + 1]
        b = np.ctypeslib.as_array(getattr(r, name))[: L + 1]
        assert np.array_equal(a, b), name
    a = np.ctypeslib.as_array(t.A)[: L + 1]
    b = np.ctypeslib.as_array(r.A)[: L + 1]
    assert np.allclose(a, b, rtol=1e-15, atol=0)
    assert (t.eps, t.tau, t.rinv, t.rinv32) == (r.eps, r.tau, r.rinv, r.rinv32)
    assert list(t.T) == list(r.T)[:256]
    assert list(t.alias) == list(r.alias)[:256]


def test_argument_checks(zig):
    call = zig.raw_call
    Z = zig
    # NULL output with n > 0, bad dtype
    assert call("zig_exponential", None, 10, 1, 0, Z.ZIG_F64, None) == Z.ZIG_E_INVAL
    assert call("zig_normal", 0x1000, 10, 1, 0, 7, None) == Z.ZIG_E_INVAL
    # n = 0 is a no-op even with a NULL pointer
    assert call("zig_normal", None, 0, 1, 0, Z.ZIG_F32, None) == Z.ZIG_OK
    # element alignment
    assert call("zig_exponential", 0x1004, 10, 1, 0, Z.ZIG_F64, None) == Z.ZIG_E_ALIGN
    assert call("zig_exponential", 0x1002, 10, 1, 0, Z.ZIG_F32, None) == Z.ZIG_E_ALIGN
    # counter range: offset + n may reach 2^64 but not pass it
    assert call("zig_normal", 0x1000, 2, 1, 2**64 - 1, Z.ZIG_F64, None) == Z.ZIG_E_RANGE
    # fringe limits
    assert call("zig_set_fringe_limits", 0, 16) == Z.ZIG_E_INVAL
    assert call("zig_set_fringe_limits", 64, -1) == Z.ZIG_E_INVAL
    assert call("zig_set_fringe_limits", 64, 16) == Z.ZIG_OK


def test_no_cpu_fallback(zig):
    """Without a usable device a valid call reports an error, never values."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    st = zig.raw_call("zig_normal", 0x1000, 1 << 10, 1, 0, zig.ZIG_F64, None)
    assert st in (zig.ZIG_E_CUDA, zig.ZIG_E_NOTINIT)


def test_tune_candidates(zig):
    f64 = zig.zig_tune_candidates(1)
    f32 = zig.zig_tune_candidates(0)
    assert len(f64) == 5 and len(f32) == 5
    # the defaults come first; all shapes distinct; outputs per thread and
    # tile fit a warp's ring reservation (32 V R <= 2048)
    assert (f64[0]["V"], f64[0]["R"], f64[0]["min_blocks"]) == (4, 8, 3)
    assert (f32[0]["V"], f32[0]["R"], f32[0]["min_blocks"]) == (8, 4, 3)
    for c in (f64, f32):
        assert len({(e["V"], e["R"], e["min_blocks"]) for e in c}) == len(c)
        assert all(32 * e["V"] * e["R"] <= 2048 for e in c)
    assert zig.zig_tune_candidates(7) == []


def test_tune_cache_roundtrip(zig, tmp_path):
    """JSON Lines cache: valid lines load, invalid ones are skipped, a later
    line replaces an earlier one for the same key, and save writes what was
    loaded (no device involved: the names are not this machine's GPUs)."""
    import json

    src = tmp_path / "in.jsonl"
    c64, c32 = zig.zig_tune_candidates(1), zig.zig_tune_candidates(0)
    a1, a2, b1 = c64[1], c64[2], c32[1]
    lines = [
        {"device": "test-device-A", "sms": 8, "dist": "normal", "dtype": "f64", "V": a1["V"],
         "R": a1["R"], "min_blocks": a1["min_blocks"], "blocks_per_sm": 3, "gsamples_s": 1.5},
        {"device": "test-device-A", "sms": 8, "dist": "normal", "dtype": "f64", "V": a2["V"],
         "R": a2["R"], "min_blocks": a2["min_blocks"], "blocks_per_sm": 2, "gsamples_s": 2.5},
        {"device": "test \"quoted\" B", "sms": 9, "dist": "exp", "dtype": "f32", "V": b1["V"],
         "R": b1["R"], "min_blocks": b1["min_blocks"], "blocks_per_sm": 0, "gsamples_s": 3.0},
        # no such candidate shape, unknown dist, missing field: skipped
        {"device": "test-device-A", "sms": 8, "dist": "exp", "dtype": "f64", "V": 3, "R": 3,
         "min_blocks": 4, "blocks_per_sm": 1},
        {"device": "test-device-A", "sms": 8, "dist": "gamma", "dtype": "f64", "V": 4, "R": 4,
         "min_blocks": 4, "blocks_per_sm": 1},
        {"device": "test-device-A", "sms": 8, "dist": "exp", "dtype": "f64", "V": 4, "R": 4},
    ]
    src.write_text("\n".join(json.dumps(x) for x in lines) + "\nnot json at all\n")
    zig.zig_tune_load(str(src))
    out = tmp_path / "out.jsonl"
    zig.zig_tune_save(str(out))
    got = [json.loads(x) for x in out.read_text().splitlines()]
    mine = {(g["device"], g["sms"], g["dist"], g["dtype"]): g for g in got
            if g["device"].startswith("test")}
    assert set(mine) == {("test-device-A", 8, "normal", "f64"), ('test "quoted" B', 9, "exp", "f32")}
    a = mine[("test-device-A", 8, "normal", "f64")]
    assert (a["V"], a["R"], a["min_blocks"], a["blocks_per_sm"]) == (
        a2["V"], a2["R"], a2["min_blocks"], 2)
    assert a["gsamples_s"] == pytest.approx(2.5)
    with pytest.raises(zig.ZigError):
        zig.zig_tune_load(str(tmp_path / "missing.jsonl"))


@pytest.mark.parametrize("bits", [8, 10])
@pytest.mark.parametrize("dist", [0, 1])
def test_wide_tables_equal_oracle_tables(zig, orc, dist, bits):
    """The library's tables at both index widths (i_max 256 and 1024) equal
    the oracle's entry for entry."""
    t = zig.zig_export_tables_ex(dist, bits)
    r = orc.tables(dist, bits, 52, 64 - bits)
    assert (t.imax, t.index_bits, t.L) == (r.imax, bits, r.L)
    L, M = t.L, t.imax
    for name in ("X", "f", "dX", "df", "X32", "f32", "dX32", "df32"):
        a = np.ctypeslib.as_array(getattr(t, name))[: L + 1]
        b = np.ctypeslib.as_array(getattr(r, name))[: L + 1]
        assert np.array_equal(a, b), name
    assert np.allclose(np.ctypeslib.as_array(t.A)[: L + 1], np.ctypeslib.as_array(r.A)[: L + 1],
                       rtol=1e-15, atol=0)
    assert (t.eps, t.tau, t.rinv, t.rinv32) == (r.eps, r.tau, r.rinv, r.rinv32)
    assert list(t.T)[:M] == list(r.T)[:M]
    assert list(t.alias)[:M] == list(r.alias)[:M]
    with pytest.raises(zig.ZigError):
        zig.zig_export_tables_ex(dist, 9)


def test_generate_argument_checks(zig):
    call = zig.raw_call
    Z = zig
    KI, KP = Z.ZIG_KEY_INDEX, Z.ZIG_KEY_PACKED
    # keying, index width and the packed FP32 word that has no room for 10 index bits
    assert call("zig_generate", 1, 2, 8, 0x1000, 10, 1, 0, Z.ZIG_F64, None) == Z.ZIG_E_INVAL
    assert call("zig_generate", 1, KI, 9, 0x1000, 10, 1, 0, Z.ZIG_F64, None) == Z.ZIG_E_INVAL
    assert call("zig_generate", 1, KP, 10, 0x1000, 10, 1, 0, Z.ZIG_F32, None) == Z.ZIG_E_INVAL
    assert call("zig_generate", 2, KI, 8, 0x1000, 10, 1, 0, Z.ZIG_F64, None) == Z.ZIG_E_INVAL
    # the same size, alignment and range rules as the plain calls
    assert call("zig_generate", 0, KP, 8, None, 0, 1, 0, Z.ZIG_F32, None) == Z.ZIG_OK
    assert call("zig_generate", 0, KP, 8, None, 4, 1, 0, Z.ZIG_F32, None) == Z.ZIG_E_INVAL
    assert call("zig_generate", 0, KI, 10, 0x1004, 4, 1, 0, Z.ZIG_F64, None) == Z.ZIG_E_ALIGN
    assert call("zig_generate", 1, KP, 10, 0x1000, 3, 1, 2**64 - 2, Z.ZIG_F64,
                None) == Z.ZIG_E_RANGE


def test_batch_validate_rules(zig):
    import numpy as np

    Z = zig
    good = dict(out=0x10000, n=1000, seed=1, offset=5, dist=1, dtype=1, p0=-2.0, p1=0.5)

    def status(**change):
        q = dict(good)
        q.update(change)
        return Z.zig_batch_validate(Z.pack_requests([good, q]))

    assert status() == Z.ZIG_OK
    assert status(dist=0, p0=0.3, p1=0.0) == Z.ZIG_OK
    assert status(dist=2) == Z.ZIG_E_INVAL
    assert status(dtype=3) == Z.ZIG_E_INVAL
    assert status(out=0) == Z.ZIG_E_INVAL
    assert status(out=0, n=0) == Z.ZIG_OK          # an empty request needs no buffer
    assert status(out=0x10004) == Z.ZIG_E_ALIGN     # FP64 needs 8-byte alignment
    assert status(out=0x10004, dtype=0) == Z.ZIG_OK  # FP32 needs 4
    assert status(n=2**40) == Z.ZIG_E_RANGE
    assert status(offset=2**64 - 999) == Z.ZIG_E_RANGE
    assert status(offset=2**64 - 1000) == Z.ZIG_OK  # the last counter is 2^64 - 1
    for bad in (0.0, -1.0, float("inf"), float("nan")):
        assert status(dist=0, p0=bad) == Z.ZIG_E_INVAL  # exponential rate
        assert status(p1=bad) == Z.ZIG_E_INVAL          # normal standard deviation
    assert status(p0=float("nan")) == Z.ZIG_E_INVAL     # normal mean
    assert Z.zig_batch_validate(np.zeros(0, dtype=Z.request_dtype())) == Z.ZIG_OK


def test_batch_tuning_argument_rules(zig):
    # host-side checks, before any device work
    for bad in (0, 4097):
        with pytest.raises(zig.ZigError) as e:
            zig.zig_batch_set_chunk(bad)
        assert e.value.status == zig.ZIG_E_INVAL
    # an empty batch or a rep count out of range
    assert zig.raw_call("zig_batch_autotune", None, 0, None, 0, 3, None, None, 0, None,
                        None) == zig.ZIG_E_INVAL
    assert zig.raw_call("zig_batch_autotune", 0x1000, 4, 0x1000, 1 << 20, 0, None, None, 0,
                        None, None) == zig.ZIG_E_INVAL
