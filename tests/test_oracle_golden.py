"""The oracle against the numbers the paper prints (tests/golden/).

Each fixture entry cites its passage; the check recomputes the quantity
from the oracle's tables and compares it at the precision printed.
"""
import json
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "paper_printed_values.json")))["values"]
BY_NAME = {g["name"]: g for g in GOLD}


def _printed(name, x):
    g = BY_NAME[name]
    return round(x, g["decimals"]) == pytest.approx(g["value"])


def test_every_fixture_has_a_citation():
    assert GOLD and all(g.get("cite") for g in GOLD)


def test_layer_count(orc):
    g = BY_NAME["L_max_exponential"]
    t = orc.tables(0)
    assert t.imax == g["imax"] and t.L == g["value"]


def test_percentages(orc):
    t = orc.tables(0)
    assert _printed("overhang_volume_percent_exponential", 100.0 * (t.imax - t.L) / t.imax)
    assert _printed("fast_exit_percent_exponential", 100.0 * t.L / t.imax)
    # eps: the widest band (chord to curve) as a share of its box height
    assert _printed("widest_band_percent_exponential", 100.0 * t.eps)
    assert _printed("rejection_tests_eliminated_percent_exponential", 100.0 * (1.0 - t.eps))


def test_packed_zero_fringe_fixture(orc):
    """tests/golden/packed_f32_zero_fringe.json (written by
    make_packed_zero.py from the oracle's Philox): each counter's packed
    FP32 first word has a layer index >= L_max and U = 0; the normal's has
    its sign bit set."""
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden",
                           "packed_f32_zero_fringe.json")) as f:
        fx = json.load(f)
    for name, dist in (("exp", orc.EXP), ("normal", orc.NORMAL)):
        w = orc.packed_words(fx["seed"], fx[name], orc.F32, 1)[0]
        assert (w & 0xFF) >= orc.tables(dist).L and (w >> 41) == 0
        if name == "normal":
            assert (w >> 8) & 1 == 1
