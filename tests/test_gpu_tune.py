"""GPU: launch shapes and the autotuner.

Every candidate shape, at full and at one CTA per SM, writes exactly the
bits of the default shape (outputs depend on the counter alone), for
ragged sizes, a misaligned start and a run across the 2^32 counter carry;
the autotuner measures every candidate, selects the fastest, and the
choice survives a save/load of the tuning cache.
"""
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def zig():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_1403_6870_gb300 import build

    build.build()
    import paper_1403_6870_gb300 as z

    z.zig_build_tables()
    yield z
    for dist in (0, 1):
        for dtype in (0, 1):
            d = z.zig_tune_candidates(dtype)[0]
            z.zig_tune_set(dist, dtype, dict(d, blocks_per_sm=0))


def _gen(z, dist, dtype, n, offset, pad):
    t = torch.full((n + pad,), float("nan"), device="cuda",
                   dtype=torch.float64 if dtype else torch.float32)
    v = t[pad:]
    (z.zig_exponential if dist == 0 else z.zig_normal)(v, seed=0x5EED, offset=offset)
    torch.cuda.synchronize()
    return v.cpu().numpy().view(np.uint64 if dtype else np.uint32).copy()


@pytest.mark.parametrize("dist", [0, 1])
@pytest.mark.parametrize("dtype", [0, 1])
def test_every_shape_writes_the_same_bits(zig, dist, dtype):
    cands = zig.zig_tune_candidates(dtype)
    cases = [(3 * 224 * 32 + 5, 0, 1), (1000003, 2**32 - 500000, 3), (7, 11, 0)]
    zig.zig_tune_set(dist, dtype, dict(cands[0], blocks_per_sm=0))
    ref = [_gen(zig, dist, dtype, *c) for c in cases]
    for c in cands:
        for bps in (0, 1):
            zig.zig_tune_set(dist, dtype, dict(c, blocks_per_sm=bps))
            assert zig.zig_tune_get(dist, dtype)["blocks_per_sm"] == bps
            for case, r in zip(cases, ref):
                got = _gen(zig, dist, dtype, *case)
                assert np.array_equal(got, r), (c, bps, case)
    assert zig.zig_status_poll() == zig.ZIG_OK
    zig.zig_tune_set(dist, dtype, dict(cands[0], blocks_per_sm=0))


def test_tune_set_rejects_unknown_shapes(zig):
    with pytest.raises(zig.ZigError):
        zig.zig_tune_set(1, 1, {"V": 3, "R": 3, "min_blocks": 4, "blocks_per_sm": 0})
    with pytest.raises(zig.ZigError):
        zig.zig_tune_set(1, 1, {"V": 4, "R": 4, "min_blocks": 4, "blocks_per_sm": -1})


def test_autotune_selects_the_fastest_and_caches_it(zig, tmp_path):
    scratch = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > L2
    chosen, results = zig.zig_autotune(1, 0, scratch, reps=2)
    cands = {(c["V"], c["R"], c["min_blocks"]) for c in zig.zig_tune_candidates(0)}
    assert {(r["V"], r["R"], r["min_blocks"]) for r in results} == cands
    assert all(r["gsamples_s"] > 0 and r["blocks_per_sm"] >= 1 for r in results)
    best = max(results, key=lambda r: r["gsamples_s"])
    assert chosen == best
    assert zig.zig_tune_get(1, 0) == chosen
    path = tmp_path / "tune.jsonl"
    zig.zig_tune_save(str(path))
    name = torch.cuda.get_device_name()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    rows = [json.loads(x) for x in path.read_text().splitlines()]
    mine = [r for r in rows if r["device"] == name and r["sms"] == sms and r["dist"] == "normal"
            and r["dtype"] == "f32"]
    assert len(mine) == 1 and (mine[0]["V"], mine[0]["R"]) == (chosen["V"], chosen["R"])
    # reset, then loading the cache restores the choice on this device
    d = zig.zig_tune_candidates(0)[0]
    zig.zig_tune_set(1, 0, dict(d, blocks_per_sm=0))
    zig.zig_tune_load(str(path))
    got = zig.zig_tune_get(1, 0)
    assert (got["V"], got["R"], got["min_blocks"], got["blocks_per_sm"]) == (
        chosen["V"], chosen["R"], chosen["min_blocks"], chosen["blocks_per_sm"])
