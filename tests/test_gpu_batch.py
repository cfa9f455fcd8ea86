"""GPU parity of the batched path (zig_batch) against the oracle.

Every element of a mixed batch (both distributions, both precisions,
sizes from 0 to several tiles, misaligned outputs, the 2^32 counter carry)
is compared with the oracle's plain map of its standard variates (rule in
tests/parity.py check_batch); then the full serving mix (4096 requests,
~3.6e9 variates) on sampled positions, with every request's completion
time recorded.
"""
import numpy as np
import pytest

import workloads as W
from parity import check_batch

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


def _tdt(dtype):
    return torch.float64 if dtype == 1 else torch.float32


def _alloc(reqs, pad_of):
    """One buffer per request, the output starting pad_of(r) elements in."""
    bufs = []
    for r, q in enumerate(reqs):
        pad = pad_of(r)
        b = torch.full((q["n"] + pad + 4,), float("nan"), dtype=_tdt(q["dtype"]), device="cuda")
        q["out"] = b.data_ptr() + pad * b.element_size()
        bufs.append((b, pad))
    return bufs


def _serve(z, reqs):
    h = z.pack_requests(reqs)
    assert z.zig_batch_validate(h) == z.ZIG_OK
    d = torch.from_numpy(h.view(np.uint8)).cuda()
    ws = torch.empty(z.zig_batch_workspace_bytes(len(reqs)), dtype=torch.uint8, device="cuda")
    done = torch.full((len(reqs),), -1, dtype=torch.int64, device="cuda")
    z.zig_batch(d, len(reqs), ws, done_ns=done)
    assert z.zig_status_poll() == z.ZIG_OK
    return done.cpu().numpy()


def _compare(orc, q, got, idx):
    """Element by element against the oracle's plain map (tests/parity.py
    check_batch): fringe draws bit-exact up to flipped decisions, fast-path
    draws within the fold's derived bound."""
    return check_batch(orc, q, got, idx)


def test_mixed_small_batch_every_element(zig, orc):
    sizes = [0, 1, 3, 5, 8, 31, 100, 1000, 3584, 3585, 3584 * 3 + 17, 70001, 250000]
    reqs = []
    rng = np.random.default_rng(99)
    for k, n in enumerate(sizes * 2):
        dist, dtype = k % 2, (k // 2) % 2
        reqs.append(dict(n=n, dist=dist, dtype=dtype, seed=W.splitmix64(k),
                         offset=int(rng.integers(0, 2**40)) if k != 7 else 2**32 - 1000,
                         p0=float(10 ** rng.uniform(-1, 1)) if dist == 0 else float(rng.uniform(-5, 5)),
                         p1=0.0 if dist == 0 else float(10 ** rng.uniform(-2, 2))))
    bufs = _alloc(reqs, lambda r: r % 3)
    done = _serve(zig, reqs)
    for q, (b, pad), d in zip(reqs, bufs, done):
        host = b.cpu().numpy()
        assert np.all(np.isnan(host[:pad])) and np.all(np.isnan(host[pad + q["n"]:]))
        if q["n"] == 0:
            assert d == 0
            continue
        assert d > 0
        got = host[pad:pad + q["n"]]
        _compare(orc, q, got, np.arange(q["n"], dtype=np.uint64))


def test_invalid_request_is_rejected(zig):
    good = dict(n=10, dist=0, dtype=1, seed=1, offset=0, p0=1.0, p1=0.0)
    bad = dict(good, p0=-1.0)
    b = torch.zeros(20, dtype=torch.float64, device="cuda")
    good["out"] = bad["out"] = b.data_ptr()
    assert zig.zig_batch_validate(zig.pack_requests([good])) == zig.ZIG_OK
    assert zig.zig_batch_validate(zig.pack_requests([good, bad])) == zig.ZIG_E_INVAL
    h = zig.pack_requests([bad])
    d = torch.from_numpy(h.view(np.uint8)).cuda()
    ws = torch.empty(zig.zig_batch_workspace_bytes(1), dtype=torch.uint8, device="cuda")
    zig.zig_batch(d, 1, ws)
    assert zig.zig_status_poll() == zig.ZIG_E_INVAL
    assert torch.all(b == 0)


def test_serving_mix_sampled(zig, orc):
    reqs = W.batch_requests()
    bufs = _alloc(reqs, lambda r: 0)
    done = _serve(zig, reqs)
    assert np.all(done[[q["n"] > 0 for q in reqs]] > 0)
    rng = np.random.default_rng(5)
    for q, (b, pad) in zip(reqs, bufs):
        n = q["n"]
        idx = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, size=8)])).astype(np.uint64)
        got = b[torch.from_numpy(idx.astype(np.int64)).cuda()].cpu().numpy()
        _compare(orc, q, got, idx)


def test_identity_parameters_equal_plain_calls(zig):
    # rate 1 and (mean 0, sd 1) make the folded fast path RN((1 + U) sX - sX)
    # and leave fringe draws unchanged, so each request equals the plain call
    # on the same key and counters bit for bit
    reqs = []
    for k, n in enumerate([1, 7, 3584 * 5 + 3, 100003, 1 << 20]):
        for dist in (0, 1):
            for dtype in (0, 1):
                reqs.append(dict(n=n, dist=dist, dtype=dtype, seed=W.splitmix64(100 + k),
                                 offset=(k * 2**31 + 77) if k != 2 else 2**32 - 5000,
                                 p0=1.0 if dist == 0 else 0.0, p1=0.0 if dist == 0 else 1.0))
    bufs = _alloc(reqs, lambda r: r % 2)
    _serve(zig, reqs)
    for q, (b, pad) in zip(reqs, bufs):
        got = b[pad:pad + q["n"]]
        want = torch.empty_like(got)
        fn = zig.zig_exponential if q["dist"] == 0 else zig.zig_normal
        fn(want, q["n"], q["seed"], q["offset"])
        it = torch.int64 if q["dtype"] == 1 else torch.int32
        assert torch.equal(got.view(it), want.view(it)), q
    assert zig.zig_status_poll() == zig.ZIG_OK


def test_graph_captured_batch_replays(zig, orc):
    """zig_batch captured once in a CUDA graph and replayed with the request
    table rewritten in place (new keys and counter offsets, same outputs):
    each replay matches the oracle element by element and stamps every
    request's completion time afresh, so the workspace state of one replay
    does not leak into the next."""
    rng = np.random.default_rng(2024)
    sizes = [1, 5, 3584, 3585, 20000, 131072 + 9, 0, 777]
    reqs = []
    for k, n in enumerate(sizes):
        dist, dtype = k % 2, (k // 2) % 2
        reqs.append(dict(n=n, dist=dist, dtype=dtype, seed=0, offset=0,
                         p0=float(10 ** rng.uniform(-1, 1)) if dist == 0 else float(rng.uniform(-5, 5)),
                         p1=0.0 if dist == 0 else float(10 ** rng.uniform(-2, 2))))
    bufs = _alloc(reqs, lambda r: r % 3)
    d = torch.from_numpy(zig.pack_requests(reqs).view(np.uint8)).cuda()
    ws = torch.empty(zig.zig_batch_workspace_bytes(len(reqs)), dtype=torch.uint8, device="cuda")
    done = torch.full((len(reqs),), -1, dtype=torch.int64, device="cuda")
    zig.zig_batch(d, len(reqs), ws, done_ns=done)  # warm-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        zig.zig_batch(d, len(reqs), ws, done_ns=done)
    for rep in range(2):
        for k, q in enumerate(reqs):
            q["seed"] = W.splitmix64(1000 * (rep + 1) + k)
            q["offset"] = 2**32 - 4000 if k == 3 else int(rng.integers(0, 2**40))
        d.copy_(torch.from_numpy(zig.pack_requests(reqs).view(np.uint8)))
        done.fill_(-1)
        for b, _ in bufs:
            b.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert zig.zig_status_poll() == zig.ZIG_OK
        stamps = done.cpu().numpy()
        for q, (b, pad), st in zip(reqs, bufs, stamps):
            host = b.cpu().numpy()
            assert np.all(np.isnan(host[:pad])) and np.all(np.isnan(host[pad + q["n"]:]))
            if q["n"] == 0:
                assert st == 0
                continue
            assert st > 0
            _compare(orc, q, host[pad:pad + q["n"]], np.arange(q["n"], dtype=np.uint64))


def test_overlapping_batches_keep_their_own_stamps(zig, orc):
    """Two batches in flight at once on two streams, each with its own
    workspace and completion array (a large one and a small one, queued
    back to back, many times): every request of each batch is stamped in its
    own array, nothing is written past the small batch's count (its array is
    padded with sentinels to the large count), and the outputs of both match
    the oracle."""
    rng = np.random.default_rng(77)

    def make(count, n_of, seed0):
        reqs = []
        for k in range(count):
            dist, dtype = k % 2, (k // 2) % 2
            reqs.append(dict(n=n_of(k), dist=dist, dtype=dtype, seed=W.splitmix64(seed0 + k),
                             offset=int(rng.integers(0, 2**40)),
                             p0=1.5 if dist == 0 else -0.25, p1=0.0 if dist == 0 else 2.0))
        return reqs

    big = make(256, lambda k: 20000 + 37 * k, 5000)
    small = make(4, lambda k: 3000 + k, 9000)
    bufs_big, bufs_small = _alloc(big, lambda r: 0), _alloc(small, lambda r: 0)
    d_big = torch.from_numpy(zig.pack_requests(big).view(np.uint8)).cuda()
    d_small = torch.from_numpy(zig.pack_requests(small).view(np.uint8)).cuda()
    ws_big = torch.empty(zig.zig_batch_workspace_bytes(len(big)), dtype=torch.uint8, device="cuda")
    ws_small = torch.empty(zig.zig_batch_workspace_bytes(len(small)), dtype=torch.uint8,
                           device="cuda")
    done_big = torch.empty(len(big), dtype=torch.int64, device="cuda")
    done_small = torch.empty(len(big), dtype=torch.int64, device="cuda")  # padded
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    for it in range(20):
        done_big.fill_(-1)
        done_small.fill_(-1)
        torch.cuda.synchronize()
        zig.zig_batch(d_big, len(big), ws_big, done_ns=done_big, stream=sa)
        zig.zig_batch(d_small, len(small), ws_small, done_ns=done_small, stream=sb)
        torch.cuda.synchronize()
        assert zig.zig_status_poll() == zig.ZIG_OK
        db, ds = done_big.cpu().numpy(), done_small.cpu().numpy()
        assert np.all(db > 0), it
        assert np.all(ds[:len(small)] > 0), it
        assert np.all(ds[len(small):] == -1), it
    for reqs, bufs in ((big[::37], bufs_big[::37]), (small, bufs_small)):
        for q, (b, pad) in zip(reqs, bufs):
            host = b.cpu().numpy()
            _compare(orc, q, host[pad:pad + q["n"]], np.arange(q["n"], dtype=np.uint64))


def test_batch_autotune_keeps_every_bit(zig):
    """zig_batch_autotune times the candidate chunk sizes on the caller's
    batch and keeps the fastest; the chunk size changes only the order in
    which tiles are served, so the outputs with the tuned chunk, with the
    smallest candidate and with the default are identical bit for bit."""
    rng = np.random.default_rng(77)
    reqs = []
    for k, n in enumerate([3584 * 40 + 3, 1, 70001, 250000, 5, 3584 * 17]):
        dist, dtype = k % 2, (k // 2) % 2
        reqs.append(dict(n=n, dist=dist, dtype=dtype, seed=W.splitmix64(500 + k),
                         offset=int(rng.integers(0, 2**40)),
                         p0=float(10 ** rng.uniform(-1, 1)) if dist == 0 else float(rng.uniform(-5, 5)),
                         p1=0.0 if dist == 0 else float(10 ** rng.uniform(-2, 2))))
    bufs = _alloc(reqs, lambda r: r % 3)
    d = torch.from_numpy(zig.pack_requests(reqs).view(np.uint8)).cuda()
    ws = torch.empty(zig.zig_batch_workspace_bytes(len(reqs)), dtype=torch.uint8, device="cuda")

    def outputs():
        return [b.cpu().numpy().view(np.uint64 if q["dtype"] else np.uint32).copy()
                for q, (b, _) in zip(reqs, bufs)]

    try:
        assert zig.zig_batch_get_chunk() == 64
        zig.zig_batch(d, len(reqs), ws)
        ref = outputs()
        chosen, table = zig.zig_batch_autotune(d, len(reqs), ws, reps=2)
        assert sorted(e["chunk"] for e in table) == [16, 32, 64, 128]
        assert all(e["ms"] > 0 for e in table)
        assert chosen == min(table, key=lambda e: e["ms"])["chunk"]
        assert zig.zig_batch_get_chunk() == chosen
        for c in (chosen, 16, 1, 4096):
            zig.zig_batch_set_chunk(c)
            for b, _ in bufs:
                b.fill_(float("nan"))
            zig.zig_batch(d, len(reqs), ws)
            got = outputs()
            assert all(np.array_equal(a, r) for a, r in zip(got, ref)), c
        assert zig.zig_status_poll() == zig.ZIG_OK
    finally:
        zig.zig_batch_set_chunk(64)


def test_batch_tile_boundaries(zig, orc):
    """Requests of 8191, 8192, 8193 and 2 x 8192 + 1 variates (the batch's
    tile is 8192 outputs for both precisions), each against the oracle's
    plain map element by element."""
    rng = np.random.default_rng(31)
    reqs = []
    for k, n in enumerate([8191, 8192, 8193, 16385] * 2):
        dist, dtype = k % 2, k // 4
        reqs.append(dict(n=n, dist=dist, dtype=dtype, seed=W.splitmix64(900 + k),
                         offset=int(rng.integers(0, 2**40)),
                         p0=float(10 ** rng.uniform(-1, 1)) if dist == 0 else float(rng.uniform(-5, 5)),
                         p1=0.0 if dist == 0 else float(10 ** rng.uniform(-2, 2))))
    bufs = _alloc(reqs, lambda r: (r * 5) % 4)
    done = _serve(zig, reqs)
    for q, (b, pad), d in zip(reqs, bufs, done):
        host = b.cpu().numpy()
        assert d > 0
        assert np.all(np.isnan(host[:pad])) and np.all(np.isnan(host[pad + q["n"]:]))
        _compare(orc, q, host[pad:pad + q["n"]], np.arange(q["n"], dtype=np.uint64))
