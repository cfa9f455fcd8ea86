"""Multi-process (world size 2, gloo, CPU) checks of the sharding logic.

Each rank takes its counter range with paper_1403_6870_gb300.shard and
computes its outputs with the oracle; gathered in rank order they equal a
single unsharded oracle run bit for bit.  Per-step weak-scaling counters
are disjoint across ranks and steps, the max-over-ranks time is what every
rank sees, and request shards cover every request once with balanced
loads.  No GPU is involved (the generation path itself needs no
collective).
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1403_6870_gb300.shard import counter_range, request_shards, step_counter  # noqa: E402

WORLD = 2
SEED = 0x0123456789ABCDEF


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    try:
        dist.init_process_group("gloo", rank=rank, world_size=WORLD)
        from oracle import oracle
        import workloads as W

        res = {}
        # (1) counter-range shards reassemble the unsharded output
        for dist_id, dtype in ((1, 1), (0, 0)):
            n_total, offset = 20011, 2**32 - 10000  # ragged, across the carry
            first, cnt = counter_range(offset, n_total, rank, WORLD)
            vals, errs, _, _ = oracle.fill(dist_id, dtype, SEED, first, cnt, nthreads=1)
            parts = [None] * WORLD
            dist.all_gather_object(parts, (first, cnt, vals.tobytes(), errs))
            res[f"parts_{dist_id}_{dtype}"] = parts
        # (2) weak-scaling counters per step
        n = 1000
        mine = [(step_counter(5, s, rank, WORLD, n), n) for s in range(3)]
        allc = [None] * WORLD
        dist.all_gather_object(allc, mine)
        res["steps"] = allc
        # (3) max over ranks of a per-rank time
        t = torch.tensor([1.5 + rank], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        res["tmax"] = float(t.item())
        # (4) request shards
        sizes = [q["n"] for q in W.batch_requests(count=512)]
        sh = request_shards(sizes, WORLD)[rank]
        allr = [None] * WORLD
        dist.all_gather_object(allr, sh)
        res["req"] = (sizes, allr)
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, res))
    except Exception as e:  # report instead of hanging the parent
        q.put((rank, repr(e)))


@pytest.fixture(scope="module")
def gathered(orc):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(WORLD):
        rank, res = q.get(timeout=300)
        out[rank] = res
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(WORLD):
        assert isinstance(out[r], dict), out[r]
    return out


@pytest.mark.parametrize("dist_id,dtype", [(1, 1), (0, 0)])
def test_shards_reassemble_the_unsharded_output(gathered, orc, dist_id, dtype):
    parts = gathered[0][f"parts_{dist_id}_{dtype}"]
    assert parts == gathered[1][f"parts_{dist_id}_{dtype}"]
    n_total, offset = 20011, 2**32 - 10000
    assert parts[0][0] == offset and parts[1][0] == parts[0][0] + parts[0][1]
    assert parts[0][1] + parts[1][1] == n_total and abs(parts[0][1] - parts[1][1]) <= 1
    npdt = np.float64 if dtype == 1 else np.float32
    joined = np.concatenate([np.frombuffer(p[2], dtype=npdt) for p in parts])
    ref, errs, _, _ = orc.fill(dist_id, dtype, SEED, offset, n_total)
    assert errs == 0 and all(p[3] == 0 for p in parts)
    assert np.array_equal(joined.view(np.uint8), ref.view(np.uint8))


def test_step_counters_are_disjoint(gathered):
    ranges = [r for rank_list in gathered[0]["steps"] for r in rank_list]
    ranges.sort()
    assert ranges[0][0] == 5
    for (a, na), (b, _) in zip(ranges, ranges[1:]):
        assert a + na == b  # adjacent, no overlap, no gap
    assert len(ranges) == 3 * WORLD


def test_max_over_ranks(gathered):
    assert gathered[0]["tmax"] == gathered[1]["tmax"] == 2.5


def test_request_shards_cover_once_and_balance(gathered):
    sizes, shards = gathered[0]["req"]
    flat = sorted(i for s in shards for i in s)
    assert flat == list(range(len(sizes)))
    loads = [sum(sizes[i] for i in s) for s in shards]
    assert max(loads) - min(loads) <= max(sizes)


def test_counter_range_arguments():
    assert counter_range(10, 7, 0, 1) == (10, 7)
    assert [counter_range(0, 10, r, 3) for r in range(3)] == [(0, 3), (3, 3), (6, 4)]
    with pytest.raises(ValueError):
        counter_range(0, 10, 3, 3)
    assert request_shards([5, 1, 1], 4) == [[0], [1], [2], []]
