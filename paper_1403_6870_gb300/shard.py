"""Host-side work partition for several GPUs (one process per GPU).

Every output is independent given its counter, so the generation path
shards without any collective: rank r of G takes a contiguous counter range
and writes exactly the bits a single call over the whole range would.  A
batch of requests shards by whole requests, balanced by size.  Pure Python
(no device work); bench.py uses it under torchrun and the gloo tests
exercise it on CPU ranks.
"""
from __future__ import annotations


def counter_range(offset: int, n_total: int, rank: int, world: int) -> tuple[int, int]:
    """(first counter, count) of rank's share of [offset, offset + n_total):
    contiguous, in rank order, sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("need 0 <= rank < world and n_total >= 0")
    lo = n_total * rank // world
    hi = n_total * (rank + 1) // world
    return offset + lo, hi - lo


def step_counter(offset: int, step: int, rank: int, world: int, n_per_rank: int) -> int:
    """First counter of rank's n_per_rank outputs at a given step when every
    rank makes n_per_rank fresh outputs per step (weak scaling): the ranks'
    ranges of one step are adjacent, and steps follow one another."""
    return offset + (step * world + rank) * n_per_rank


def request_shards(sizes, world: int) -> list[list[int]]:
    """Split request indices over world ranks by size, largest first onto the
    least-loaded rank (ties to the lower rank); each rank's list is in
    increasing index order.  The loads differ by at most the largest size."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    load = [0] * world
    shards: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        shards[r].append(i)
        load[r] += int(sizes[i])
    return [sorted(s) for s in shards]
