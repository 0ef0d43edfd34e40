"""Sharding one decision's sieve points across ranks (one process per GPU).

The 2^k sieve evaluations of Lemma 6.5 are independent (the paper vectorises
over them, Sec. 8), so rank r of W evaluates a contiguous range of points with
``tmotif_decide(..., point_begin, point_end)`` on its own replica of the graph.
The per-point sums are combined by XOR.  Collective libraries offer no XOR
reduction, so the exchange is one all-gather of 8 bytes per point followed by
a local XOR.
"""
from __future__ import annotations

import numpy as np


def shard_range(npts: int, rank: int, world: int):
    """Contiguous share [begin, end) of npts points for `rank` of `world`."""
    base, extra = divmod(npts, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def gather_xor(local: np.ndarray, npts: int, group=None):
    """All-gather every rank's per-point sums (rank order) and XOR them."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    width = -(-npts // world)
    buf = torch.zeros(width, dtype=torch.int64)
    if len(local):
        buf[: len(local)] = torch.from_numpy(np.ascontiguousarray(local).view(np.int64))
    if dist.get_backend(group) == "nccl":
        buf = buf.cuda()
    parts = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    per_point = []
    for r, part in enumerate(parts):
        b, e = shard_range(npts, r, world)
        per_point.append(part.cpu().numpy().view(np.uint64)[: e - b])
    per_point = np.concatenate(per_point)
    total = int(np.bitwise_xor.reduce(per_point)) if len(per_point) else 0
    return per_point, total


def tmotif_decide_sharded(graph, k, multiset, *, group=None, evaluate=None, **query):
    """Decide on this rank's share of the points and combine across ranks.

    `evaluate(begin, end)` returns the per-point sums of [begin, end); by
    default it is the library's tmotif_decide on `graph`.  Returns
    (found, sieve_sum, per_point) for the whole query (first repeat)."""
    import torch.distributed as dist

    npts = 1 << k
    b, e = shard_range(npts, dist.get_rank(group), dist.get_world_size(group))
    if evaluate is None:
        from . import tmotif_decide

        def evaluate(lo, hi):
            return tmotif_decide(graph, k, multiset, point_begin=lo, point_end=hi, **query).per_point

    local = evaluate(b, e) if e > b else np.zeros(0, np.uint64)
    per_point, total = gather_xor(local, npts, group)
    return total != 0, total, per_point
