"""Multi-rank path on CPU: sieve points sharded over gloo ranks.

Each rank evaluates its contiguous share of the 2^k points (the oracle stands
in for the per-rank GPU evaluation here, since the test runs without a GPU),
the shares are all-gathered and XOR-combined; every rank must end with the
same per-point sums and decision as one full evaluation.
"""
import json
import os
import socket

import numpy as np
import pytest

import oracle
import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, outdir, k_override):
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    from paper_2001_07158_gb300.sharded import shard_range, tmotif_decide_sharded

    g, q = synth.config1_brute()
    k = k_override or q.k
    ms = list(q.multiset[:k]) + [0] * max(0, k - len(q.multiset))

    def evaluate(b, e):
        return oracle.decide(g.n, g.src, g.dst, g.time, g.color, g.num_colors, k, ms, seed=7, point_begin=b,
                             point_end=e)[2]

    found, total, pp = tmotif_decide_sharded(None, k, ms, evaluate=evaluate)
    b, e = shard_range(1 << k, rank, world)
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
        json.dump({"found": bool(found), "total": int(total), "pp": [int(x) for x in pp], "share": [b, e]}, f)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,k", [(2, 0), (3, 0), (3, 2)])
def test_sharded_decision_matches_full(tmp_path, oracle_mod, world, k):
    import torch.multiprocessing as mp

    import __graft_entry__

    __graft_entry__.build()
    port = _free_port()
    mp.spawn(_worker, args=(world, port, str(tmp_path), k), nprocs=world, join=True)
    g, q = synth.config1_brute()
    kk = k or q.k
    ms = list(q.multiset[:kk]) + [0] * max(0, kk - len(q.multiset))
    f, s, pp = oracle.decide(g.n, g.src, g.dst, g.time, g.color, g.num_colors, kk, ms, seed=7)
    shares = []
    for r in range(world):
        res = json.load(open(tmp_path / f"rank{r}.json"))
        assert res["found"] == f and res["total"] == s
        assert np.array_equal(np.array(res["pp"], dtype=np.uint64), pp)
        shares.append(tuple(res["share"]))
    # the shares tile [0, 2^k) in rank order
    assert shares[0][0] == 0 and shares[-1][1] == 1 << kk
    assert all(shares[i][1] == shares[i + 1][0] for i in range(world - 1))
