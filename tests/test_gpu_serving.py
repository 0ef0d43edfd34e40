"""Batching and serving: every result is the same alone and in the mix.

The batch path and the request server advance many decisions together in
shared layer launches (different graphs, k, seeds, layers); GF(2^64)
arithmetic is exact, so each sieve sum, decision and extracted path must equal
the one tmotif_decide / tmotif_extract give for the same query alone.
"""
import random
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2001_07158_gb300 as tm

    return tm


def small_graphs(tm, count, seed):
    rng = random.Random(seed)
    out = []
    for i in range(count):
        n = rng.randint(50, 800)
        g = synth.tour_graph(n, 8, 288, 12, seed=seed * 1000 + i)
        G = tm.tmotif_create_graph(g.n, g.src, g.dst, g.time, g.color, g.num_colors)
        k = rng.randint(3, 7)
        ms = [rng.randrange(12) for _ in range(k)]
        out.append((G, {"k": k, "multiset": ms, "seed": rng.getrandbits(40), "t_max": rng.choice([0, 200])}))
    return out


def test_batch_equals_individual_decisions(tm):
    # packed form (every query one repeat over all points): windows, start and
    # end vertices and EC timestamp tuples mixed in
    items = small_graphs(tm, 60, seed=3)
    rng = random.Random(33)
    for i, (G, q) in enumerate(items):
        if i % 5 == 1:
            q["start"] = rng.randrange(G.n)
        if i % 5 == 2:
            q["end"] = rng.randrange(G.n)
        if i % 7 == 3:
            q["timestamps"] = sorted(rng.sample(range(1, 289), q["k"] - 1))
            q["t_max"] = 0
    graphs = [G for G, _ in items]
    queries = [q for _, q in items]
    res = tm.tmotif_decide_batch(graphs, queries)
    for (G, q), r in zip(items, res):
        alone = tm.tmotif_decide(G, **q)
        assert r.found == alone.found and r.sieve_sum == alone.sieve_sum
        assert np.array_equal(r.per_point, alone.per_point)
    # scheduler form (a query with two repeats takes the batch off the packed path)
    queries[0] = dict(queries[0], repeats=2)
    res = tm.tmotif_decide_batch(graphs[:20], queries[:20])
    for G, q, r in zip(graphs[:20], queries[:20], res):
        alone = tm.tmotif_decide(G, **q)
        assert r.found == alone.found and r.sieve_sum == alone.sieve_sum
        assert np.array_equal(r.per_point, alone.per_point)


def _serve_all(tm, srv, jobs, poll_sleep=0.0005, timeout=600):
    tickets = []
    for G, q, ex in jobs:
        tickets.append(tm.tmotif_submit(srv, G, q["k"], q["multiset"], is_extract=ex, seed=q["seed"],
                                        t_max=q.get("t_max", 0)))
    results = [None] * len(jobs)
    t0 = time.time()
    while any(r is None for r in results):
        for i, t in enumerate(tickets):
            if results[i] is None:
                r = tm.tmotif_poll(srv, t, jobs[i][1]["k"])
                if r is not None:
                    results[i] = r
        assert time.time() - t0 < timeout
        time.sleep(poll_sleep)
    return results


def test_server_mixed_requests_equal_alone(tm):
    rng = random.Random(11)
    g1, q1 = synth.config1_tiny()
    g2 = synth.powerlaw_graph(20000, 200000, 500, 10, seed=19)
    G1 = tm.tmotif_create_graph(g1.n, g1.src, g1.dst, g1.time, g1.color, g1.num_colors)
    G2 = tm.tmotif_create_graph(g2.n, g2.src, g2.dst, g2.time, g2.color, g2.num_colors)
    jobs = []
    for i in range(40):
        G, nc = (G1, 8) if rng.random() < 0.5 else (G2, 10)
        k = rng.randint(3, 8)
        q = {"k": k, "multiset": [rng.randrange(nc) for _ in range(k)], "seed": rng.getrandbits(40),
             "t_max": rng.choice([0, 0, 300])}
        jobs.append((G, q, rng.random() < 0.3))
    srv = tm.tmotif_server_create(0)
    results = _serve_all(tm, srv, jobs)
    srv.close()
    for (G, q, ex), (dec, verts, times) in zip(jobs, results):
        if ex:
            f, v, t = tm.tmotif_extract(G, q["k"], q["multiset"], seed=q["seed"], t_max=q["t_max"])
            assert dec.found == f
            if f:
                assert np.array_equal(verts, v) and np.array_equal(times, t)
        else:
            alone = tm.tmotif_decide(G, q["k"], q["multiset"], seed=q["seed"], t_max=q["t_max"])
            assert dec.found == alone.found and dec.sieve_sum == alone.sieve_sum
            assert np.array_equal(dec.per_point, alone.per_point)


def test_server_budget_admission(tm):
    g, q = synth.config1_tiny()
    G = tm.tmotif_create_graph(g.n, g.src, g.dst, g.time, g.color, g.num_colors)
    # a budget below one request's need is refused at submission
    tiny = tm.tmotif_server_create(1 << 16)
    with pytest.raises(tm.TmotifError) as e:
        tm.tmotif_submit(tiny, G, q.k, q.multiset, seed=1)
    assert e.value.code == 7
    tiny.close()
    # a budget for about one request at a time still completes them all
    one = tm.tmotif_server_create(24 << 20)
    jobs = [(G, {"k": q.k, "multiset": q.multiset, "seed": s}, False) for s in range(1, 13)]
    res = _serve_all(tm, one, jobs)
    one.close()
    for (G_, qq, _), (dec, _, _) in zip(jobs, res):
        alone = tm.tmotif_decide(G, q.k, q.multiset, seed=qq["seed"])
        assert dec.sieve_sum == alone.sieve_sum and np.array_equal(dec.per_point, alone.per_point)
    other = tm.tmotif_server_create(0)
    with pytest.raises(tm.TmotifError) as e:
        tm.tmotif_poll(other, 12345, 4)
    assert e.value.code == 6
    other.close()


def test_server_wait_times_out_then_completes(tm):
    # a k = 10 request on a mid-size graph takes milliseconds: a zero-timeout
    # wait reports TIMEOUT (4) and leaves it pending; a long wait returns the
    # result, which equals the decision alone
    g = synth.powerlaw_graph(100000, 1500000, 500, 10, seed=23)
    G = tm.tmotif_create_graph(g.n, g.src, g.dst, g.time, g.color, g.num_colors)
    ms = list(range(10))
    srv = tm.tmotif_server_create(0)
    t = tm.tmotif_submit(srv, G, 10, ms, seed=4)
    with pytest.raises(tm.TmotifError) as e:
        tm.tmotif_wait(srv, t, 10, 0)
    assert e.value.code == 4
    dec, _, _ = tm.tmotif_wait(srv, t, 10, 600000)
    alone = tm.tmotif_decide(G, 10, ms, seed=4)
    assert dec.found == alone.found and dec.sieve_sum == alone.sieve_sum
    assert np.array_equal(dec.per_point, alone.per_point)
    with pytest.raises(tm.TmotifError) as e:  # a finished ticket is forgotten
        tm.tmotif_wait(srv, t, 10, 0)
    assert e.value.code == 6
    srv.close()
    G.close()


def test_packed_batch_edge_cases(tm):
    # the packed form with k = 2..9 (1 to 8 rounds of 64 points), undirected
    # graphs, a graph without arcs, a multiset whose colours are absent, and
    # graphs of different colour counts: every per-point value equals the
    # decision alone
    rng = random.Random(77)
    items = []
    for i in range(40):
        n = rng.randint(2, 300)
        m = 0 if i == 5 else rng.randint(1, 6 * n)
        ncol = rng.randint(1, 9)
        g = synth.Graph(n, np.array([rng.randrange(n) for _ in range(m)], np.uint32),
                        np.array([rng.randrange(n) for _ in range(m)], np.uint32),
                        np.array([rng.randint(1, 30) for _ in range(m)], np.uint32),
                        np.array([rng.randrange(ncol) for _ in range(n)], np.uint32), ncol, i % 3 == 0)
        G = tm.tmotif_create_graph(g.n, g.src, g.dst, g.time, g.color, g.num_colors, undirected=g.undirected)
        k = 2 + i % 8
        ms = [rng.randrange(ncol) for _ in range(k)]
        if i == 7:
            ms = [ncol - 1] * k if ncol > 1 else ms
        q = {"k": k, "multiset": ms, "seed": rng.getrandbits(40)}
        if i % 4 == 1:
            q["start"] = rng.randrange(n)
        if i % 4 == 2:
            q["end"] = rng.randrange(n)
        items.append((G, q))
    res = tm.tmotif_decide_batch([G for G, _ in items], [q for _, q in items])
    for (G, q), r in zip(items, res):
        alone = tm.tmotif_decide(G, **q)
        assert np.array_equal(r.per_point, alone.per_point) and r.found == alone.found
    for G, _ in items:
        G.close()


def test_server_cancel(tm):
    # a queue of k = 10 decisions (large requests run one at a time): the last
    # one is still waiting when it is cancelled and completes with CANCELLED
    # (8); every request not cancelled equals its decision alone; a request
    # cancelled after it finished keeps its result; an unknown ticket is
    # NOT_FOUND
    g = synth.powerlaw_graph(100000, 1500000, 500, 10, seed=23)
    G = tm.tmotif_create_graph(g.n, g.src, g.dst, g.time, g.color, g.num_colors)
    ms = list(range(10))
    want = [tm.tmotif_decide(G, 10, ms, seed=s).per_point for s in range(1, 12)]
    small = tm.tmotif_decide(G, 4, ms[:4], seed=3).per_point
    srv = tm.tmotif_server_create(0)
    tickets = [tm.tmotif_submit(srv, G, 10, ms, seed=s) for s in range(1, 13)]
    tm.tmotif_cancel(srv, tickets[-1])
    for i, t in enumerate(tickets[:-1]):
        dec, _, _ = tm.tmotif_wait(srv, t, 10, 600000)
        assert np.array_equal(dec.per_point, want[i]), i
    with pytest.raises(tm.TmotifError) as e:
        tm.tmotif_wait(srv, tickets[-1], 10, 600000)
    assert e.value.code == 8
    # cancelled after it finished: the result stays
    t = tm.tmotif_submit(srv, G, 4, ms[:4], seed=3)
    time.sleep(2.0)
    tm.tmotif_cancel(srv, t)
    dec, _, _ = tm.tmotif_wait(srv, t, 4, 600000)
    assert np.array_equal(dec.per_point, small)
    with pytest.raises(tm.TmotifError) as e:
        tm.tmotif_cancel(srv, 987654321)
    assert e.value.code == 6
    srv.close()
    G.close()
