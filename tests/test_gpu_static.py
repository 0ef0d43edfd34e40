"""GPU parity of the static preprocessing sieve (Sec. 8.1 (ii)).

Bit-exact against the oracle: the per-vertex sums Q_u, the per-point sums of
the decision on the preprocessed graph, and the extracted paths (both
procedures) on it.
"""
import random

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
ANY = oracle.ANY


@pytest.fixture(scope="module")
def tm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2001_07158_gb300 as tm

    return tm


def gpu_graph(tm, g):
    return tm.tmotif_create_graph(g.n, g.src, g.dst, g.time, g.color, g.num_colors, undirected=g.undirected)


def rand_case(rng, i):
    n = rng.randint(3, 80)
    m = rng.randint(0, 5 * n)
    ncol = rng.randint(1, 5)
    g = synth.Graph(n, np.array([rng.randrange(n) for _ in range(m)], np.uint32),
                    np.array([rng.randrange(n) for _ in range(m)], np.uint32),
                    np.array([rng.randint(1, 12) for _ in range(m)], np.uint32),
                    np.array([rng.randrange(ncol) for _ in range(n)], np.uint32), ncol, rng.random() < 0.3)
    k = rng.randint(2, 8)
    ms = [rng.randrange(ncol) for _ in range(k)]
    kw = {"seed": rng.getrandbits(63)}
    if i % 5 == 1:
        kw["start"] = rng.randrange(n)
    if i % 5 == 2:
        kw["end"] = rng.randrange(n)
    return g, k, ms, kw


def test_static_sums_match_oracle(tm):
    rng = random.Random(4040)
    nonzero = 0
    for i in range(100):
        g, k, ms, kw = rand_case(rng, i)
        G = gpu_graph(tm, g)
        qv, kept = tm.tmotif_static_sieve(G, k, ms, **kw)
        ref = oracle.static_through(g.n, g.src, g.dst, g.time, g.color, g.num_colors, k, ms,
                                    undirected=g.undirected, **kw)
        assert np.array_equal(qv, ref), i
        assert kept == int(np.count_nonzero(ref))
        nonzero += kept > 0
        G.close()
    assert nonzero > 30


def test_static_sums_config1(tm):
    g, q = synth.config1_tiny()
    G = gpu_graph(tm, g)
    for seed in (1, 2, 3):
        qv, _ = tm.tmotif_static_sieve(G, q.k, q.multiset, seed=seed)
        ref = oracle.static_through(g.n, g.src, g.dst, g.time, g.color, g.num_colors, q.k, q.multiset, seed=seed)
        assert np.array_equal(qv, ref)
    G.close()


def test_preprocessed_decision_matches_oracle(tm):
    rng = random.Random(4141)
    for i in range(60):
        g, k, ms, kw = rand_case(rng, i)
        G = gpu_graph(tm, g)
        d = tm.tmotif_decide(G, k, ms, preprocess=True, **kw)
        f, s, pp, keep = oracle.decide_preprocessed(g.n, g.src, g.dst, g.time, g.color, g.num_colors, k, ms,
                                                    undirected=g.undirected, **kw)
        assert np.array_equal(d.per_point, pp) and d.sieve_sum == s and d.found == f, i
        plain = tm.tmotif_decide(G, k, ms, **kw)
        assert plain.found == d.found
        G.close()


def test_preprocessed_extraction_matches_oracle(tm):
    g, q = synth.config1_tiny()
    G = gpu_graph(tm, g)
    for seed in (q.seed, 5):
        _, _, _, keep = oracle.decide_preprocessed(g.n, g.src, g.dst, g.time, g.color, g.num_colors, q.k,
                                                   q.multiset, seed=seed)
        sel = keep[g.src] & keep[g.dst]
        args = (g.n, g.src[sel], g.dst[sel], g.time[sel], g.color, g.num_colors, q.k, q.multiset)
        f, v, t = tm.tmotif_extract(G, q.k, q.multiset, seed=seed, preprocess=True)
        fo, vo, to = oracle.extract_localized(*args, seed=seed)
        assert f == fo and np.array_equal(v, vo) and np.array_equal(t, to)
        f, v, t = tm.tmotif_extract(G, q.k, q.multiset, seed=seed, preprocess=True, method="halving")
        fo, vo, to, _ = oracle.extract(*args, seed=seed)
        assert f == fo and np.array_equal(v, vo) and np.array_equal(t, to)
    G.close()


def test_preprocessing_prunes_a_sparse_match(tm):
    # one planted path with a rare colour pattern in a large random graph:
    # the static sieve keeps few vertices and the decision is unchanged
    g = synth.uniform_graph(20000, 60000, 500, 12, seed=91)
    ms = [11, 10, 11, 10, 11]
    g2, _ = synth.plant_paths(g, ms, 1, seed=92)
    G = gpu_graph(tm, g2)
    qv, kept = tm.tmotif_static_sieve(G, 5, ms, seed=3)
    assert 5 <= kept < 1000
    d = tm.tmotif_decide(G, 5, ms, seed=3, preprocess=True)
    assert d.found == tm.tmotif_decide(G, 5, ms, seed=3).found
    assert d.found
    G.close()


def test_batch_and_server_reject_preprocessing(tm):
    g, q = synth.config1_tiny()
    G = gpu_graph(tm, g)
    with pytest.raises(tm.TmotifError) as e:
        tm.tmotif_decide_batch([G], [{"k": q.k, "multiset": q.multiset, "preprocess": True}])
    assert e.value.code == 5
    srv = tm.tmotif_server_create(0)
    with pytest.raises(tm.TmotifError) as e:
        tm.tmotif_submit(srv, G, q.k, q.multiset, preprocess=True)
    assert e.value.code == 5
    srv.close()
    G.close()


def test_preprocessing_with_window_and_ec_tuple(tm):
    # the static sieve ignores times (the merged graph); the decision on the
    # kept vertices then applies the window or the EC tuple
    rng = random.Random(4242)
    for i in range(40):
        g, k, ms, kw = rand_case(rng, i)
        t_hi = int(g.time.max()) if len(g.time) else 1
        if i % 2 and t_hi >= k - 1:
            kw["timestamps"] = sorted(rng.sample(range(1, t_hi + 1), k - 1))
        else:
            kw["t_min"], kw["t_max"] = 2, 9
        G = gpu_graph(tm, g)
        d = tm.tmotif_decide(G, k, ms, preprocess=True, **kw)
        f, s, pp, _ = oracle.decide_preprocessed(g.n, g.src, g.dst, g.time, g.color, g.num_colors, k, ms,
                                                 undirected=g.undirected, **kw)
        assert np.array_equal(d.per_point, pp) and d.sieve_sum == s and d.found == f, i
        G.close()
