"""The seeded input generators follow the stated recipe (CPU only).

The benchmark and the parity tests stand synthetic graphs in for the paper's
datasets (Sec. 9): power-law out-degrees with destinations uniform, uniform
timestamps, uniform or Zipf colours, planted matching paths (Sec. 10.1),
tour-style and timetable graphs for the transport setting (Sec. 9.3).  These
tests pin the shapes, ranges and determinism of those generators, so that a
change to a workload shows up here rather than as a silent shift in the
measured numbers.
"""
import numpy as np
import pytest

import synth


def _valid(g):
    assert g.src.dtype == g.dst.dtype == g.time.dtype == g.color.dtype == np.uint32
    assert len(g.src) == len(g.dst) == len(g.time)
    assert len(g.color) == g.n
    assert int(g.src.max()) < g.n and int(g.dst.max()) < g.n
    assert int(g.time.min()) >= 1
    assert int(g.color.max()) < g.num_colors


def test_generators_are_deterministic():
    a, qa = synth.config1_tiny()
    b, qb = synth.config1_tiny()
    for f in ("src", "dst", "time", "color"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    assert np.array_equal(qa.multiset, qb.multiset)
    c = synth.powerlaw_graph(5000, 40000, 100, 8, seed=1)
    d = synth.powerlaw_graph(5000, 40000, 100, 8, seed=2)
    assert not np.array_equal(c.dst, d.dst)


def test_config1_shapes():
    g, q = synth.config1_tiny()
    _valid(g)
    assert (g.n, g.m, g.num_colors, q.k) == (1000, 10_000, 8, 4)
    assert int(g.time.max()) <= 100
    b, qb = synth.config1_brute()
    _valid(b)
    assert (b.n, b.m, qb.k) == (30, 120, 4)


def test_powerlaw_out_degrees():
    # discrete power law of exponent 2.1 rescaled to sum to m: most vertices
    # have a small out-degree, a few hubs a large one; destinations uniform
    n, m = 200_000, 2_000_000
    g = synth.powerlaw_graph(n, m, 1000, 16, seed=3)
    _valid(g)
    assert g.m == m
    deg = np.bincount(g.src, minlength=n)
    assert deg.sum() == m
    assert np.median(deg) < m / n          # skewed: median below the mean
    assert deg.max() > 50 * m / n          # hubs
    indeg = np.bincount(g.dst, minlength=n)
    assert indeg.max() < 6 * m / n         # uniform destinations: no in-hubs
    assert 1 <= int(g.time.min()) and int(g.time.max()) <= 1000


def test_config2_mid_recipe():
    g, q = synth.config2_mid(n=100_000, m=1_000_000)
    _valid(g)
    assert g.num_colors == 16 and q.k == 6
    assert g.m == 1_000_000 + 10 * (q.k - 1)  # the planted paths' arcs
    # Zipf(1.0) colours: colour 0 about twice as common as colour 1
    cnt = np.bincount(g.color, minlength=16)
    assert cnt[0] > 1.6 * cnt[1] > 1.6 * 0.6 * cnt[2]
    assert np.all(np.diff(cnt[:4]) < 0)
    # one colour twice, the rest distinct
    vals, reps = np.unique(q.multiset, return_counts=True)
    assert len(vals) == 5 and sorted(reps.tolist()) == [1, 1, 1, 1, 2]
    # planted paths: distinct vertices, colours equal M, strictly increasing times
    assert len(q.planted) == 10
    arcs = set(zip(g.src.tolist(), g.dst.tolist(), g.time.tolist()))
    for verts, times in q.planted:
        assert len(set(verts)) == q.k
        assert sorted(g.color[verts].tolist()) == sorted(q.multiset.tolist())
        assert all(a < b for a, b in zip(times, times[1:]))
        for i in range(q.k - 1):
            assert (verts[i], verts[i + 1], times[i]) in arcs


def test_config3_batch_recipe():
    items = synth.config3_batch(num_graphs=40)
    assert len(items) == 40
    for g, q in items:
        _valid(g)
        assert 100 <= g.n <= 5000
        assert g.m == 8 * g.n
        assert int(g.time.max()) <= 288
        assert g.num_colors == 12 and 5 <= q.k <= 8


def test_config4_large_recipe_scaled():
    g, q = synth.config4_large(m=1_000_000, n=20_000, k=5, seed=5)
    _valid(g)
    assert g.num_colors == 32 and q.k == 5 and int(g.time.max()) <= 10_000
    cnt = np.bincount(g.color, minlength=32)
    assert cnt.min() > 0.6 * cnt.mean()    # uniform colours


def test_config5_serving_requests():
    g, reqs = synth.config5_serving(n=20_000, m=200_000, requests=2000)
    _valid(g)
    ks = np.array([q.k for q, _ in reqs])
    assert ks.min() == 3 and ks.max() == 10
    assert np.all(np.bincount(ks)[3:] > 150)   # k ~ U{3..10}
    ex = np.mean([e for _, e in reqs])
    assert 0.26 < ex < 0.34                     # 30 % extract
    for q, _ in reqs[:50]:
        assert len(q.multiset) == q.k and int(q.multiset.max()) < 16


def test_tour_and_transit_graphs():
    t = synth.tour_graph(2000, 8, 288, 12, seed=9)
    _valid(t)
    assert t.m == 16000 and int(t.time.max()) <= 288
    g, q = synth.config_transit(n_stops=5000, routes=200, trips=20)
    _valid(g)
    assert q.k == 8 and g.num_colors == 12 and int(g.time.max()) <= 1440
    pairs = set(zip(g.src.tolist(), g.dst.tolist()))
    assert g.m % 20 == 0 and g.m >= 20 * len(pairs)          # every hop repeats once per trip
    assert np.all(g.src != g.dst)                            # a route's stops are distinct


@pytest.mark.parametrize("k,nc", [(4, 8), (8, 12), (10, 16)])
def test_draw_multiset(k, nc):
    ms = synth.draw_multiset(k, nc, seed=k * 31 + nc)
    assert len(ms) == k and ms.dtype == np.uint32
    assert np.all(np.diff(ms.astype(np.int64)) >= 0) and int(ms.max()) < nc
