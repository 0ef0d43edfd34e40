"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle.

GF(2^64) arithmetic is exact, so every comparison is bit-exact: each per-point
sieve sum Q^A, each decision and each extracted path (Lemma 6.5 sieve over
eq. gen-polynomial:3; extraction of Sec. 6.9).
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


def gpu_graph(tm, g, undirected=None):
    und = g.undirected if undirected is None else undirected
    return tm.tmotif_create_graph(g.n, g.src, g.dst, g.time, g.color, g.num_colors, undirected=und)


def both(tm, G, g, k, ms, und=False, **kw):
    d = tm.tmotif_decide(G, k, ms, **kw)
    f, s, pp = oracle.decide(g.n, g.src, g.dst, g.time, g.color, g.num_colors, k, ms, undirected=und, **kw)
    return d, (f, s, pp)


def assert_same(d, o):
    f, s, pp = o
    assert np.array_equal(d.per_point, pp), (d.per_point[:8], pp[:8])
    assert d.sieve_sum == s
    assert d.found == f


def test_device_multiply_bit_exact(tm):
    rng = np.random.default_rng(101)
    n = 1 << 20
    a = rng.integers(0, 2**64, n, dtype=np.uint64)
    b = rng.integers(0, 2**64, n, dtype=np.uint64)
    sp = np.array([0, 1, 2, 1 << 63, 2**64 - 1, 0x1B, 0x8000000000000001, 0xFFFFFFFF, 0xFFFFFFFF00000000],
                  dtype=np.uint64)
    a[:81] = np.repeat(sp, 9)
    b[:81] = np.tile(sp, 9)
    assert np.array_equal(tm.tmotif_gf_mul_batch(a, b), oracle.gf_mul_batch(a, b))


def test_config1_tiny_per_point(tm):
    g, q = synth.config1_tiny()
    G = gpu_graph(tm, g)
    for seed in (q.seed, 2, 3, 12345):
        assert_same(*both(tm, G, g, q.k, q.multiset, seed=seed))


def test_config1_brute_instance_many_seeds(tm):
    g, q = synth.config1_brute()
    G = gpu_graph(tm, g)
    for seed in range(1, 60):
        assert_same(*both(tm, G, g, q.k, q.multiset, seed=seed))


def test_paper_example(tm):
    g = synth.paper_example()
    G = gpu_graph(tm, g)
    for seed in range(1, 10):
        d, o = both(tm, G, g, 3, [0, 0, 0], und=True, seed=seed)
        assert_same(d, o)
        assert d.found
        d, o = both(tm, G, g, 3, [0, 0, 0], und=True, seed=seed, t_max=1)
        assert_same(d, o)
        assert not d.found


def _random_case(rng):
    n = rng.randint(2, 60)
    m = rng.randint(0, 6 * n)
    t_hi = rng.randint(1, 12)
    ncol = rng.randint(1, 5)
    src = np.array([rng.randrange(n) for _ in range(m)], np.uint32)
    dst = np.array([rng.randrange(n) for _ in range(m)], np.uint32)
    time = np.array([rng.randint(1, t_hi) for _ in range(m)], np.uint32)
    color = np.array([rng.randrange(ncol) for _ in range(n)], np.uint32)
    und = rng.random() < 0.3
    g = synth.Graph(n, src, dst, time, color, ncol, und)
    k = rng.randint(2, 7)
    ms = [rng.randrange(ncol) for _ in range(k)]
    kw = {"seed": rng.getrandbits(63)}
    r = rng.random()
    if r < 0.15:
        kw["start"] = rng.randrange(n)
    elif r < 0.3:
        kw["end"] = rng.randrange(n)
    if rng.random() < 0.25:
        kw["t_min"] = rng.randint(0, min(4, t_hi))
        kw["t_max"] = rng.randint(kw["t_min"], t_hi + 1)
    if rng.random() < 0.2:
        kw["repeats"] = rng.randint(2, 3)
    return g, k, ms, kw


def test_random_graphs_and_constraints(tm):
    rng = random.Random(2024)
    for _ in range(120):
        g, k, ms, kw = _random_case(rng)
        G = gpu_graph(tm, g)
        assert_same(*both(tm, G, g, k, ms, und=g.undirected, **kw))
        G.close()


def test_lane_batches_and_point_ranges(tm):
    # k = 7, 8, 9: 128..512 points run as several lane batches; partial ranges
    # (sharding) must equal the matching slice of the full evaluation.
    g = synth.uniform_graph(400, 5000, 60, 6, seed=77)
    G = gpu_graph(tm, g)
    for k in (7, 8, 9):
        ms = [i % 6 for i in range(k)]
        d, o = both(tm, G, g, k, ms, seed=k)
        assert_same(d, o)
        hi = (1 << k) - 3
        sub = tm.tmotif_decide(G, k, ms, seed=k, point_begin=37, point_end=hi)
        assert np.array_equal(sub.per_point, o[2][37:hi])


def test_layer_shapes_give_identical_results(tm):
    # every launch shape the autotuner can pick (arcs per chunk x register
    # bound) gives the same per-point sums; the tuner's pick is one of them
    # (layers of at least 2^22 arc-lanes are tuned)
    g = synth.powerlaw_graph(30000, 400000, 300, 4, seed=71)
    for k, L in ((4, 16), (5, 32), (6, 64), (7, 128)):
        ms = [i % 4 for i in range(k)]
        G = gpu_graph(tm, g)
        assert tm.tmotif_get_layer_shape(G, L) is None
        tuned = tm.tmotif_decide(G, k, ms, seed=9)
        chunk, variant = tm.tmotif_get_layer_shape(G, L)
        variants = {16: (0, 1, 2), 32: (0, 3, 4), 64: (0, 1, 2, 4), 128: (0, 1, 4)}[L]
        assert chunk in (64, 128, 256, 512, 1024) and variant in variants
        if k in (4, 7):
            ref = oracle.decide(g.n, g.src, g.dst, g.time, g.color, g.num_colors, k, ms, seed=9)
            assert_same(tuned, ref)
        for c in (64, 128, 256, 512, 1024):
            for v in variants:
                tm.tmotif_set_layer_shape(G, L, c, v)
                d = tm.tmotif_decide(G, k, ms, seed=9)
                assert np.array_equal(d.per_point, tuned.per_point), (L, c, v)
        with pytest.raises(tm.TmotifError):
            tm.tmotif_set_layer_shape(G, L, 100, 0)
        G.close()


def test_edge_cases(tm):
    # empty edge set, only self-loops, duplicated input edges, absent colours,
    # k larger than the vertex count
    n = 5
    color = np.array([0, 1, 2, 0, 1], np.uint32)
    cases = [
        (np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.uint32)),
        (np.array([1, 2, 3], np.uint32), np.array([1, 2, 3], np.uint32), np.array([1, 2, 3], np.uint32)),
        (np.array([0, 0, 1, 1, 1], np.uint32), np.array([1, 1, 2, 2, 2], np.uint32), np.array([1, 1, 2, 2, 2], np.uint32)),
    ]
    for src, dst, time in cases:
        g = synth.Graph(n, src, dst, time, color, 4, False)
        G = gpu_graph(tm, g)
        for k, ms in ((2, [0, 1]), (3, [0, 1, 2]), (3, [3, 3, 3]), (6, [0, 0, 1, 1, 2, 2])):
            assert_same(*both(tm, G, g, k, ms, seed=5))
        info = tm.tmotif_graph_get_info(G)
        assert info["m_arcs"] == len(oracle.canon(n, src, dst, time)[0])
        G.close()


def test_errors_are_reported(tm):
    g, q = synth.config1_brute()
    G = gpu_graph(tm, g)
    with pytest.raises(tm.TmotifError) as e:
        tm.tmotif_decide(G, 1, [0])
    assert e.value.code == 5
    with pytest.raises(tm.TmotifError) as e:
        tm.tmotif_decide(G, 3, [0, 1, 99])
    assert e.value.code == 1
    with pytest.raises(tm.TmotifError) as e:
        tm.tmotif_decide(G, 3, [0, 1, 2], repeats=0)
    assert e.value.code == 1
    with pytest.raises(tm.TmotifError) as e:
        tm.tmotif_decide(G, 3, [0, 1, 2], start=10**6)
    assert e.value.code == 1
    # the handle stays usable after an error
    assert_same(*both(tm, G, g, q.k, q.multiset, seed=3))


def test_largest_k(tm):
    # k = TMOTIF_KMAX = 20: 2^20 points in 8192 lane batches on a small graph
    # with a planted 20-vertex path; three ragged ranges of points against the
    # oracle; k = 21 is refused
    g = synth.uniform_graph(60, 500, 40, 4, seed=55)
    ms = [i % 4 for i in range(20)]
    g2, _ = synth.plant_paths(g, ms, 1, seed=56, t_max=40)
    G = gpu_graph(tm, g2)
    d = tm.tmotif_decide(G, 20, ms, seed=8)
    assert d.found
    for lo, hi in ((0, 300), (524_000, 524_611), ((1 << 20) - 257, 1 << 20)):
        _, _, pp = oracle.decide(g2.n, g2.src, g2.dst, g2.time, g2.color, g2.num_colors, 20, ms, seed=8,
                                 point_begin=lo, point_end=hi)
        assert np.array_equal(d.per_point[lo:hi], pp), (lo, hi)
    with pytest.raises(tm.TmotifError) as e:
        tm.tmotif_decide(G, 21, ms + [0])
    assert e.value.code == 5
    G.close()


def test_invalid_graphs_are_rejected(tm):
    n = 4
    src = np.array([0, 1, 2], np.uint32)
    dst = np.array([1, 2, 3], np.uint32)
    time = np.array([1, 2, 3], np.uint32)
    color = np.zeros(n, np.uint32)
    bad = [
        (src, dst, np.array([1, 0, 3], np.uint32), color, 1, "timestamp"),
        (src, np.array([1, 2, 9], np.uint32), time, color, 1, "vertex"),
        (src, dst, time, np.array([0, 0, 5, 0], np.uint32), 2, "color"),
    ]
    for s, d, t, c, nc, word in bad:
        with pytest.raises(tm.TmotifError) as e:
            tm.tmotif_create_graph(n, s, d, t, c, nc)
        assert e.value.code == 1 and word in str(e.value)
    G = tm.tmotif_create_graph(n, src, dst, time, color, 1)  # the library is still usable
    assert tm.tmotif_graph_get_info(G)["m_arcs"] == 3


def test_device_graph_build_matches_canonical_set(tm):
    # radix-sorted device build == the oracle's canonical arc set, directed and
    # undirected, with duplicates, self-loops and wide ids/timestamps
    rng = np.random.default_rng(5)
    for n, m, tmax, und in ((50, 400, 9, False), (50, 400, 9, True), (3_000_000, 20000, 3_000_000, False),
                            (70000, 50000, 1, True)):
        src = rng.integers(0, n, m, dtype=np.uint32)
        dst = rng.integers(0, n, m, dtype=np.uint32)
        time = rng.integers(1, tmax + 1, m, dtype=np.uint32)
        src[: m // 10] = dst[: m // 10]                      # self-loops
        src[m // 10: m // 5] = src[m // 5: 3 * m // 10]      # duplicates
        dst[m // 10: m // 5] = dst[m // 5: 3 * m // 10]
        time[m // 10: m // 5] = time[m // 5: 3 * m // 10]
        G = tm.tmotif_create_graph(n, src, dst, time, np.zeros(n, np.uint32), 1, undirected=und)
        info = tm.tmotif_graph_get_info(G)
        cs, cd, ct = oracle.canon(n, src, dst, time, und)
        assert info["m_arcs"] == len(cs)
        assert info["self_loops"] == int(np.sum(src == dst))
        G.close()


def test_wide_arc_keys_build_and_sieve(tm):
    # 17-bit vertex ids with timestamps up to 2^32 - 1: dst | time | src needs
    # 66 bits, so the device build sorts (time | src, dst) pairs instead of one
    # key; the arc set, decisions, extraction and optimum time must still
    # equal the oracle's
    rng = np.random.default_rng(17)
    n, m = 70000, 120000
    src = rng.integers(0, n, m, dtype=np.uint32)
    dst = rng.integers(0, n, m, dtype=np.uint32)
    time = rng.integers(1, 2**32, m, dtype=np.uint64).astype(np.uint32)
    time[: m // 3] = rng.integers(2**31, 2**31 + 40, m // 3).astype(np.uint32)  # many time ties
    time[-5:] = 2**32 - 1
    src[: m // 20] = dst[: m // 20]                          # self-loops
    src[m // 20: m // 10] = src[m // 10: 3 * m // 20]        # duplicates
    dst[m // 20: m // 10] = dst[m // 10: 3 * m // 20]
    time[m // 20: m // 10] = time[m // 10: 3 * m // 20]
    color = rng.integers(0, 3, n, dtype=np.uint32)
    for und in (False, True):
        G = tm.tmotif_create_graph(n, src, dst, time, color, 3, undirected=und)
        info = tm.tmotif_graph_get_info(G)
        cs, cd, ct = oracle.canon(n, src, dst, time, und)
        assert info["m_arcs"] == len(cs)
        assert info["self_loops"] == int(np.sum(src == dst))
        for k, ms, kw in ((3, [0, 1, 2], {}), (4, [0, 0, 1, 2], {"t_min": 2**31, "t_max": 2**31 + 30}),
                          (4, [1, 2, 2, 0], {"end": int(cd[7])})):
            d = tm.tmotif_decide(G, k, ms, seed=3, **kw)
            o = oracle.decide(n, src, dst, time, color, 3, k, ms, undirected=und, seed=3, **kw)
            assert_same(d, o)
            f, v, t = tm.tmotif_extract(G, k, ms, seed=3, method="halving", **kw)
            fo, vo, to, _ = oracle.extract(n, src, dst, time, color, 3, k, ms, undirected=und, seed=3, **kw)
            assert f == fo and np.array_equal(v, vo) and np.array_equal(t, to)
        t_opt = tm.tmotif_optimum_time(G, 4, [0, 1, 2, 0], seed=5)
        assert t_opt == oracle.optimum_time(n, src, dst, time, color, 3, 4, [0, 1, 2, 0], undirected=und, seed=5)
        G.close()


def test_arc_filter_over_ragged_tiles(tm):
    # the per-query arc filter works on 4096-arc tiles with a keep mask of one
    # bit per arc: graphs of several tiles and a ragged last tile, with time
    # windows, EC tuples, masked (extraction) and preprocessed subgraphs,
    # must give the oracle's per-point sums and paths
    for m, seed in ((4096 * 3 + 123, 41), (4096 * 5, 42), (4095, 43)):
        g = synth.uniform_graph(2500, m, 40, 4, seed=seed)
        G = gpu_graph(tm, g)
        for k, ms, kw in ((4, [0, 1, 2, 3], {}), (5, [0, 0, 1, 2, 3], {"t_min": 5, "t_max": 33}),
                          (3, [1, 2, 2], {"t_max": 20, "start": 7})):
            assert_same(*both(tm, G, g, k, ms, **kw))
            f, v, t = tm.tmotif_extract(G, k, ms, method="halving", **kw)
            fo, vo, to, _ = oracle.extract(g.n, g.src, g.dst, g.time, g.color, g.num_colors, k, ms, **kw)
            assert f == fo and np.array_equal(v, vo) and np.array_equal(t, to)
        d, o = _ec_both(tm, G, g, 4, [0, 1, 2, 3], [3, 9, 17])
        assert_same(d, o)
        d = tm.tmotif_decide(G, 4, [0, 1, 2, 3], seed=5, preprocess=True)
        fo, so, po, _ = oracle.decide_preprocessed(g.n, g.src, g.dst, g.time, g.color, g.num_colors, 4, [0, 1, 2, 3],
                                                  seed=5)
        assert_same(d, (fo, so, po))
        G.close()


def test_arc_filter_by_vertex_and_by_tiles(tm):
    # the filter's first pass goes by flagged destination (one warp walks each
    # in-segment) when such arcs are under 30 % of all (from the graph's
    # colour-pair counts), else by tiles of arcs.  One graph, queries on both
    # sides of that switch, with an in-segment spanning several tiles, empty
    # vertices between segments, arcs into the last vertex, a window, an EC
    # tuple, and the subgraphs of extraction and preprocessing: the oracle's
    # sums and paths
    rng = np.random.default_rng(77)
    n, nc = 60000, 12
    dst = np.concatenate([np.full(9000, 50), rng.integers(0, 100, 5000), rng.integers(100, n, 6000),
                          np.full(40, n - 1)]).astype(np.uint32)
    src = rng.integers(0, n, len(dst)).astype(np.uint32)
    time = rng.integers(1, 61, len(dst)).astype(np.uint32)
    color = rng.integers(0, nc, n).astype(np.uint32)
    g = synth.Graph(n, src, dst, time, color, nc, False, "filter-passes")
    hub = int(color[50])
    others = [c for c in range(nc) if c != hub]

    def share(ms):
        return np.isin(color[dst], ms).mean()

    few = [others[0], others[1], others[1]]              # hub's colour out: few flagged destinations
    many = [hub, others[0], others[2], others[3]]        # hub's colour in: most arcs
    assert share(few) < 0.2 and share(many) > 0.4
    G = gpu_graph(tm, g)
    for k, ms, kw in ((3, few, {}), (4, many, {}), (3, few, {"t_min": 10, "t_max": 50}),
                      (3, many[:3], {"t_max": 40, "end": 50}), (3, [others[4], others[4], others[5]], {"start": n - 1})):
        assert_same(*both(tm, G, g, k, ms, **kw))
        f, v, t = tm.tmotif_extract(G, k, ms, method="halving", **kw)
        fo, vo, to, _ = oracle.extract(g.n, g.src, g.dst, g.time, g.color, g.num_colors, k, ms, **kw)
        assert f == fo and np.array_equal(v, vo) and np.array_equal(t, to)
    assert_same(*_ec_both(tm, G, g, 3, few, [4, 20]))
    d = tm.tmotif_decide(G, 3, few, seed=9, preprocess=True)
    fo, so, po, _ = oracle.decide_preprocessed(g.n, g.src, g.dst, g.time, g.color, g.num_colors, 3, few, seed=9)
    assert_same(d, (fo, so, po))
    G.close()


def test_coefficients_by_multiplier_table(tm):
    # lists of at least 2^20 vertex-lanes at up to 32 lanes take x_u^A by
    # multiplier table: tables of W_d^A for 16, 8 or 4 lanes per block
    # (k <= 6, 7..12, 13..20), the active vertices grouped by colour, repeated
    # colours (two slots); every per-point sum equals the oracle's (and the
    # 64-lane case, one warp per vertex, too); an extraction through such lists
    # returns a valid path
    g = synth.uniform_graph(100000, 300000, 50, 4, seed=91)
    G = gpu_graph(tm, g)
    for k, ms, kw in ((4, [0, 1, 2, 3], {}), (5, [0, 1, 1, 2, 3], {}),
                      (7, [0, 0, 1, 1, 2, 3, 3], {"point_begin": 0, "point_end": 32}),
                      (13, [0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3, 0], {"point_begin": 4000, "point_end": 4032}),
                      (7, [0, 0, 1, 1, 2, 3, 3], {"point_begin": 64, "point_end": 128})):
        assert_same(*both(tm, G, g, k, ms, **kw))
    ms = [0, 1, 1, 2, 3]
    f, v, t = tm.tmotif_extract(G, 5, ms, method="halving")
    assert f
    arcs = set(zip(g.src.tolist(), g.dst.tolist(), g.time.tolist()))
    assert len(set(v.tolist())) == 5 and sorted(g.color[v].tolist()) == sorted(ms)
    for r in range(4):
        assert (int(v[r]), int(v[r + 1]), int(t[r])) in arcs
        assert r == 0 or t[r] > t[r - 1]
    G.close()


# ---------------------------------------------------------------------------
# Extraction (Sec. 6.9): same deterministic procedure -> the same path
# ---------------------------------------------------------------------------
def test_extraction_matches_oracle(tm):
    g, q = synth.config1_tiny()
    G = gpu_graph(tm, g)
    for seed in (1, 2, 3):
        f, v, t = tm.tmotif_extract(G, q.k, q.multiset, seed=seed, method="halving")
        fo, vo, to, _ = oracle.extract(g.n, g.src, g.dst, g.time, g.color, g.num_colors, q.k, q.multiset, seed=seed)
        assert f == fo and np.array_equal(v, vo) and np.array_equal(t, to)
    rng = random.Random(99)
    for _ in range(30):
        g, k, ms, kw = _random_case(rng)
        kw.pop("repeats", None)
        G = gpu_graph(tm, g)
        f, v, t = tm.tmotif_extract(G, k, ms, method="halving", **kw)
        fo, vo, to, _ = oracle.extract(g.n, g.src, g.dst, g.time, g.color, g.num_colors, k, ms,
                                       undirected=g.undirected, **kw)
        assert f == fo
        if f:
            assert np.array_equal(v, vo) and np.array_equal(t, to)
        G.close()


def test_localized_extraction_matches_oracle(tm):
    g, q = synth.config1_tiny()
    G = gpu_graph(tm, g)
    for seed in (1, 2, 3):
        f, v, t = tm.tmotif_extract(G, q.k, q.multiset, seed=seed)
        fo, vo, to = oracle.extract_localized(g.n, g.src, g.dst, g.time, g.color, g.num_colors, q.k, q.multiset,
                                              seed=seed)
        assert f and fo and np.array_equal(v, vo) and np.array_equal(t, to)
    rng = random.Random(123)
    for _ in range(40):
        g, k, ms, kw = _random_case(rng)
        G = gpu_graph(tm, g)
        f, v, t = tm.tmotif_extract(G, k, ms, **kw)
        fo, vo, to = oracle.extract_localized(g.n, g.src, g.dst, g.time, g.color, g.num_colors, k, ms,
                                              undirected=g.undirected, **kw)
        assert f == fo
        if f:
            assert np.array_equal(v, vo) and np.array_equal(t, to)
        G.close()


def test_optimum_time_and_optimum_extraction(tm):
    rng = random.Random(77)
    for trial in range(25):
        g, k, ms, kw = _random_case(rng)
        kw = {"seed": kw["seed"]}
        G = gpu_graph(tm, g)
        f, t = tm.tmotif_optimum_time(G, k, ms, **kw)
        fo, to = oracle.optimum_time(g.n, g.src, g.dst, g.time, g.color, g.num_colors, k, ms,
                                     undirected=g.undirected, **kw)
        assert f == fo and (not f or t == to)
        if f:
            ff, v, tt = tm.tmotif_extract(G, k, ms, optimum=True, **kw)
            assert ff and int(tt.max()) == t  # the extracted path ends at the optimum time
            fe, ve, te = oracle.extract_localized(g.n, g.src, g.dst, g.time, g.color, g.num_colors, k, ms,
                                                  undirected=g.undirected, t_max=t, **kw)
            assert np.array_equal(v, ve) and np.array_equal(tt, te)
        G.close()


def test_vertex_localized_sieve_matches_oracle(tm):
    rng = random.Random(321)
    cases = [synth.config1_brute(), synth.config1_tiny()]
    for g, q in cases:
        G = gpu_graph(tm, g)
        d, pv = tm.tmotif_localize(G, q.k, q.multiset, seed=9)
        cs, cd, ct = oracle.canon(g.n, g.src, g.dst, g.time)
        pb = oracle.Problem(g.n, cs, cd, ct, g.color, g.num_colors, q.k, q.multiset)
        arc = oracle.arc_sums(pb, oracle.query_seed(9, 0))
        want = np.zeros(g.n, np.uint64)
        np.bitwise_xor.at(want, cd.astype(np.int64), arc)
        assert np.array_equal(pv, want)
        assert d.sieve_sum == int(np.bitwise_xor.reduce(want))


def test_arc_localisation_in_every_layer_shape(tm):
    # arc-localised sums (per-vertex Q_u, localised extraction) in every
    # pinned launch shape at 32, 64 and 128 lanes, including two 64-lane teams
    # per chunk at 128 lanes, whose teams add to the same arcs, and the staged
    # form (variant 4)
    g = synth.powerlaw_graph(4000, 60000, 120, 5, seed=23)
    cs, cd, ct = oracle.canon(g.n, g.src, g.dst, g.time)
    for k, L, variants in ((5, 32, (0, 3, 4)), (6, 64, (0, 1, 2, 4)), (7, 128, (0, 1, 4))):
        ms = [i % 5 for i in range(k)]
        pb = oracle.Problem(g.n, cs, cd, ct, g.color, g.num_colors, k, ms)
        arc = oracle.arc_sums(pb, oracle.query_seed(4, 0))
        want = np.zeros(g.n, np.uint64)
        np.bitwise_xor.at(want, cd.astype(np.int64), arc)
        fo, vo, to = oracle.extract_localized(g.n, g.src, g.dst, g.time, g.color, g.num_colors, k, ms, seed=4)
        G = gpu_graph(tm, g)
        for v in variants:
            for c in (64, 256, 1024):
                tm.tmotif_set_layer_shape(G, L, c, v)
                d, pv = tm.tmotif_localize(G, k, ms, seed=4)
                assert np.array_equal(pv, want), (L, c, v)
                f, verts, times = tm.tmotif_extract(G, k, ms, seed=4)
                assert f == fo and np.array_equal(verts, vo) and np.array_equal(times, to), (L, c, v)
        G.close()


# ---------------------------------------------------------------------------
# EC-PathMotif (Sec. 7.3): the path's arc times are a given tuple T
# ---------------------------------------------------------------------------
def _ec_both(tm, G, g, k, ms, T, **kw):
    d = tm.tmotif_decide(G, k, ms, timestamps=T, **kw)
    o = oracle.decide_ec(g.n, g.src, g.dst, g.time, g.color, g.num_colors, k, ms, T, undirected=g.undirected,
                         **kw)
    return d, o


def test_ec_pathmotif_matches_oracle(tm):
    rng = random.Random(606)
    cases = 0
    for i in range(150):
        if i % 2:
            g, k, ms, kw = _random_case(rng)
        else:  # dense: many EC walks
            n = rng.randint(8, 40)
            g = synth.uniform_graph(n, rng.randint(5 * n, 30 * n), 8, 3, seed=900 + i)
            g.undirected = rng.random() < 0.3
            k = rng.randint(2, 6)
            ms = [rng.randrange(3) for _ in range(k)]
            kw = {"seed": rng.getrandbits(63)}
        t_hi = int(g.time.max()) if len(g.time) else 1
        if t_hi < k - 1:
            continue
        T = sorted(rng.sample(range(1, t_hi + 1), k - 1))
        G = gpu_graph(tm, g)
        assert_same(*_ec_both(tm, G, g, k, ms, T, **kw))
        G.close()
        cases += 1
    assert cases > 100


def test_ec_pathmotif_planted_tuple_and_extraction(tm):
    # T taken from a path that exists: EC says YES, and the extracted path
    # (both procedures) has exactly the times T
    g, q = synth.config1_tiny()
    G = gpu_graph(tm, g)
    f, v, t, _ = oracle.extract(g.n, g.src, g.dst, g.time, g.color, g.num_colors, q.k, q.multiset, seed=q.seed)
    assert f
    T = [int(x) for x in t]
    arcs = set(zip(g.src.tolist(), g.dst.tolist(), g.time.tolist()))
    for seed in (1, 2, 3):
        d, o = _ec_both(tm, G, g, q.k, q.multiset, T, seed=seed)
        assert_same(d, o)
        assert d.found
        for method in ("localized", "halving"):
            fe, ve, te = tm.tmotif_extract(G, q.k, q.multiset, seed=seed, timestamps=T, method=method)
            assert fe and te.tolist() == T
            assert len(set(ve.tolist())) == q.k
            assert sorted(g.color[ve].tolist()) == sorted(q.multiset.tolist())
            assert all((int(ve[r]), int(ve[r + 1]), T[r]) in arcs for r in range(q.k - 1))
    # a tuple with the order of two times swapped is rejected; one shifted
    # past every arc finds nothing
    with pytest.raises(tm.TmotifError) as e:
        tm.tmotif_decide(G, q.k, q.multiset, timestamps=[T[1], T[0]] + T[2:])
    assert e.value.code == 1
    late = [1000 + i for i in range(q.k - 1)]
    d, o = _ec_both(tm, G, g, q.k, q.multiset, late, seed=4)
    assert_same(d, o)
    assert not d.found and d.sieve_sum == 0
    G.close()


# ---------------------------------------------------------------------------
# Full size (the benchmark workload): sampled points against the oracle
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def cfg2(tm):
    g, q = synth.config2_mid()
    return g, q, gpu_graph(tm, g)


def test_config2_full_size_sampled_points(tm, cfg2):
    g, q, G = cfg2
    d = tm.tmotif_decide(G, q.k, q.multiset, seed=q.seed)
    assert d.found  # planted paths
    # a ragged sample of the 64 points, each computed by the oracle on its own
    # (oracle calls run concurrently in threads; ctypes releases the GIL)
    import concurrent.futures as cf

    ranges = ((5, 6), (33, 35), (62, 64))

    def run(r):
        lo, hi = r
        return oracle.decide(g.n, g.src, g.dst, g.time, g.color, g.num_colors, q.k, q.multiset, seed=q.seed,
                             point_begin=lo, point_end=hi, nthreads=hi - lo)[2]

    with cf.ThreadPoolExecutor(len(ranges)) as ex:
        for (lo, hi), pp in zip(ranges, ex.map(run, ranges)):
            assert np.array_equal(d.per_point[lo:hi], pp)


def test_config2_full_size_extraction_is_valid(tm, cfg2):
    g, q, G = cfg2
    f, v, t = tm.tmotif_extract(G, q.k, q.multiset, seed=q.seed)
    assert f
    arcs = set(zip(g.src.tolist(), g.dst.tolist(), g.time.tolist()))
    assert len(set(v.tolist())) == q.k
    assert sorted(g.color[v].tolist()) == sorted(q.multiset.tolist())
    for r in range(q.k - 1):
        assert (int(v[r]), int(v[r + 1]), int(t[r])) in arcs
        if r:
            assert t[r] > t[r - 1]
