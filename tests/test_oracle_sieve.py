"""Pins for the oracle's sieve, decision and extraction.

Each check compares the oracle with something fixed independently of it:
the polynomials printed in the paper's worked example (Fig.
tempwalk-encoding-demo, Sec. 6.4), direct enumeration of temporal walks
(Sec. 6.3), the determinant form of the sieve sum in characteristic 2
(Lemmas 6.3/6.5), cancellation of walks that repeat a vertex (Lemma 6.1),
exhaustive temporal DFS (the Sec. 9.1 baseline) and the k-path reduction of
Lemma 5.1.
"""
import itertools
import os
import random
import re

import numpy as np
import pytest

import oracle
import synth

ANY = oracle.ANY
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_example_terms.txt")


def rand_graph(rng, n_lo=3, n_hi=9, t_hi=6, colors=3, undirected=False):
    n = rng.randint(n_lo, n_hi)
    m = rng.randint(n, 4 * n)
    src = [rng.randrange(n) for _ in range(m)]
    dst = [rng.randrange(n) for _ in range(m)]
    time = [rng.randint(1, t_hi) for _ in range(m)]
    color = [rng.randrange(colors) for _ in range(n)]
    return n, src, dst, time, color, undirected


def problem(n, src, dst, time, color, undirected, k, ms, num_colors=3, **kw):
    cs, cd, ct = oracle.canon(n, src, dst, time, undirected)
    return oracle.Problem(n, cs, cd, ct, color, num_colors, k, ms, **kw)


# ---------------------------------------------------------------------------
# The paper's worked example
# ---------------------------------------------------------------------------
def _eval_term(term, qs, x):
    val = 1
    for f in term.split("*"):
        f = f.strip()
        mx = re.fullmatch(r"x([123])", f)
        my = re.fullmatch(r"y\[v([123])v([123]),(\d+),(\d+)\]", f)
        if mx:
            val = oracle.gf_mul(val, x[int(mx.group(1)) - 1])
        elif my:
            a, b, p, t = (int(g) for g in my.groups())
            # y_{ab,p,t}: the walk arrives at a from b, i.e. arc b -> a.
            val = oracle.gf_mul(val, oracle.coef_y(qs, b - 1, a - 1, t, p))
        else:
            raise AssertionError(f"bad factor {f!r}")
    return val


def test_paper_example_polynomials(oracle_mod):
    g = synth.paper_example()
    k, ms = 3, [0, 0, 0]
    pb = problem(g.n, g.src, g.dst, g.time, g.color, True, k, ms, num_colors=1)
    lines = [ln for ln in open(GOLDEN) if ln.startswith("P ")]
    assert len(lines) == 18
    for seed in (1, 2, 3):
        qs = oracle.query_seed(seed, 0)
        for point in (1, 5, 7):
            table, _ = oracle.literal_table(pb, qs, point, T=2)
            x = [oracle.vertex_x(qs, k, ms, 1, 0, u, point) for u in range(3)]
            for ln in lines:
                lhs, rhs = ln[2:].split("=")
                v, ell, i = lhs.split()
                want = 0
                if rhs.strip() != "0":
                    for term in rhs.split("+"):
                        want ^= _eval_term(term, qs, x)
                assert int(table[int(v[1]) - 1, int(ell), int(i)]) == want, ln


def test_paper_example_decisions(oracle_mod):
    g = synth.paper_example()
    args = (g.n, g.src, g.dst, g.time, g.color, 1)
    # k = 3: exactly the two bold paths v1->v2->v3 and v3->v2->v1, times (1,2).
    pb = problem(*args[:5], True, 3, [0, 0, 0], num_colors=1)
    count, first_v, first_t = oracle.count_paths(pb)
    assert count == 2
    assert list(first_v) == [0, 1, 2] and list(first_t) == [1, 2]
    for seed in range(1, 40):
        assert oracle.decide(*args, 3, [0, 0, 0], undirected=True, seed=seed)[0]
        # k = 4 cannot be met by 3 vertices; restricting to time 1 empties
        # P_{.,3,1} (panel (e)).
        f4, q4, _ = oracle.decide(*args, 4, [0, 0, 0, 0], undirected=True, seed=seed)
        assert not f4 and q4 == 0
        f1, q1, _ = oracle.decide(*args, 3, [0, 0, 0], undirected=True, seed=seed, t_max=1)
        assert not f1 and q1 == 0


# ---------------------------------------------------------------------------
# Recurrence == walk enumeration == literal table == determinant identity
# ---------------------------------------------------------------------------
def _constraints(rng, n, t_hi):
    kw = {}
    r = rng.random()
    if r < 0.2:
        kw["start"] = rng.randrange(n)
    elif r < 0.4:
        kw["end"] = rng.randrange(n)
    if rng.random() < 0.3:
        kw["t_min"] = rng.randint(1, 3)
        kw["t_max"] = rng.randint(kw["t_min"], t_hi)
    if rng.random() < 0.3:
        kw["alive"] = [rng.random() < 0.8 for _ in range(n)]
    return kw


@pytest.mark.parametrize("trial", range(40))
def test_dp_equals_walk_enumeration(oracle_mod, trial):
    rng = random.Random(1000 + trial)
    n, src, dst, time, color, _ = rand_graph(rng)
    und = trial % 3 == 0
    k = rng.randint(2, 5)
    ms = [rng.randrange(3) for _ in range(k)]
    kw = _constraints(rng, n, 6)
    pb = problem(n, src, dst, time, color, und, k, ms, **kw)
    qs = oracle.query_seed(rng.getrandbits(63), 0)
    dp = oracle.sieve_points(pb, qs)
    bf, nwalks = oracle.brute_points(pb, qs)
    assert np.array_equal(dp, bf)
    qdet, nw2 = oracle.brute_det(pb, qs)
    assert nw2 == nwalks
    assert int(np.bitwise_xor.reduce(dp)) == qdet
    for point in (1, (1 << k) - 1):
        _, ql = oracle.literal_table(pb, qs, point, T=6)
        assert ql == int(dp[point])


def test_dp_equals_enumeration_on_config1_brute_instance(oracle_mod):
    g, q = synth.config1_brute()
    for seed in range(1, 6):
        pb = problem(g.n, g.src, g.dst, g.time, g.color, False, q.k, q.multiset, num_colors=g.num_colors)
        qs = oracle.query_seed(seed, 0)
        dp = oracle.sieve_points(pb, qs)
        bf, nwalks = oracle.brute_points(pb, qs)
        assert nwalks > 0
        assert np.array_equal(dp, bf)
        assert int(np.bitwise_xor.reduce(dp)) == oracle.brute_det(pb, qs)[0]


# ---------------------------------------------------------------------------
# Cancellation and one-sidedness
# ---------------------------------------------------------------------------
def test_repeated_vertex_walk_cancels(oracle_mod):
    # a->b at 1, b->a at 2: the only 3-vertex walk is a,b,a (Lemma 6.1).
    n, src, dst, time = 2, [0, 1], [1, 0], [1, 2]
    color = [0, 1]
    pb = problem(n, src, dst, time, color, False, 3, [0, 1, 0], num_colors=2)
    _, nwalks = oracle.brute_points(pb, oracle.query_seed(1, 0))
    assert nwalks == 1
    for seed in range(1, 200):
        f, q, pp = oracle.decide(n, src, dst, time, color, 2, 3, [0, 1, 0], seed=seed)
        assert not f and q == 0
        assert np.any(pp != 0)  # individual points are nonzero; only the sum cancels


def test_duplicate_arc_cancels_without_dedupe(oracle_mod):
    # Identical arcs carry the same y and would cancel in characteristic 2;
    # canon() keeps one copy (E^tau is a set).
    n, src, dst, time, color = 3, [0, 1], [1, 2], [1, 2], [0, 1, 2]
    qs = oracle.query_seed(9, 0)
    dup = oracle.Problem(n, [0, 0, 1], [1, 1, 2], [1, 1, 2], color, 3, 3, [0, 1, 2])
    one = oracle.Problem(n, [1], [2], [2], color, 3, 3, [0, 1, 2])
    assert np.array_equal(oracle.sieve_points(dup, qs), oracle.sieve_points(one, qs))
    cs, cd, ct = oracle.canon(n, [0, 0, 1, 1], [1, 1, 2, 1], [1, 1, 2, 5])
    assert list(zip(cs, cd, ct)) == [(0, 1, 1), (1, 2, 2)]
    f, q, _ = oracle.decide(n, [0, 0, 1], [1, 1, 2], [1, 1, 2], color, 3, 3, [0, 1, 2], seed=3)
    assert f and q != 0


def test_equal_times_are_not_consecutive(oracle_mod):
    # Strictly increasing times (Sec. 4): a->b and b->c both at time 4 form no path.
    f, q, _ = oracle.decide(3, [0, 1], [1, 2], [4, 4], [0, 1, 2], 3, 3, [0, 1, 2], seed=5)
    assert not f and q == 0
    f, q, _ = oracle.decide(3, [0, 1], [1, 2], [4, 5], [0, 1, 2], 3, 3, [0, 1, 2], seed=5)
    assert f


@pytest.mark.parametrize("trial", range(60))
def test_decision_equals_exhaustive_dfs(oracle_mod, trial):
    rng = random.Random(5000 + trial)
    n, src, dst, time, color, _ = rand_graph(rng, n_hi=10, t_hi=5)
    und = trial % 4 == 0
    k = rng.randint(2, 5)
    ms = [rng.randrange(3) for _ in range(k)]
    kw = _constraints(rng, n, 5)
    pb = problem(n, src, dst, time, color, und, k, ms, **kw)
    truth = oracle.count_paths(pb, limit=1)[0] > 0
    for s in range(8):
        f, q, _ = oracle.decide(n, src, dst, time, color, 3, k, ms, undirected=und, seed=trial * 100 + s, **kw)
        assert f == truth
        if not truth:
            assert q == 0


def test_decision_many_seeds_config1_brute(oracle_mod):
    g, q = synth.config1_brute()
    pb = problem(g.n, g.src, g.dst, g.time, g.color, False, q.k, q.multiset, num_colors=g.num_colors)
    truth = oracle.count_paths(pb, limit=1)[0] > 0
    ms_no = [7, 7, 7, 7]
    pb_no = problem(g.n, g.src, g.dst, g.time, g.color, False, 4, ms_no, num_colors=g.num_colors)
    truth_no = oracle.count_paths(pb_no, limit=1)[0] > 0
    for seed in range(1, 1001):
        f, _, _ = oracle.decide(g.n, g.src, g.dst, g.time, g.color, g.num_colors, q.k, q.multiset, seed=seed)
        assert f == truth
    for seed in range(1, 201):
        f, qq, _ = oracle.decide(g.n, g.src, g.dst, g.time, g.color, g.num_colors, 4, ms_no, seed=seed)
        assert f == truth_no
        if not truth_no:
            assert qq == 0


def _static_kpath(n, edges, k):
    adj = {u: set() for u in range(n)}
    for a, b in edges:
        if a != b:
            adj[a].add(b)
    for start in range(n):
        stack = [(start, (start,))]
        while stack:
            u, path = stack.pop()
            if len(path) == k:
                return True
            for v in adj[u]:
                if v not in path:
                    stack.append((v, path + (v,)))
    return False


@pytest.mark.parametrize("trial", range(20))
def test_ktemppath_reduction(oracle_mod, trial):
    # Lemma 5.1: a static graph has a k-path iff the temporal graph with every
    # edge present at times 1..k-1 has a temporal path on k vertices; with a
    # single colour, PathMotif with M = {1^k} is k-TempPath.
    rng = random.Random(9000 + trial)
    n = rng.randint(4, 8)
    edges = [(rng.randrange(n), rng.randrange(n)) for _ in range(rng.randint(3, 10))]
    k = rng.randint(2, 5)
    src, dst, time = [], [], []
    for a, b in edges:
        for t in range(1, k):
            src.append(a); dst.append(b); time.append(t)
    color = [0] * n
    f, _, _ = oracle.decide(n, src, dst, time, color, 1, k, [0] * k, seed=trial + 1)
    assert f == _static_kpath(n, edges, k)


def test_multiset_order_does_not_matter(oracle_mod):
    g, q = synth.config1_brute()
    base = oracle.decide(g.n, g.src, g.dst, g.time, g.color, g.num_colors, q.k, q.multiset, seed=4)
    perm = list(reversed(list(q.multiset)))
    other = oracle.decide(g.n, g.src, g.dst, g.time, g.color, g.num_colors, q.k, perm, seed=4)
    assert base[1] == other[1] and np.array_equal(base[2], other[2])


def test_point_range_matches_full(oracle_mod):
    g, q = synth.config1_brute()
    full = oracle.decide(g.n, g.src, g.dst, g.time, g.color, g.num_colors, q.k, q.multiset, seed=8)[2]
    part = oracle.decide(g.n, g.src, g.dst, g.time, g.color, g.num_colors, q.k, q.multiset, seed=8,
                         point_begin=3, point_end=11)[2]
    assert np.array_equal(full[3:11], part)


# ---------------------------------------------------------------------------
# Extraction (Sec. 6.9)
# ---------------------------------------------------------------------------
def verify_path(n, src, dst, time, color, undirected, k, ms, verts, times, start=ANY, end=ANY, t_min=0, t_max=0):
    arcs = set(zip(src, dst, time))
    if undirected:
        arcs |= set(zip(dst, src, time))
    assert len(verts) == k and len(set(int(v) for v in verts)) == k
    assert sorted(int(color[v]) for v in verts) == sorted(int(c) for c in ms)
    for r in range(k - 1):
        assert (int(verts[r]), int(verts[r + 1]), int(times[r])) in arcs
        if r:
            assert times[r] > times[r - 1]
        assert times[r] >= t_min and (t_max == 0 or times[r] <= t_max)
    if start != ANY:
        assert verts[0] == start
    if end != ANY:
        assert verts[-1] == end


@pytest.mark.parametrize("trial", range(25))
def test_extraction_returns_valid_path(oracle_mod, trial):
    rng = random.Random(7000 + trial)
    n, src, dst, time, color, _ = rand_graph(rng, n_lo=5, n_hi=12, t_hi=6)
    und = trial % 3 == 0
    k = rng.randint(2, 4)
    ms = [rng.randrange(3) for _ in range(k)]
    kw = {}
    if trial % 5 == 1:
        kw["t_max"] = 4
    pb = problem(n, src, dst, time, color, und, k, ms, **kw)
    truth = oracle.count_paths(pb, limit=1)[0] > 0
    found, verts, times, probes = oracle.extract(n, src, dst, time, color, 3, k, ms, undirected=und,
                                                 seed=trial + 3, **kw)
    assert found == truth
    if found:
        verify_path(n, src, dst, time, color, und, k, ms, verts, times, **kw)
        assert probes >= 1


def test_extraction_on_config1(oracle_mod):
    g, q = synth.config1_tiny()
    found, verts, times, probes = oracle.extract(g.n, g.src, g.dst, g.time, g.color, g.num_colors, q.k,
                                                 q.multiset, seed=q.seed)
    assert found
    verify_path(g.n, g.src, g.dst, g.time, g.color, False, q.k, q.multiset, verts, times)
    # O(k log n) probes by halving, far fewer than n
    assert probes < 200


def test_time_window_bounds_are_inclusive(oracle_mod):
    # Path 0 -(3)-> 1 -(7)-> 2: the window [t_min, t_max] keeps arcs with
    # t_min <= t <= t_max (the optimum-timestamp search of Sec. 6.8 asks for
    # walks ending at latest time t').
    n, src, dst, time, color = 3, [0, 1], [1, 2], [3, 7], [0, 1, 2]
    for seed in range(1, 30):
        dec = lambda **kw: oracle.decide(n, src, dst, time, color, 3, 3, [0, 1, 2], seed=seed, **kw)[0]
        assert dec(t_min=3, t_max=7)
        assert not dec(t_min=3, t_max=6)
        assert not dec(t_min=4, t_max=7)
        assert dec(t_max=7) and not dec(t_max=6)
        assert dec(t_min=3) and not dec(t_min=4)


# ---------------------------------------------------------------------------
# Localised sieve and extraction by localisation (Sec. 6.7, Sec. 6.9)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("trial", range(30))
def test_arc_sums_equal_walk_enumeration(oracle_mod, trial):
    rng = random.Random(4000 + trial)
    n, src, dst, time, color, _ = rand_graph(rng)
    und = trial % 3 == 0
    k = rng.randint(2, 5)
    ms = [rng.randrange(3) for _ in range(k)]
    kw = _constraints(rng, n, 6)
    pb = problem(n, src, dst, time, color, und, k, ms, **kw)
    qs = oracle.query_seed(rng.getrandbits(63), 0)
    s = oracle.arc_sums(pb, qs)
    bf, _ = oracle.brute_arc_det(pb, qs)
    assert np.array_equal(s, bf)
    # localising is a split of the whole sieve: XOR of all arc sums == Q
    assert int(np.bitwise_xor.reduce(s)) == int(np.bitwise_xor.reduce(oracle.sieve_points(pb, qs)))


@pytest.mark.parametrize("trial", range(40))
def test_localized_extraction_returns_valid_path(oracle_mod, trial):
    rng = random.Random(8000 + trial)
    n, src, dst, time, color, _ = rand_graph(rng, n_lo=5, n_hi=12, t_hi=7)
    und = trial % 3 == 0
    k = rng.randint(2, 5)
    ms = [rng.randrange(3) for _ in range(k)]
    kw = {}
    r = rng.random()
    if r < 0.2:
        kw["start"] = rng.randrange(n)
    elif r < 0.4:
        kw["end"] = rng.randrange(n)
    if rng.random() < 0.3:
        kw["t_max"] = rng.randint(2, 7)
    pb = problem(n, src, dst, time, color, und, k, ms, **kw)
    truth = oracle.count_paths(pb, limit=1)[0] > 0
    found, verts, times = oracle.extract_localized(n, src, dst, time, color, 3, k, ms, undirected=und,
                                                   seed=trial + 11, **kw)
    assert found == truth
    if found:
        verify_path(n, src, dst, time, color, und, k, ms, verts, times, **kw)


def test_localized_extraction_on_config1(oracle_mod):
    g, q = synth.config1_tiny()
    for seed in (1, 2, 3):
        found, verts, times = oracle.extract_localized(g.n, g.src, g.dst, g.time, g.color, g.num_colors, q.k,
                                                       q.multiset, seed=seed)
        assert found
        verify_path(g.n, g.src, g.dst, g.time, g.color, False, q.k, q.multiset, verts, times)


# ---------------------------------------------------------------------------
# Optimum timestamp (Sec. 6.8)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("trial", range(40))
def test_optimum_time_equals_brute_force(oracle_mod, trial):
    rng = random.Random(6000 + trial)
    n, src, dst, time, color, _ = rand_graph(rng, n_lo=4, n_hi=10, t_hi=12)
    und = trial % 4 == 0
    k = rng.randint(2, 4)
    ms = [rng.randrange(3) for _ in range(k)]
    kw = {}
    if trial % 5 == 1:
        kw["t_min"] = rng.randint(1, 4)
    pb = problem(n, src, dst, time, color, und, k, ms, **kw)
    want = oracle.min_last_time(pb)
    found, t = oracle.optimum_time(n, src, dst, time, color, 3, k, ms, undirected=und, seed=trial + 5, **kw)
    assert found == (want is not None)
    if found:
        assert t == want
