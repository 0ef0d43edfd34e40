"""Pins for the oracle's EC-PathMotif sieve (Sec. 7.3).

EC-PathMotif fixes the arc times of the path to a strictly increasing tuple
T = (j_1, ..., j_{k-1}).  The oracle evaluates the paper's EC recurrence (one
value per vertex and walk length, layer l using only arcs at time j_{l-1}).
It is checked against things fixed independently of that recurrence:
enumeration of the temporal walks whose arc times are exactly T (Sec. 6.3),
exhaustive DFS for the decision, and the reduction of Lemma ectemppath:1
(a static k-path exists iff the temporal graph with every edge present at
times 1..k-1 has an EC path with T = (1, ..., k-1)).
"""
import random

import numpy as np
import pytest

import oracle

ANY = oracle.ANY


def rand_case(rng, n_lo=3, n_hi=9, t_hi=7, colors=3):
    n = rng.randint(n_lo, n_hi)
    m = rng.randint(n, 5 * n)
    src = [rng.randrange(n) for _ in range(m)]
    dst = [rng.randrange(n) for _ in range(m)]
    time = [rng.randint(1, t_hi) for _ in range(m)]
    color = [rng.randrange(colors) for _ in range(n)]
    return n, src, dst, time, color


def tuple_arcs(src, dst, time, T):
    keep = [i for i, t in enumerate(time) if t in set(T)]
    return [src[i] for i in keep], [dst[i] for i in keep], [time[i] for i in keep]


def rand_tuple(rng, k, t_hi):
    return sorted(rng.sample(range(1, t_hi + 1), k - 1))


@pytest.mark.parametrize("trial", range(40))
def test_ec_equals_enumeration_of_walks_with_those_times(oracle_mod, trial):
    # A temporal walk of k-1 arcs with strictly increasing times drawn from
    # the k-1 values of T uses them all, in order: enumerating the temporal
    # walks of the arcs whose time is in T gives exactly the EC walks.
    rng = random.Random(21000 + trial)
    n, src, dst, time, color = rand_case(rng, n_hi=7, t_hi=5)
    src, dst, time = src * 2, dst[::-1] + dst, time + time[::-1]  # denser: walks exist
    und = trial % 3 == 0
    k = rng.randint(2, 5)
    T = rand_tuple(rng, k, 5)
    ms = [rng.randrange(3) for _ in range(k)]
    kw = {}
    if trial % 5 == 1:
        kw["start"] = rng.randrange(n)
    if trial % 5 == 2:
        kw["end"] = rng.randrange(n)
    if trial % 4 == 3:
        kw["alive"] = [rng.random() < 0.8 for _ in range(n)]
    seed = rng.getrandbits(40)
    _, _, pp = oracle.decide_ec(n, src, dst, time, color, 3, k, ms, T, undirected=und, seed=seed, **kw)
    fs, fd, ft = tuple_arcs(src, dst, time, T)
    cs, cd, ct = oracle.canon(n, fs, fd, ft, und)
    pb = oracle.Problem(n, cs, cd, ct, color, 3, k, ms, **kw)
    bf, _ = oracle.brute_points(pb, oracle.query_seed(seed, 0))
    assert np.array_equal(pp, bf)


def test_ec_start_and_end_restrict_the_walks(oracle_mod):
    # complete digraph on 5 vertices, every arc at times 1..4; every point's
    # value with an end (start) vertex equals the enumeration of the walks
    # ending (starting) there, and the ends together give the unrestricted value
    n = 5
    arcs = [(a, b, t) for a in range(n) for b in range(n) if a != b for t in range(1, 5)]
    src, dst, time = (list(x) for x in zip(*arcs))
    color = [0, 1, 2, 0, 1]
    k, ms, T = 3, [0, 1, 2], [1, 3]
    fs, fd, ft = tuple_arcs(src, dst, time, T)
    cs, cd, ct = oracle.canon(n, fs, fd, ft)
    qs = oracle.query_seed(31, 0)
    total = oracle.decide_ec(n, src, dst, time, color, 3, k, ms, T, seed=31)[2]
    acc = np.zeros_like(total)
    for u in range(n):
        for key in ("start", "end"):
            pp = oracle.decide_ec(n, src, dst, time, color, 3, k, ms, T, seed=31, **{key: u})[2]
            bf, _ = oracle.brute_points(oracle.Problem(n, cs, cd, ct, color, 3, k, ms, **{key: u}), qs)
            assert np.array_equal(pp, bf)
            if key == "end":
                acc ^= pp
    assert np.array_equal(acc, total) and np.any(total != 0)


@pytest.mark.parametrize("trial", range(40))
def test_ec_decision_equals_exhaustive_dfs(oracle_mod, trial):
    rng = random.Random(22000 + trial)
    n, src, dst, time, color = rand_case(rng, n_hi=10, t_hi=6)
    k = rng.randint(2, 5)
    T = rand_tuple(rng, k, 6)
    ms = [rng.randrange(3) for _ in range(k)]
    fs, fd, ft = tuple_arcs(src, dst, time, T)
    cs, cd, ct = oracle.canon(n, fs, fd, ft)
    truth = oracle.count_paths(oracle.Problem(n, cs, cd, ct, color, 3, k, ms), limit=1)[0] > 0
    for s in range(6):
        f, q, _ = oracle.decide_ec(n, src, dst, time, color, 3, k, ms, T, seed=trial * 50 + s)
        assert f == truth
        if not truth:
            assert q == 0


def _static_kpath(n, edges, k):
    adj = {u: set() for u in range(n)}
    for a, b in edges:
        if a != b:
            adj[a].add(b)
    for s in range(n):
        stack = [(s, (s,))]
        while stack:
            u, path = stack.pop()
            if len(path) == k:
                return True
            for v in adj[u]:
                if v not in path:
                    stack.append((v, path + (v,)))
    return False


@pytest.mark.parametrize("trial", range(20))
def test_ectemppath_reduction(oracle_mod, trial):
    # Lemma ectemppath:1 with one colour (EC-TempPath = EC-PathMotif, M = {1^k}).
    rng = random.Random(23000 + trial)
    n = rng.randint(4, 8)
    edges = [(rng.randrange(n), rng.randrange(n)) for _ in range(rng.randint(3, 10))]
    k = rng.randint(2, 5)
    src, dst, time = [], [], []
    for a, b in edges:
        for t in range(1, k):
            src.append(a); dst.append(b); time.append(t)
    f, _, _ = oracle.decide_ec(n, src, dst, time, [0] * n, 1, k, [0] * k, list(range(1, k)), seed=trial + 3)
    assert f == _static_kpath(n, edges, k)


def test_arcs_at_other_times_change_nothing(oracle_mod):
    rng = random.Random(24000)
    n, src, dst, time, color = rand_case(rng, n_lo=8, n_hi=8, t_hi=9)
    T = [2, 5, 8]
    base = oracle.decide_ec(n, src, dst, time, color, 3, 4, [0, 1, 2, 1], T, seed=77)[2]
    extra = [t for t in range(1, 12) if t not in T]
    s2 = src + [rng.randrange(n) for _ in range(40)]
    d2 = dst + [rng.randrange(n) for _ in range(40)]
    t2 = time + [rng.choice(extra) for _ in range(40)]
    assert np.array_equal(base, oracle.decide_ec(n, s2, d2, t2, color, 3, 4, [0, 1, 2, 1], T, seed=77)[2])


def test_tuple_order_is_enforced(oracle_mod):
    # a->b at 5 then b->c at 2: the times of the walk are (5, 2), not a tuple
    # with j_1 < j_2, so T = (2, 5) finds nothing and T = (5, 2) is invalid.
    n, src, dst, time, color = 3, [0, 1], [1, 2], [5, 2], [0, 1, 2]
    f, q, _ = oracle.decide_ec(n, src, dst, time, color, 3, 3, [0, 1, 2], [2, 5], seed=1)
    assert not f and q == 0
    with pytest.raises(ValueError):
        oracle.decide_ec(n, src, dst, time, color, 3, 3, [0, 1, 2], [5, 2], seed=1)
    f, _, _ = oracle.decide_ec(n, [0, 1], [1, 2], [2, 5], color, 3, 3, [0, 1, 2], [2, 5], seed=1)
    assert f


def test_ec_time_window_applies_too(oracle_mod):
    # arcs outside [t_min, t_max] are unused: a window that cuts off j_1
    # leaves no EC walk; a window covering T changes nothing
    n = 4
    arcs = [(a, b, t) for a in range(n) for b in range(n) if a != b for t in (1, 2, 3)]
    src, dst, time = (list(x) for x in zip(*arcs))
    color = [0, 1, 2, 1]
    k, ms, T = 3, [0, 1, 2], [1, 3]
    full = oracle.decide_ec(n, src, dst, time, color, 3, k, ms, T, seed=5)
    assert full[0]
    assert np.array_equal(full[2], oracle.decide_ec(n, src, dst, time, color, 3, k, ms, T, seed=5, t_min=1,
                                                    t_max=3)[2])
    cut = oracle.decide_ec(n, src, dst, time, color, 3, k, ms, T, seed=5, t_min=2)
    assert not cut[0] and not np.any(cut[2])
