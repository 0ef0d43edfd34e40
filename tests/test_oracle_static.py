"""Pins for the oracle's static preprocessing sieve (Sec. 8.1 (ii)).

The temporal graph is merged into a static graph, and a vertex is kept iff it
lies on some static path whose colours are M.  The oracle's forward/backward
recurrence over eq. gen-polynomial:1 is checked against enumeration of the
static walks (per-point monomials and the determinant identity of Lemmas
6.3/6.5), against a direct search for the vertices on static matching paths,
and for soundness: removing the other vertices never changes a decision, and
the preprocessed per-point values equal the temporal sieve on the graph
restricted to the searched vertex set.
"""
import random

import numpy as np
import pytest

import oracle

ANY = oracle.ANY


def rand_case(rng, n_lo=4, n_hi=10, colors=3, t_hi=6):
    n = rng.randint(n_lo, n_hi)
    m = rng.randint(n, 3 * n)
    src = [rng.randrange(n) for _ in range(m)]
    dst = [rng.randrange(n) for _ in range(m)]
    time = [rng.randint(1, t_hi) for _ in range(m)]
    color = [rng.randrange(colors) for _ in range(n)]
    return n, src, dst, time, color


def on_static_match(n, src, dst, color, k, ms, undirected=False, start=ANY, end=ANY, alive=None):
    """Vertices that lie on a static path of k distinct vertices with colour
    multiset ms (first = start, last = end when given), by exhaustive search."""
    adj = {u: set() for u in range(n)}
    for a, b in zip(src, dst):
        if a != b:
            adj[a].add(b)
            if undirected:
                adj[b].add(a)
    ok = [alive is None or bool(alive[u]) for u in range(n)]
    want = sorted(ms)
    hit = set()

    def rec(path):
        if len(path) == k:
            if (end == ANY or path[-1] == end) and sorted(color[u] for u in path) == want:
                hit.update(path)
            return
        for v in adj[path[-1]]:
            if v not in path and ok[v]:
                rec(path + [v])

    for u in range(n):
        if ok[u] and (start == ANY or u == start):
            rec([u])
    return hit


def _kw(rng, n, trial):
    kw = {}
    if trial % 5 == 1:
        kw["start"] = rng.randrange(n)
    if trial % 5 == 2:
        kw["end"] = rng.randrange(n)
    if trial % 4 == 3:
        kw["alive"] = [rng.random() < 0.8 for _ in range(n)]
    return kw


@pytest.mark.parametrize("trial", range(30))
def test_static_recurrence_equals_walk_enumeration(oracle_mod, trial):
    rng = random.Random(31000 + trial)
    n, src, dst, time, color = rand_case(rng)
    und = trial % 3 == 0
    k = rng.randint(2, 4)
    ms = [rng.randrange(3) for _ in range(k)]
    kw = _kw(rng, n, trial)
    seed = rng.getrandbits(40)
    dp = oracle.static_through(n, src, dst, time, color, 3, k, ms, undirected=und, seed=seed, **kw)
    bf, nw = oracle.static_brute(n, src, dst, time, color, 3, k, ms, undirected=und, seed=seed, **kw)
    bd, nw2 = oracle.static_brute(n, src, dst, time, color, 3, k, ms, undirected=und, seed=seed, det_mode=True,
                                  **kw)
    assert nw == nw2
    assert np.array_equal(dp, bf)
    assert np.array_equal(dp, bd)


@pytest.mark.parametrize("trial", range(30))
def test_nonzero_exactly_on_static_matches(oracle_mod, trial):
    rng = random.Random(32000 + trial)
    n, src, dst, time, color = rand_case(rng, n_hi=12)
    und = trial % 3 == 0
    k = rng.randint(2, 5)
    ms = [rng.randrange(3) for _ in range(k)]
    kw = _kw(rng, n, trial)
    hit = on_static_match(n, src, dst, color, k, ms, undirected=und, **kw)
    for s in range(6):
        qv = oracle.static_through(n, src, dst, time, color, 3, k, ms, undirected=und, seed=trial * 40 + s, **kw)
        assert {u for u in range(n) if qv[u]} == hit


@pytest.mark.parametrize("trial", range(30))
def test_preprocessing_is_sound(oracle_mod, trial):
    # every temporal path is a static path, so the kept vertices carry every
    # temporal match: the decision is unchanged, and the per-point values are
    # the temporal sieve restricted to the searched vertex set
    rng = random.Random(33000 + trial)
    n, src, dst, time, color = rand_case(rng, n_hi=11, t_hi=5)
    und = trial % 4 == 0
    k = rng.randint(2, 5)
    ms = [rng.randrange(3) for _ in range(k)]
    kw = _kw(rng, n, trial)
    hit = on_static_match(n, src, dst, color, k, ms, undirected=und, **kw)
    mask = np.array([u in hit for u in range(n)], np.uint8)
    seed = trial + 100
    f, s, pp, keep = oracle.decide_preprocessed(n, src, dst, time, color, 3, k, ms, undirected=und, seed=seed, **kw)
    assert np.array_equal(keep, mask.astype(bool))
    kw2 = {key: v for key, v in kw.items() if key != "alive"}
    f2, s2, pp2 = oracle.decide(n, src, dst, time, color, 3, k, ms, undirected=und, seed=seed, alive=mask, **kw2)
    assert f == f2 and s == s2 and np.array_equal(pp, pp2)
    f3, _, _ = oracle.decide(n, src, dst, time, color, 3, k, ms, undirected=und, seed=seed, **kw)
    assert f == f3


def test_static_merges_times(oracle_mod):
    # a->b at times 1 and 5 is one static arc; b->c at time 2 makes the
    # static path a,b,c although the only temporal path is a->b (1), b->c (2)
    n, color = 3, [0, 1, 2]
    src, dst, time = [0, 0, 1], [1, 1, 2], [1, 5, 2]
    qv = oracle.static_through(n, src, dst, time, color, 3, 3, [0, 1, 2], seed=9)
    assert all(qv != 0)
    # reversed times: no temporal path, but the static path keeps all three
    f, _, _, keep = oracle.decide_preprocessed(n, src, dst, [5, 5, 2], color, 3, 3, [0, 1, 2], seed=9)
    assert not f and keep.all()
    # colours not matching M: nothing kept
    qv = oracle.static_through(n, src, dst, time, color, 3, 3, [0, 0, 2], seed=9)
    assert not np.any(qv)
