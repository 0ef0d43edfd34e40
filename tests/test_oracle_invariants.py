"""Invariants of the oracle's sieve that follow from the definitions alone.

Each check relates two oracle evaluations whose answers the mathematics ties
together, independently of how the oracle computes either one:

- an undirected graph is the directed graph with both orientations of every
  edge (Sec. 4, N_i(u) of Sec. 6.4), and the coefficients y are keyed by the
  ordered arc, so the two evaluations agree bit for bit;
- the decision is a property of the graph up to isomorphism: relabelling the
  vertices (with their colours) or shifting every timestamp by a constant
  changes the coefficients but not whether a matching temporal path exists;
- a time window [t_min, t_max] is the same as deleting the arcs outside it;
- every arc whose colour pair cannot occur in a path with colours M is
  irrelevant (the filter of Sec. 8.1 (i)): dropping such arcs changes no
  per-point value.
"""
import random

import numpy as np

import oracle

ANY = oracle.ANY


def _graph(rng, n_lo=4, n_hi=10, t_hi=7, colors=3):
    n = rng.randint(n_lo, n_hi)
    m = rng.randint(n, 4 * n)
    src = np.array([rng.randrange(n) for _ in range(m)], np.uint32)
    dst = np.array([rng.randrange(n) for _ in range(m)], np.uint32)
    time = np.array([rng.randint(1, t_hi) for _ in range(m)], np.uint32)
    color = np.array([rng.randrange(colors) for _ in range(n)], np.uint32)
    return n, src, dst, time, color


def test_undirected_equals_both_orientations():
    rng = random.Random(701)
    for _ in range(60):
        n, src, dst, time, color = _graph(rng)
        k = rng.randint(2, 5)
        ms = [rng.randrange(3) for _ in range(k)]
        seed = rng.getrandbits(40)
        u = oracle.decide(n, src, dst, time, color, 3, k, ms, undirected=True, seed=seed)
        s2 = np.concatenate([src, dst])
        d2 = np.concatenate([dst, src])
        t2 = np.concatenate([time, time])
        d = oracle.decide(n, s2, d2, t2, color, 3, k, ms, seed=seed)
        assert u[0] == d[0] and u[1] == d[1]
        assert np.array_equal(u[2], d[2])


def test_decision_invariant_under_relabelling():
    rng = random.Random(702)
    for _ in range(80):
        n, src, dst, time, color = _graph(rng)
        k = rng.randint(2, 5)
        ms = [rng.randrange(3) for _ in range(k)]
        perm = np.array(rng.sample(range(n), n), np.uint32)   # old id -> new id
        color2 = np.zeros(n, np.uint32)
        color2[perm] = color
        a = oracle.decide(n, src, dst, time, color, 3, k, ms, seed=5)
        b = oracle.decide(n, perm[src], perm[dst], time, color2, 3, k, ms, seed=5)
        # one-sided error: a YES is certain; over GF(2^64) a NO is wrong with
        # probability about 2k / 2^64, so the decisions agree
        assert a[0] == b[0]


def test_decision_invariant_under_time_shift():
    rng = random.Random(703)
    for _ in range(80):
        n, src, dst, time, color = _graph(rng)
        k = rng.randint(2, 5)
        ms = [rng.randrange(3) for _ in range(k)]
        c = rng.randint(1, 1000)
        a = oracle.decide(n, src, dst, time, color, 3, k, ms, seed=9)
        b = oracle.decide(n, src, dst, time + c, color, 3, k, ms, seed=9)
        assert a[0] == b[0]
        # a window moves with the times
        lo, hi = 2, 5
        w1 = oracle.decide(n, src, dst, time, color, 3, k, ms, seed=9, t_min=lo, t_max=hi)
        w2 = oracle.decide(n, src, dst, time + c, color, 3, k, ms, seed=9, t_min=lo + c, t_max=hi + c)
        assert w1[0] == w2[0]


def test_window_equals_deleting_arcs_outside_it():
    rng = random.Random(704)
    for _ in range(60):
        n, src, dst, time, color = _graph(rng)
        k = rng.randint(2, 5)
        ms = [rng.randrange(3) for _ in range(k)]
        lo = rng.randint(1, 4)
        hi = rng.randint(lo, 7)
        seed = rng.getrandbits(40)
        w = oracle.decide(n, src, dst, time, color, 3, k, ms, seed=seed, t_min=lo, t_max=hi)
        keep = (time >= lo) & (time <= hi)
        d = oracle.decide(n, src[keep], dst[keep], time[keep], color, 3, k, ms, seed=seed)
        assert w[0] == d[0] and w[1] == d[1]
        assert np.array_equal(w[2], d[2])


def test_arcs_off_the_query_colours_change_nothing():
    rng = random.Random(705)
    for _ in range(60):
        n, src, dst, time, color = _graph(rng, colors=4)
        k = rng.randint(2, 4)
        ms = [rng.randrange(3) for _ in range(k)]   # colour 3 never queried
        seed = rng.getrandbits(40)
        a = oracle.decide(n, src, dst, time, color, 4, k, ms, seed=seed)
        inm = np.isin(color, np.array(ms, np.uint32))
        keep = inm[src] & inm[dst]
        b = oracle.decide(n, src[keep], dst[keep], time[keep], color, 4, k, ms, seed=seed)
        assert a[0] == b[0] and a[1] == b[1]
        assert np.array_equal(a[2], b[2])
