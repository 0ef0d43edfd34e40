"""Seeded synthetic temporal graphs and motif queries.

These generators stand in for the paper's datasets (KONECT/SNAP graphs and
transport feeds, Sec. 9) with the shapes its experiments use: configuration-
model style power-law out-degrees, uniform timestamps, uniform or Zipf vertex
colours, planted matching paths (Sec. 9.3 and 10.1).  They hold none of the sieve's
arithmetic: both the GPU library and the CPU oracle receive the plain arrays
they return.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

ANY = 0xFFFFFFFF


@dataclass
class Graph:
    n: int
    src: np.ndarray          # uint32, m
    dst: np.ndarray          # uint32, m
    time: np.ndarray         # uint32, m (>= 1)
    color: np.ndarray        # uint32, n
    num_colors: int
    undirected: bool = False
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.src.shape[0])


@dataclass
class Query:
    k: int
    multiset: np.ndarray     # uint32, k
    start: int = ANY
    end: int = ANY
    t_min: int = 0
    t_max: int = 0
    seed: int = 1
    repeats: int = 1
    planted: list = field(default_factory=list)


def _rng(seed):
    return np.random.default_rng(np.random.SeedSequence(int(seed)))


def uniform_graph(n, m, t_max, num_colors, seed, name="uniform"):
    """Endpoints uniform (self-loops allowed in the input; the library drops
    them), timestamps uniform in [1, t_max], colours uniform."""
    r = _rng(seed)
    src = r.integers(0, n, m, dtype=np.uint32)
    dst = r.integers(0, n, m, dtype=np.uint32)
    time = r.integers(1, t_max + 1, m, dtype=np.uint32)
    color = r.integers(0, num_colors, n, dtype=np.uint32)
    return Graph(n, src, dst, time, color, num_colors, False, name)


def powerlaw_degrees(n, m, exponent, r):
    """Discrete power-law out-degrees P(d) ~ d^-exponent on [1, n-1], rescaled
    so that they sum to exactly m."""
    u = r.random(n)
    d = np.floor((1.0 - u) ** (-1.0 / (exponent - 1.0))).astype(np.float64)
    d = np.minimum(d, n - 1)
    d = d * (m / d.sum())
    deg = np.floor(d).astype(np.int64)
    rem = m - int(deg.sum())
    if rem > 0:
        extra = r.choice(n, rem, replace=True)
        np.add.at(deg, extra, 1)
    return deg


def zipf_colors(n, num_colors, s, r):
    w = 1.0 / np.arange(1, num_colors + 1) ** s
    w /= w.sum()
    return r.choice(num_colors, n, p=w).astype(np.uint32), w


def powerlaw_graph(n, m, t_max, num_colors, seed, exponent=2.1, color_dist="uniform", name="powerlaw"):
    """Power-law out-degree (exponent 2.1), destinations uniform, timestamps
    uniform in [1, t_max]; colours uniform or Zipf(1.0)."""
    r = _rng(seed)
    deg = powerlaw_degrees(n, m, exponent, r)
    src = np.repeat(np.arange(n, dtype=np.uint32), deg)
    dst = r.integers(0, n, m, dtype=np.uint32)
    time = r.integers(1, t_max + 1, m, dtype=np.uint32)
    if color_dist == "zipf":
        color, _ = zipf_colors(n, num_colors, 1.0, r)
    else:
        color = r.integers(0, num_colors, n, dtype=np.uint32)
    return Graph(n, src, dst, time, color, num_colors, False, name)


def tour_graph(n, avg_deg, t_max, num_colors, seed, name="tour"):
    """Transport-style graph: vehicles run tours of 4-39 hops over random
    stops; a tour starts in the first half of the day and each hop departs
    1-3 slots after the previous one.  Tours are drawn in vectorised blocks."""
    r = _rng(seed)
    m_target = int(avg_deg * n)
    srcs, dsts, times = [], [], []
    total = 0
    while total < m_target:
        cnt = max(16, (m_target - total) // 15)
        length = r.integers(4, 40, cnt)                   # hops per tour
        t0 = r.integers(1, max(2, t_max // 2), cnt)       # first departure
        first = np.cumsum(length) - length                # first hop of each tour
        tour = np.repeat(np.arange(cnt), length)          # tour of each hop
        steps = r.integers(1, 4, int(length.sum()))
        cs = np.cumsum(steps)
        start = (cs - steps)[first]                       # steps before each tour
        ts = t0[tour] + (cs - start[tour]) - steps[first][tour]
        stops = r.integers(0, n, int(length.sum()) + cnt)  # length+1 stops per tour
        h = np.arange(len(steps)) + tour
        ok = ts <= t_max
        srcs.append(stops[h][ok]); dsts.append(stops[h + 1][ok]); times.append(ts[ok])
        total += int(ok.sum())
    src = np.concatenate(srcs)[:m_target].astype(np.uint32)
    dst = np.concatenate(dsts)[:m_target].astype(np.uint32)
    time = np.concatenate(times)[:m_target].astype(np.uint32)
    color = r.integers(0, num_colors, n, dtype=np.uint32)
    return Graph(n, src, dst, time, color, num_colors, False, name)


def transit_graph(n_stops, routes, trips, num_colors, seed, t_max=1440, name="transit"):
    """Timetable-style graph (the paper's transport feeds, Sec. 9.3): each
    route visits 10-39 distinct random stops with 1-5 minutes between stops;
    each of its `trips` departures (uniform over the day) adds one arc per hop,
    so every static (stop, stop) pair repeats at many times."""
    r = _rng(seed)
    length = r.integers(10, 40, routes)                          # stops per route
    first = np.cumsum(length) - length
    stops = np.concatenate([r.choice(n_stops, int(L), replace=False) for L in length]).astype(np.uint32)
    route_of = np.repeat(np.arange(routes), length)
    hop = r.integers(1, 6, int(length.sum()))                      # minutes from the previous stop
    hop[first] = 0
    offs = np.cumsum(hop)
    offs = offs - offs[first][route_of]                            # minutes since the route's first stop
    span = offs[first + length - 1]                                # route duration
    has_next = np.arange(len(stops)) + 1 < (first + length)[route_of]
    a = np.flatnonzero(has_next)                                   # hop a -> a + 1 of its route
    dep = r.integers(1, np.maximum(2, t_max - span), (trips, routes))  # departure per trip and route
    t = dep[:, route_of[a]] + offs[a + 1][None, :]
    src = np.broadcast_to(stops[a], t.shape).reshape(-1).astype(np.uint32)
    dst = np.broadcast_to(stops[a + 1], t.shape).reshape(-1).astype(np.uint32)
    time = t.reshape(-1).astype(np.uint32)
    color = r.integers(0, num_colors, n_stops, dtype=np.uint32)
    return Graph(n_stops, src, dst, time, color, num_colors, False, name)


def config_transit(n_stops=100_000, routes=10_000, trips=100, k=8, seed=12):
    """Timetable graph (100,000 stops, 10,000 routes of 10-39 stops, 100 trips
    each: about 2.4e7 arcs over about 2.4e5 static pairs), 12 colours, and a
    k = 8 query (seed 12)."""
    g = transit_graph(n_stops, routes, trips, 12, seed=seed, name=f"transit-{n_stops}x{routes}x{trips}")
    q = Query(k, draw_multiset(k, 12, seed=seed), seed=seed)
    return g, q


def plant_paths(g: Graph, multiset, count, seed, t_max=None):
    """Plant `count` temporal paths whose colours equal `multiset`: pick
    distinct vertices with the needed colours and add arcs between
    consecutive ones at strictly increasing random times (Sec. 10.1 planted
    solutions).  Returns the new graph and the planted (verts, times)."""
    r = _rng(seed)
    k = len(multiset)
    t_max = int(g.time.max()) if t_max is None else t_max
    by_color = {}
    for c in set(int(c) for c in multiset):
        by_color[c] = np.flatnonzero(g.color == c)
    planted = []
    add_s, add_d, add_t = [], [], []
    for _ in range(count):
        used = set()
        verts = []
        for c in multiset:
            pool = by_color[int(c)]
            if len(pool) == 0:
                raise ValueError("colour absent from graph")
            for _try in range(64):
                v = int(pool[r.integers(0, len(pool))])
                if v not in used:
                    break
            used.add(v)
            verts.append(v)
        verts = [verts[i] for i in r.permutation(k)]
        ts = np.sort(r.choice(np.arange(1, t_max + 1), k - 1, replace=False))
        for i in range(k - 1):
            add_s.append(verts[i]); add_d.append(verts[i + 1]); add_t.append(int(ts[i]))
        planted.append((verts, [int(t) for t in ts]))
    src = np.concatenate([g.src, np.array(add_s, np.uint32)])
    dst = np.concatenate([g.dst, np.array(add_d, np.uint32)])
    time = np.concatenate([g.time, np.array(add_t, np.uint32)])
    return Graph(g.n, src, dst, time, g.color, g.num_colors, g.undirected, g.name), planted


def draw_multiset(k, num_colors, seed, weights=None, repeat_one=False):
    """k colours drawn with replacement (weights: colour distribution); with
    repeat_one, k-1 distinct colours are drawn and the first is doubled."""
    r = _rng(seed)
    if repeat_one:
        p = None if weights is None else weights / weights.sum()
        distinct = r.choice(num_colors, k - 1, replace=False, p=p)
        ms = np.concatenate([distinct, distinct[:1]])
    else:
        p = None if weights is None else weights / weights.sum()
        ms = r.choice(num_colors, k, replace=True, p=p)
    return np.sort(ms).astype(np.uint32)


# ---------------------------------------------------------------------------
# The five workloads (sizes, distributions and seeds of the benchmark suite).
# ---------------------------------------------------------------------------
def config1_tiny():
    """n=1000, m=10^4 directed, uniform endpoints (seed 1), t in [1,100],
    8 uniform colours; k=4 drawn with replacement (seed 1)."""
    g = uniform_graph(1000, 10_000, 100, 8, seed=1, name="cfg1-uniform-1e4")
    q = Query(4, draw_multiset(4, 8, seed=1), seed=1)
    return g, q


def config1_brute():
    """The 30-vertex / 120-edge instance of config 1 (seed 2), brute-forced."""
    g = uniform_graph(30, 120, 100, 8, seed=2, name="cfg1-uniform-30x120")
    q = Query(4, draw_multiset(4, 8, seed=2), seed=2)
    return g, q


def config2_mid(n=1_000_000, m=10_000_000, plant=10):
    """Power-law out-degree (2.1), n=10^6, m=10^7, t in [1,1000], 16 colours
    Zipf(1.0) (seed 3); k=6 with one colour repeated (seed 3); planted paths."""
    r = _rng(3)
    g = powerlaw_graph(n, m, 1000, 16, seed=3, color_dist="zipf", name=f"cfg2-powerlaw-{n}x{m}")
    _, w = zipf_colors(1, 16, 1.0, r)
    ms = draw_multiset(6, 16, seed=3, weights=w, repeat_one=True)
    planted = []
    if plant:
        g, planted = plant_paths(g, ms, plant, seed=33)
    q = Query(6, ms, seed=3, planted=planted)
    return g, q


def config3_batch(num_graphs=10_000, n_lo=100, n_hi=5000, seed=4):
    """10,000 tour-style graphs, n ~ U[100,5000], average degree 8, t in
    [1,288], 12 uniform colours; per-graph k ~ U{5..8} (seed 4)."""
    r = _rng(seed)
    out = []
    for gi in range(num_graphs):
        n = int(r.integers(n_lo, n_hi + 1))
        g = tour_graph(n, 8, 288, 12, seed=seed * 1_000_003 + gi, name=f"cfg3-tour-{gi}")
        k = int(r.integers(5, 9))
        q = Query(k, draw_multiset(k, 12, seed=seed * 7_000_001 + gi), seed=seed * 13 + gi)
        out.append((g, q))
    return out


def config4_large(m=500_000_000, n=10_000_000, k=5, seed=5):
    """Power-law (2.1), n=10^7, m=5*10^8 (seed 5) with k=5, or m=10^8 (seed 6)
    with k=10; t in [1,10^4], 32 uniform colours."""
    g = powerlaw_graph(n, m, 10_000, 32, seed=seed, name=f"cfg4-powerlaw-{n}x{m}")
    q = Query(k, draw_multiset(k, 32, seed=seed), seed=seed)
    return g, q


def config5_serving(n=2_000_000, m=20_000_000, requests=4096, seed=7):
    """Resident power-law graph n=2*10^6, m=2*10^7, t in [1,1000], 16 colours
    (seed 7); request stream (seed 8): k ~ U{3..10}, 30% extract."""
    g = powerlaw_graph(n, m, 1000, 16, seed=seed, name=f"cfg5-powerlaw-{n}x{m}")
    r = _rng(8)
    reqs = []
    for i in range(requests):
        k = int(r.integers(3, 11))
        ms = draw_multiset(k, 16, seed=8_000_000 + i)
        reqs.append((Query(k, ms, seed=int(r.integers(1, 2**63))), bool(r.random() < 0.3)))
    return g, reqs


def paper_example():
    """The worked example of Fig. tempwalk-encoding-demo: V={v1,v2,v3},
    undirected edges (v1,v2,1),(v1,v2,2),(v2,v3,1),(v2,v3,2).  Vertices are
    numbered 0,1,2 for v1,v2,v3; every vertex has colour 0."""
    src = np.array([0, 0, 1, 1], np.uint32)
    dst = np.array([1, 1, 2, 2], np.uint32)
    time = np.array([1, 2, 1, 2], np.uint32)
    color = np.zeros(3, np.uint32)
    return Graph(3, src, dst, time, color, 1, True, "paper-example")
