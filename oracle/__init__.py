"""CPU oracle for constrained multilinear sieving of temporal path motifs.

TEST INFRASTRUCTURE ONLY: the plain C reference in ``tmotif_oracle.c`` that the
GPU library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The product
library never calls it, and the two share no code.

Every function cites the passage of the paper it follows (Thejaswi, Gionis,
Lauri, arXiv 2001.07158); see ``tmotif_oracle.c`` for the arithmetic.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

ANY = 0xFFFFFFFF
KMAX = 20
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tmotif_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

u64 = C.c_uint64
u32 = C.c_uint32
i64 = C.c_int64
P = C.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP over sieve points)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        sig = {
            "or_gf_mul": (u64, [u64, u64]),
            "or_gf_pow": (u64, [u64, u64]),
            "or_gf_mul_batch": (None, [P, P, P, u64]),
            "or_gf_inv": (u64, [u64]),
            "or_fmix64": (u64, [u64]),
            "or_query_seed": (u64, [u64, u32]),
            "or_probe_seed": (u64, [u64, u32]),
            "or_coef_v": (u64, [u64, u32, u32]),
            "or_coef_w": (u64, [u64, u32, u32]),
            "or_coef_y": (u64, [u64, u32, u32, u32, u32]),
            "or_slots": (C.c_int, [u32, P, u32, P, P]),
            "or_vertex_x": (u64, [u64, u32, P, P, u32, u32, u64]),
            "or_canon": (i64, [u32, u64, P, P, P, C.c_int, P, P, P]),
            "or_sieve_points": (C.c_int, [u32, u64, P, P, P, P, u32, P, u32, P, u32, u32, u32, u32,
                                          u64, u64, u64, P, C.c_int]),
            "or_literal_table": (C.c_int, [u32, u64, P, P, P, P, u32, P, u32, P, u32, u32, u32, u32,
                                           u64, u64, u32, P, P]),
            "or_brute_points": (i64, [u32, u64, P, P, P, P, u32, P, u32, P, u32, u32, u32, u32,
                                      u64, u64, u64, P]),
            "or_brute_det": (i64, [u32, u64, P, P, P, P, u32, P, u32, P, u32, u32, u32, u32, u64, P]),
            "or_count_paths": (i64, [u32, u64, P, P, P, P, u32, P, u32, P, u32, u32, u32, u32, u64,
                                     P, P]),
            "or_brute_arc_det": (i64, [u32, u64, P, P, P, P, u32, P, u32, P, u32, u32, u32, u32, u64, P]),
            "or_arc_sums": (C.c_int, [u32, u64, P, P, P, P, u32, P, u32, P, u32, u32, u32, u32, u64, P]),
            "or_optimum_time": (C.c_int, [u32, u64, P, P, P, C.c_int, P, u32, u32, P, u32, u32, u32, u32, u64, u32,
                                          P, P, C.c_int]),
            "or_min_last_time": (i64, [u32, u64, P, P, P, P, u32, u32, P, u32, u32, u32, u32, P]),
            "or_extract_localized": (C.c_int, [u32, u64, P, P, P, C.c_int, P, u32, u32, P, u32, u32, u32, u32,
                                               u64, u32, P, P, P]),
            "or_decide": (C.c_int, [u32, u64, P, P, P, C.c_int, P, u32, P, u32, P, u32, u32, u32, u32,
                                    u64, u32, u64, u64, P, P, P, C.c_int]),
            "or_static_through": (C.c_int, [u32, u64, P, P, P, C.c_int, P, u32, P, u32, P, u32, u32, u64, P,
                                            C.c_int]),
            "or_static_brute": (i64, [u32, u64, P, P, P, C.c_int, P, u32, P, u32, P, u32, u32, u64, C.c_int, P]),
            "or_decide_ec": (C.c_int, [u32, u64, P, P, P, C.c_int, P, u32, P, u32, P, u32, u32, u32, u32,
                                       P, u64, u32, u64, u64, P, P, P, C.c_int]),
            "or_extract": (C.c_int, [u32, u64, P, P, P, C.c_int, P, u32, u32, P, u32, u32, u32, u32,
                                     u64, u32, P, P, P, P, C.c_int]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _u32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(P)


# --------------------------------------------------------------------------
# GF(2^64) and coefficients (Sec. 6.5 / Lemma 6.5)
# --------------------------------------------------------------------------
def gf_mul(a: int, b: int) -> int:
    """Product in GF(2^64) = GF(2)[x]/(x^64 + x^4 + x^3 + x + 1)."""
    return _load().or_gf_mul(a, b)


def gf_mul_batch(a, b):
    """Element-wise products of two uint64 arrays."""
    a = np.ascontiguousarray(np.asarray(a, np.uint64))
    b = np.ascontiguousarray(np.asarray(b, np.uint64))
    out = np.zeros_like(a)
    _load().or_gf_mul_batch(_ptr(a), _ptr(b), _ptr(out), len(a))
    return out


def gf_pow(a: int, e: int) -> int:
    return _load().or_gf_pow(a, e)


def gf_inv(a: int) -> int:
    return _load().or_gf_inv(a)


def fmix64(z: int) -> int:
    """splitmix64 output finaliser (Steele, Lea, Flood 2014)."""
    return _load().or_fmix64(z)


def query_seed(seed: int, r: int = 0) -> int:
    return _load().or_query_seed(seed, r)


def probe_seed(seed: int, i: int) -> int:
    return _load().or_probe_seed(seed, i)


def coef_v(qs: int, u: int, d: int) -> int:
    return _load().or_coef_v(qs, u, d)


def coef_w(qs: int, d: int, j: int) -> int:
    return _load().or_coef_w(qs, d, j)


def coef_y(qs: int, a: int, b: int, t: int, p: int) -> int:
    """y for arc a->b at time t used at walk position p (Sec. 6.3)."""
    return _load().or_coef_y(qs, a, b, t, p)


def slots(k, multiset, num_colors):
    ms = _u32(multiset)
    sb = np.zeros(num_colors, np.uint32)
    sc = np.zeros(num_colors, np.uint32)
    rc = _load().or_slots(k, _ptr(ms), num_colors, _ptr(sb), _ptr(sc))
    if rc != 0:
        raise ValueError("bad multiset")
    return sb, sc


def vertex_x(qs, k, multiset, num_colors, color_u, u, point):
    sb, sc = slots(k, multiset, num_colors)
    return _load().or_vertex_x(qs, k, _ptr(sb), _ptr(sc), color_u, u, point)


# --------------------------------------------------------------------------
# Graphs
# --------------------------------------------------------------------------
def canon(n, src, dst, time, undirected=False):
    """Canonical arc set (Sec. 4: E^tau is a set; undirected = two arcs;
    self-loops dropped), sorted by (time, src, dst)."""
    src, dst, time = _u32(src), _u32(dst), _u32(time)
    m = len(src)
    cap = (2 * m if undirected else m) + 1
    os_, od, ot = (np.zeros(cap, np.uint32) for _ in range(3))
    mc = _load().or_canon(n, m, _ptr(src), _ptr(dst), _ptr(time), int(bool(undirected)),
                          _ptr(os_), _ptr(od), _ptr(ot))
    if mc < 0:
        raise ValueError("invalid graph")
    return os_[:mc].copy(), od[:mc].copy(), ot[:mc].copy()


class Problem:
    """A query on canonical arcs (already passed through :func:`canon`)."""

    def __init__(self, n, src, dst, time, color, num_colors, k, multiset, start=ANY, end=ANY,
                 t_min=0, t_max=0, alive=None):
        self.n = int(n)
        self.src, self.dst, self.time = _u32(src), _u32(dst), _u32(time)
        self.m = len(self.src)
        self.color = _u32(color)
        self.num_colors = int(num_colors)
        self.k = int(k)
        self.multiset = _u32(multiset)
        self.start, self.end = int(start), int(end)
        self.t_min, self.t_max = int(t_min), int(t_max)
        self.alive = None if alive is None else np.ascontiguousarray(np.asarray(alive, np.uint8))

    def _args(self):
        return (self.n, self.m, _ptr(self.src), _ptr(self.dst), _ptr(self.time), _ptr(self.color),
                self.num_colors, _ptr(self.alive), self.k, _ptr(self.multiset), self.start, self.end,
                self.t_min, self.t_max)


def sieve_points(pb: Problem, qs: int, p_begin=0, p_end=None, nthreads=0):
    """Q^A for points [p_begin, p_end): eq. gen-polynomial:3 with the time index
    rolled, sieve substitution of Lemma 6.5."""
    if p_end is None:
        p_end = 1 << pb.k
    out = np.zeros(p_end - p_begin, np.uint64)
    rc = _load().or_sieve_points(*pb._args(), qs, p_begin, p_end, _ptr(out), nthreads)
    if rc != 0:
        raise ValueError("oracle sieve failed")
    return out


def literal_table(pb: Problem, qs: int, point: int, T: int):
    """Full table P_{u,l,i}, l in [0,k], i in [0,T] (eq. gen-polynomial:3 as printed)."""
    table = np.zeros(pb.n * (pb.k + 1) * (T + 1), np.uint64)
    q = np.zeros(1, np.uint64)
    rc = _load().or_literal_table(*pb._args(), qs, point, T, _ptr(table), _ptr(q))
    if rc != 0:
        raise ValueError("oracle literal table failed")
    return table.reshape(pb.n, pb.k + 1, T + 1), int(q[0])


def brute_points(pb: Problem, qs: int, p_begin=0, p_end=None):
    """Per-point sums of walk monomials (walk enumeration, Sec. 6.3)."""
    if p_end is None:
        p_end = 1 << pb.k
    out = np.zeros(p_end - p_begin, np.uint64)
    nw = _load().or_brute_points(*pb._args(), qs, p_begin, p_end, _ptr(out))
    if nw < 0:
        raise ValueError("oracle brute force failed")
    return out, nw


def brute_det(pb: Problem, qs: int):
    """Whole-sieve value from sum_walks prod(y) det(Z_walk)."""
    q = np.zeros(1, np.uint64)
    nw = _load().or_brute_det(*pb._args(), qs, _ptr(q))
    if nw < 0:
        raise ValueError("oracle det failed")
    return int(q[0]), nw


def count_paths(pb: Problem, limit=0):
    """Exhaustive temporal DFS (Sec. 9.1 baseline): number of matching temporal
    paths (stops at `limit` if > 0) and the first one found."""
    fv = np.zeros(KMAX, np.uint32)
    ft = np.zeros(KMAX, np.uint32)
    c = _load().or_count_paths(*pb._args(), limit, _ptr(fv), _ptr(ft))
    if c < 0:
        raise ValueError("oracle dfs failed")
    return int(c), fv[:pb.k].copy(), ft[:pb.k - 1].copy()


def decide(n, src, dst, time, color, num_colors, k, multiset, *, undirected=False, start=ANY, end=ANY,
           t_min=0, t_max=0, seed=1, repeats=1, point_begin=0, point_end=0, alive=None, nthreads=0):
    """Decision (Lemma 6.5): returns (found, sieve_sum, per_point) from the raw
    edge list.  per_point covers [point_begin, point_end) (0,0 = all 2^k)."""
    src, dst, time, color, ms = _u32(src), _u32(dst), _u32(time), _u32(color), _u32(multiset)
    npts = (1 << k) if point_end == 0 else point_end - point_begin
    pp = np.zeros(max(npts, 1), np.uint64)
    found = C.c_int(0)
    q = u64(0)
    al = None if alive is None else np.ascontiguousarray(np.asarray(alive, np.uint8))
    rc = _load().or_decide(n, len(src), _ptr(src), _ptr(dst), _ptr(time), int(bool(undirected)), _ptr(color),
                           num_colors, _ptr(al), k, _ptr(ms), start, end, t_min, t_max, seed, repeats,
                           point_begin, point_end, C.byref(found), C.byref(q), _ptr(pp), nthreads)
    if rc != 0:
        raise ValueError("oracle decide: invalid input")
    return bool(found.value), int(q.value), pp[:npts]


def decide_ec(n, src, dst, time, color, num_colors, k, multiset, timestamps, *, undirected=False, start=ANY,
              end=ANY, t_min=0, t_max=0, seed=1, repeats=1, point_begin=0, point_end=0, alive=None, nthreads=0):
    """EC-PathMotif decision (Sec. 7.3): the path's arc times must equal the
    strictly increasing tuple `timestamps` (k-1 entries).  Returns (found,
    sieve_sum, per_point) like decide()."""
    src, dst, time, color, ms = _u32(src), _u32(dst), _u32(time), _u32(color), _u32(multiset)
    T = _u32(timestamps)
    if len(T) != k - 1:
        raise ValueError("oracle decide_ec: need k-1 timestamps")
    npts = (1 << k) if point_end == 0 else point_end - point_begin
    pp = np.zeros(max(npts, 1), np.uint64)
    found = C.c_int(0)
    q = u64(0)
    al = None if alive is None else np.ascontiguousarray(np.asarray(alive, np.uint8))
    rc = _load().or_decide_ec(n, len(src), _ptr(src), _ptr(dst), _ptr(time), int(bool(undirected)), _ptr(color),
                              num_colors, _ptr(al), k, _ptr(ms), start, end, t_min, t_max, _ptr(T), seed, repeats,
                              point_begin, point_end, C.byref(found), C.byref(q), _ptr(pp), nthreads)
    if rc != 0:
        raise ValueError("oracle decide_ec: invalid input")
    return bool(found.value), int(q.value), pp[:npts]


def static_through(n, src, dst, time, color, num_colors, k, multiset, *, undirected=False, start=ANY, end=ANY,
                   seed=1, alive=None, nthreads=0):
    """Static preprocessing sieve (Sec. 8.1 (ii)): per-vertex sums Q_u over
    the merged static graph; Q_u != 0 iff u lies on a static path with
    colours M (w.h.p.).  Returns n uint64 values."""
    src, dst, time, color, ms = _u32(src), _u32(dst), _u32(time), _u32(color), _u32(multiset)
    qv = np.zeros(max(n, 1), np.uint64)
    al = None if alive is None else np.ascontiguousarray(np.asarray(alive, np.uint8))
    rc = _load().or_static_through(n, len(src), _ptr(src), _ptr(dst), _ptr(time), int(bool(undirected)),
                                   _ptr(color), num_colors, _ptr(al), k, _ptr(ms), start, end, seed, _ptr(qv),
                                   nthreads)
    if rc != 0:
        raise ValueError("oracle static_through: invalid input")
    return qv[:n]


def static_brute(n, src, dst, time, color, num_colors, k, multiset, *, undirected=False, start=ANY, end=ANY,
                 seed=1, alive=None, det_mode=False):
    """Static sums by walk enumeration (det_mode: via det(Z)).  Returns
    (Q_u values, number of static walks)."""
    src, dst, time, color, ms = _u32(src), _u32(dst), _u32(time), _u32(color), _u32(multiset)
    qv = np.zeros(max(n, 1), np.uint64)
    al = None if alive is None else np.ascontiguousarray(np.asarray(alive, np.uint8))
    nw = _load().or_static_brute(n, len(src), _ptr(src), _ptr(dst), _ptr(time), int(bool(undirected)),
                                 _ptr(color), num_colors, _ptr(al), k, _ptr(ms), start, end, seed,
                                 int(bool(det_mode)), _ptr(qv))
    if nw < 0:
        raise ValueError("oracle static_brute: invalid input")
    return qv[:n], int(nw)


def decide_preprocessed(n, src, dst, time, color, num_colors, k, multiset, *, undirected=False, start=ANY,
                        end=ANY, t_min=0, t_max=0, seed=1, repeats=1, point_begin=0, point_end=0, alive=None,
                        timestamps=None, nthreads=0):
    """Decision after the static preprocessing sieve: vertices with Q_u = 0
    are removed (Sec. 8.1 (ii)), then the temporal sieve runs on the rest.
    Returns (found, sieve_sum, per_point, keep_mask)."""
    qv = static_through(n, src, dst, time, color, num_colors, k, multiset, undirected=undirected, start=start,
                        end=end, seed=seed, alive=alive, nthreads=nthreads)
    keep = qv != 0
    if alive is not None:
        keep &= np.asarray(alive, bool)
    kw = dict(undirected=undirected, start=start, end=end, t_min=t_min, t_max=t_max, seed=seed, repeats=repeats,
              point_begin=point_begin, point_end=point_end, alive=keep.astype(np.uint8), nthreads=nthreads)
    if timestamps is None:
        f, s, pp = decide(n, src, dst, time, color, num_colors, k, multiset, **kw)
    else:
        f, s, pp = decide_ec(n, src, dst, time, color, num_colors, k, multiset, timestamps, **kw)
    return f, s, pp, keep


def extract(n, src, dst, time, color, num_colors, k, multiset, *, undirected=False, start=ANY, end=ANY,
            t_min=0, t_max=0, seed=1, repeats=1, nthreads=0):
    """Extraction by self-reducibility + temporal DFS (Sec. 6.9).  Returns
    (found, verts[k], times[k-1], probes)."""
    src, dst, time, color, ms = _u32(src), _u32(dst), _u32(time), _u32(color), _u32(multiset)
    verts = np.zeros(KMAX, np.uint32)
    times = np.zeros(KMAX, np.uint32)
    found = C.c_int(0)
    probes = u32(0)
    rc = _load().or_extract(n, len(src), _ptr(src), _ptr(dst), _ptr(time), int(bool(undirected)), _ptr(color),
                            num_colors, k, _ptr(ms), start, end, t_min, t_max, seed, repeats, _ptr(verts),
                            _ptr(times), C.byref(found), C.byref(probes), nthreads)
    if rc != 0:
        raise ValueError("oracle extract: invalid input")
    return bool(found.value), verts[:k].copy(), times[:k - 1].copy(), int(probes.value)


def brute_arc_det(pb: Problem, qs: int):
    """Per-arc sieve values from walk enumeration and the determinant identity:
    for each arc, the sum over walks ending with it of prod(y) det(Z_walk)."""
    out = np.zeros(max(pb.m, 1), np.uint64)
    nw = _load().or_brute_arc_det(*pb._args(), qs, _ptr(out))
    if nw < 0:
        raise ValueError("oracle arc det failed")
    return out[:pb.m], nw


def arc_sums(pb: Problem, qs: int):
    """Arc-localised sieve (Sec. 6.7 localisation, split by the last arc):
    S_e = sum over points of the last-layer term of eq. gen-polynomial:3 that
    arc e contributes.  Arcs of pb must be canonical (sorted by time)."""
    out = np.zeros(max(pb.m, 1), np.uint64)
    rc = _load().or_arc_sums(*pb._args(), qs, _ptr(out))
    if rc != 0:
        raise ValueError("oracle arc sums failed")
    return out[:pb.m]


def extract_localized(n, src, dst, time, color, num_colors, k, multiset, *, undirected=False, start=ANY, end=ANY,
                      t_min=0, t_max=0, seed=1, repeats=1):
    """Extraction by localisation: k-1 arc-localised sieves on shrinking
    problems, the path built backwards from its last arc (Sec. 6.9, second
    approach).  Returns (found, verts[k], times[k-1])."""
    src, dst, time, color, ms = _u32(src), _u32(dst), _u32(time), _u32(color), _u32(multiset)
    verts = np.zeros(KMAX, np.uint32)
    times = np.zeros(KMAX, np.uint32)
    found = C.c_int(0)
    rc = _load().or_extract_localized(n, len(src), _ptr(src), _ptr(dst), _ptr(time), int(bool(undirected)),
                                      _ptr(color), num_colors, k, _ptr(ms), start, end, t_min, t_max, seed, repeats,
                                      _ptr(verts), _ptr(times), C.byref(found))
    if rc != 0:
        raise ValueError("oracle localized extract: invalid input")
    return bool(found.value), verts[:k].copy(), times[:k - 1].copy()


def optimum_time(n, src, dst, time, color, num_colors, k, multiset, *, undirected=False, start=ANY, end=ANY,
                 t_min=0, t_max=0, seed=1, repeats=1, nthreads=0):
    """Optimum timestamp (Sec. 6.8): least t' with a matching path using only
    arcs in [t_min, t'], by binary search.  Returns (found, t_opt)."""
    src, dst, time, color, ms = _u32(src), _u32(dst), _u32(time), _u32(color), _u32(multiset)
    t = u32(0)
    found = C.c_int(0)
    rc = _load().or_optimum_time(n, len(src), _ptr(src), _ptr(dst), _ptr(time), int(bool(undirected)), _ptr(color),
                                 num_colors, k, _ptr(ms), start, end, t_min, t_max, seed, repeats, C.byref(t),
                                 C.byref(found), nthreads)
    if rc != 0:
        raise ValueError("oracle optimum time: invalid input")
    return bool(found.value), int(t.value)


def min_last_time(pb: Problem):
    """Least last-arc time over all matching paths (exhaustive DFS); None if none."""
    t = u32(0)
    c = _load().or_min_last_time(pb.n, pb.m, _ptr(pb.src), _ptr(pb.dst), _ptr(pb.time), _ptr(pb.color),
                                 pb.num_colors, pb.k, _ptr(pb.multiset), pb.start, pb.end, pb.t_min, pb.t_max,
                                 C.byref(t))
    if c < 0:
        raise ValueError("oracle dfs failed")
    return int(t.value) if c > 0 else None

