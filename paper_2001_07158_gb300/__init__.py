"""Python binding of the GB300 temporal path-motif sieve (libtmotif.so).

Argument marshalling only: every step of the sieve runs in the CUDA library
behind ``include/tmotif.h``.  Functions carry the C names.  Importing the
package loads the in-tree library and raises if it has not been built; there
is no CPU fallback.

Method: Thejaswi, Gionis, Lauri, "Finding path motifs in large temporal graphs
using algebraic fingerprints" -- the constrained multilinear sieve (Lemma 6.5)
over the temporal-walk generating function (eq. gen-polynomial:3) in GF(2^64),
and extraction by self-reducibility (Sec. 6.9).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

TMOTIF_ANY = 0xFFFFFFFF
TMOTIF_KMAX = 20
TMOTIF_EXTRACT_HALVING = 1
TMOTIF_EXTRACT_OPTIMUM = 2
TMOTIF_PREPROCESS_STATIC = 4
ERRORS = {0: "OK", 1: "INVALID", 2: "OOM", 3: "CUDA", 4: "TIMEOUT", 5: "UNSUPPORTED", 6: "NOT_FOUND", 7: "BUSY",
          8: "CANCELLED"}

_HERE = os.path.dirname(os.path.abspath(__file__))
# TMOTIF_LIB selects another build of the library (the checked build,
# _build_checked/libtmotif_checked.so, for device bounds checks)
LIB_PATH = os.environ.get("TMOTIF_LIB") or os.path.join(_HERE, "_build", "libtmotif.so")


class TmotifError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"tmotif error {ERRORS.get(code, code)}: {msg}")
        self.code = code


class _GraphDesc(C.Structure):
    _fields_ = [("n", C.c_uint32), ("m", C.c_uint64), ("src", C.c_void_p), ("dst", C.c_void_p),
                ("time", C.c_void_p), ("color", C.c_void_p), ("num_colors", C.c_uint32),
                ("undirected", C.c_uint32), ("cuda_stream", C.c_void_p)]


class _Query(C.Structure):
    _fields_ = [("k", C.c_uint32), ("multiset", C.c_void_p), ("start", C.c_uint32), ("end", C.c_uint32),
                ("t_min", C.c_uint32), ("t_max", C.c_uint32), ("seed", C.c_uint64), ("repeats", C.c_uint32),
                ("point_begin", C.c_uint32), ("point_end", C.c_uint32), ("flags", C.c_uint32),
                ("timestamps", C.c_void_p)]


class _Decision(C.Structure):
    _fields_ = [("found", C.c_int), ("sieve_sum", C.c_uint64), ("per_point", C.c_void_p), ("ms", C.c_double)]


class _Info(C.Structure):
    _fields_ = [("n", C.c_uint32), ("m_input", C.c_uint64), ("m_arcs", C.c_uint64), ("self_loops", C.c_uint64),
                ("duplicates", C.c_uint64), ("max_time", C.c_uint32), ("device_bytes", C.c_uint64)]


class _Stats(C.Structure):
    _fields_ = [("launches", C.c_uint64), ("layer_launches", C.c_uint64), ("layer_ms", C.c_double),
                ("prep_ms", C.c_double), ("coef_ms", C.c_double), ("other_ms", C.c_double),
                ("layer_arc_lanes", C.c_uint64), ("layer_cp_lanes", C.c_uint64), ("layer_bytes", C.c_uint64),
                ("layer_gf_muls", C.c_uint64), ("layer_table_muls", C.c_uint64),
                ("layer_table_builds", C.c_uint64), ("static_launches", C.c_uint64), ("static_ms", C.c_double),
                ("static_gf_muls", C.c_uint64), ("static_table_muls", C.c_uint64),
                ("static_table_builds", C.c_uint64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libtmotif.so is not built ({LIB_PATH}); run paper_2001_07158_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    sig = {
        "tmotif_create_graph": (C.c_int, [C.POINTER(_GraphDesc), C.POINTER(P)]),
        "tmotif_destroy_graph": (None, [P]),
        "tmotif_graph_get_info": (C.c_int, [P, C.POINTER(_Info)]),
        "tmotif_decide": (C.c_int, [P, C.POINTER(_Query), C.POINTER(_Decision)]),
        "tmotif_extract": (C.c_int, [P, C.POINTER(_Query), P, P, C.POINTER(C.c_int)]),
        "tmotif_localize": (C.c_int, [P, C.POINTER(_Query), P, C.POINTER(_Decision)]),
        "tmotif_static_sieve": (C.c_int, [P, C.POINTER(_Query), P, C.POINTER(C.c_uint32)]),
        "tmotif_optimum_time": (C.c_int, [P, C.POINTER(_Query), C.POINTER(C.c_uint32), C.POINTER(C.c_int)]),
        "tmotif_decide_batch": (C.c_int, [P, P, C.c_uint32, P]),
        "tmotif_server_create": (C.c_int, [C.c_size_t, C.POINTER(P)]),
        "tmotif_submit": (C.c_int, [P, P, C.POINTER(_Query), C.c_int, C.POINTER(C.c_uint64)]),
        "tmotif_poll": (C.c_int, [P, C.c_uint64, C.POINTER(_Decision), P, P, C.POINTER(C.c_int)]),
        "tmotif_wait": (C.c_int, [P, C.c_uint64, C.c_uint32, C.POINTER(_Decision), P, P]),
        "tmotif_cancel": (C.c_int, [P, C.c_uint64]),
        "tmotif_server_destroy": (None, [P]),
        "tmotif_set_profiling": (C.c_int, [P, C.c_int]),
        "tmotif_set_layer_shape": (C.c_int, [P, C.c_uint32, C.c_uint32, C.c_uint32]),
        "tmotif_get_layer_shape": (C.c_int, [P, C.c_uint32, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]),
        "tmotif_get_stats": (C.c_int, [P, C.POINTER(_Stats)]),
        "tmotif_gf_mul_batch": (C.c_int, [P, P, P, C.c_uint64]),
        "tmotif_gf_probe": (C.c_int, [C.c_int, C.c_uint32, C.POINTER(C.c_double), C.POINTER(C.c_uint64)]),
        "tmotif_decide_noalloc": (C.c_int, [P, P, P, C.c_uint64, P, C.c_uint32, C.c_uint32, C.POINTER(_Query), P, P]),
        "tmotif_checked_build": (C.c_uint32, []),
        "tmotif_debug_stage_timeout": (C.c_int, [C.c_int]),
        "tmotif_memory_stats": (C.c_int, [C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                                          C.c_int]),
        "tmotif_tuner_export": (C.c_int, [C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]),
        "tmotif_tuner_import": (C.c_int, [C.c_char_p]),
        "tmotif_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def _check(rc):
    if rc != 0:
        raise TmotifError(rc, _lib.tmotif_last_error().decode())


def _u32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


@dataclass
class Decision:
    found: bool
    sieve_sum: int
    per_point: np.ndarray | None
    ms: float


class Graph:
    """A resident graph handle (tmotif_graph_t)."""

    def __init__(self, handle, n, num_colors, keep):
        self._h = handle
        self.n = n
        self.num_colors = num_colors
        self._keep = keep

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            _lib.tmotif_destroy_graph(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tmotif_create_graph(n, src, dst, time, color, num_colors, undirected=False, stream=None) -> Graph:
    src, dst, time, color = _u32(src), _u32(dst), _u32(time), _u32(color)
    d = _GraphDesc(n, len(src), src.ctypes.data, dst.ctypes.data, time.ctypes.data, color.ctypes.data,
                   num_colors, int(bool(undirected)), _stream_handle(stream))
    h = C.c_void_p()
    _check(_lib.tmotif_create_graph(C.byref(d), C.byref(h)))
    return Graph(h.value, n, num_colors, None)


def tmotif_destroy_graph(g: Graph):
    g.close()


def tmotif_graph_get_info(g: Graph) -> dict:
    info = _Info()
    _check(_lib.tmotif_graph_get_info(g.handle, C.byref(info)))
    return {f: getattr(info, f) for f, _ in _Info._fields_}


def _query(k, multiset, start, end, t_min, t_max, seed, repeats, point_begin, point_end, flags=0,
           timestamps=None):
    ms = _u32(multiset)
    ts = None if timestamps is None else _u32(timestamps)
    if ts is not None and len(ts) != k - 1:
        raise TmotifError(1, "EC timestamps: need k-1 values")
    q = _Query(k, ms.ctypes.data, start, end, t_min, t_max, seed & (2**64 - 1), repeats, point_begin, point_end,
               flags, None if ts is None else ts.ctypes.data)
    return q, (ms, ts)


def tmotif_decide(g: Graph, k, multiset, *, start=TMOTIF_ANY, end=TMOTIF_ANY, t_min=0, t_max=0, seed=1,
                  repeats=1, point_begin=0, point_end=0, per_point=True, timestamps=None,
                  preprocess=False) -> Decision:
    """PathMotif decision; with `timestamps` (k-1 strictly increasing times)
    the EC-PathMotif decision of Sec. 7.3; with `preprocess` the static
    preprocessing sieve first (TMOTIF_PREPROCESS_STATIC)."""
    q, keep = _query(k, multiset, start, end, t_min, t_max, seed, repeats, point_begin, point_end,
                     TMOTIF_PREPROCESS_STATIC if preprocess else 0, timestamps)
    npts = (1 << k) if point_end == 0 else max(point_end - point_begin, 0)
    pp = np.zeros(max(npts, 1), np.uint64) if per_point else None
    d = _Decision(0, 0, pp.ctypes.data if per_point else None, 0.0)
    _check(_lib.tmotif_decide(g.handle, C.byref(q), C.byref(d)))
    return Decision(bool(d.found), int(d.sieve_sum), pp[:npts] if per_point else None, float(d.ms))


def tmotif_extract(g: Graph, k, multiset, *, start=TMOTIF_ANY, end=TMOTIF_ANY, t_min=0, t_max=0, seed=1,
                   repeats=1, method="localized", optimum=False, timestamps=None, preprocess=False):
    """method: "localized" (default) or "halving" (TMOTIF_EXTRACT_HALVING);
    optimum: extract a path with the least latest time (TMOTIF_EXTRACT_OPTIMUM);
    timestamps: the EC-PathMotif tuple (Sec. 7.3), or None."""
    flags = (TMOTIF_EXTRACT_HALVING if method == "halving" else 0) | (TMOTIF_EXTRACT_OPTIMUM if optimum else 0)
    flags |= TMOTIF_PREPROCESS_STATIC if preprocess else 0
    q, keep = _query(k, multiset, start, end, t_min, t_max, seed, repeats, 0, 0, flags, timestamps)
    verts = np.zeros(k, np.uint32)
    times = np.zeros(max(k - 1, 1), np.uint32)
    found = C.c_int(0)
    _check(_lib.tmotif_extract(g.handle, C.byref(q), verts.ctypes.data, times.ctypes.data, C.byref(found)))
    return bool(found.value), verts, times[:k - 1]


def tmotif_optimum_time(g: Graph, k, multiset, *, start=TMOTIF_ANY, end=TMOTIF_ANY, t_min=0, t_max=0, seed=1,
                        repeats=1, timestamps=None, preprocess=False):
    """Optimum timestamp (Sec. 6.8): (found, least t' with a path in [t_min, t'])."""
    q, keep = _query(k, multiset, start, end, t_min, t_max, seed, repeats, 0, 0,
                     TMOTIF_PREPROCESS_STATIC if preprocess else 0, timestamps)
    t = C.c_uint32(0)
    f = C.c_int(0)
    _check(_lib.tmotif_optimum_time(g.handle, C.byref(q), C.byref(t), C.byref(f)))
    return bool(f.value), int(t.value)


def tmotif_localize(g: Graph, k, multiset, *, start=TMOTIF_ANY, end=TMOTIF_ANY, t_min=0, t_max=0, seed=1,
                    timestamps=None, preprocess=False):
    """Vertex-localised sieve: (decision, per_vertex Q_u for every vertex)."""
    q, keep = _query(k, multiset, start, end, t_min, t_max, seed, 1, 0, 0,
                     TMOTIF_PREPROCESS_STATIC if preprocess else 0, timestamps)
    pv = np.zeros(max(g.n, 1), np.uint64)
    d = _Decision(0, 0, None, 0.0)
    _check(_lib.tmotif_localize(g.handle, C.byref(q), pv.ctypes.data, C.byref(d)))
    return Decision(bool(d.found), int(d.sieve_sum), None, float(d.ms)), pv[:g.n]


def tmotif_static_sieve(g: Graph, k, multiset, *, start=TMOTIF_ANY, end=TMOTIF_ANY, seed=1):
    """Static preprocessing sieve (Sec. 8.1 (ii)): (per-vertex Q_u, number of
    kept vertices); Q_u != 0 iff u lies on a static path with colours M."""
    q, keep = _query(k, multiset, start, end, 0, 0, seed, 1, 0, 0)
    qv = np.zeros(max(g.n, 1), np.uint64)
    kept = C.c_uint32(0)
    _check(_lib.tmotif_static_sieve(g.handle, C.byref(q), qv.ctypes.data, C.byref(kept)))
    return qv[:g.n], int(kept.value)


def tmotif_decide_batch(graphs, queries):
    """queries: list of dicts with the keyword arguments of tmotif_decide."""
    n = len(graphs)
    hs = (C.c_void_p * n)(*[g.handle for g in graphs])
    qarr = (_Query * n)()
    keep = []
    pps = []
    darr = (_Decision * n)()
    for i, qd in enumerate(queries):
        qd = dict(qd)
        k = qd.pop("k")
        ms = qd.pop("multiset")
        q, kp = _query(k, ms, qd.get("start", TMOTIF_ANY), qd.get("end", TMOTIF_ANY), qd.get("t_min", 0),
                       qd.get("t_max", 0), qd.get("seed", 1), qd.get("repeats", 1), 0, 0,
                       TMOTIF_PREPROCESS_STATIC if qd.get("preprocess") else 0, qd.get("timestamps"))
        qarr[i] = q
        keep.append(kp)
        pp = np.zeros(1 << k, np.uint64)
        pps.append(pp)
        darr[i] = _Decision(0, 0, pp.ctypes.data, 0.0)
    _check(_lib.tmotif_decide_batch(hs, qarr, n, darr))
    return [Decision(bool(darr[i].found), int(darr[i].sieve_sum), pps[i], float(darr[i].ms)) for i in range(n)]


def tmotif_set_profiling(g: Graph, on=True):
    _check(_lib.tmotif_set_profiling(g.handle, int(bool(on))))


def tmotif_set_layer_shape(g: Graph, L: int, chunk: int, variant: int = 0):
    """Pin the layer kernel's launch shape for lane width L (results never
    depend on it; the autotuner picks one when none is set)."""
    _check(_lib.tmotif_set_layer_shape(g.handle, L, chunk, variant))


def tmotif_get_layer_shape(g: Graph, L: int):
    """(chunk, variant) for lane width L, or None when none is set yet."""
    c, v = C.c_uint32(0), C.c_uint32(0)
    rc = _lib.tmotif_get_layer_shape(g.handle, L, C.byref(c), C.byref(v))
    if rc == 6:
        return None
    _check(rc)
    return int(c.value), int(v.value)


def tmotif_get_stats(g: Graph) -> dict:
    s = _Stats()
    _check(_lib.tmotif_get_stats(g.handle, C.byref(s)))
    return {f: getattr(s, f) for f, _ in _Stats._fields_}


def tmotif_gf_mul_batch(a, b) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, np.uint64))
    b = np.ascontiguousarray(np.asarray(b, np.uint64))
    out = np.zeros_like(a)
    _check(_lib.tmotif_gf_mul_batch(a.ctypes.data, b.ctypes.data, out.ctypes.data, len(a)))
    return out


def tmotif_decide_noalloc(d_src, d_dst, d_time, m, d_color, n, num_colors, k, multiset, d_per_point, *,
                          start=TMOTIF_ANY, end=TMOTIF_ANY, t_min=0, t_max=0, seed=1, point_begin=0, point_end=0,
                          stream=None):
    """Allocation-free decision for callers that cannot allocate device memory
    (their allocator owns the device, or an allocation would synchronise a
    latency-bound loop).  d_* are device addresses (ints) of caller-owned
    arrays in the resident layout (canonical arcs sorted by (dst, time,
    src)); the per-point sieve sums land in d_per_point.  All intermediates
    live in the library's fixed scratch array of TMOTIF_NOALLOC_SCRATCH_BYTES,
    shared by every call: do not overlap calls on the GPU."""
    q, keep = _query(k, multiset, start, end, t_min, t_max, seed, 1, point_begin, point_end)
    _check(_lib.tmotif_decide_noalloc(d_src, d_dst, d_time, m, d_color, n, num_colors, C.byref(q), d_per_point,
                                      _stream_handle(stream)))


TMOTIF_NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024


def tmotif_gf_probe(method: int, iters: int = 256):
    """Throughput probe of a GF(2^64) product form: returns (ms, products)."""
    ms = C.c_double(0)
    n = C.c_uint64(0)
    _check(_lib.tmotif_gf_probe(method, iters, C.byref(ms), C.byref(n)))
    return ms.value, n.value


def tmotif_memory_stats(reset=False) -> dict:
    """Device memory of the library's pool: used, used_high (since the last
    reset) and reserved bytes; reset restarts the high-water mark."""
    u, h, r = C.c_uint64(0), C.c_uint64(0), C.c_uint64(0)
    _check(_lib.tmotif_memory_stats(C.byref(u), C.byref(h), C.byref(r), int(bool(reset))))
    return {"used": u.value, "used_high": h.value, "reserved": r.value}


def tmotif_tuner_export() -> str:
    """The autotuner's shapes as text lines "device L log2_arcs chunk variant"."""
    n = C.c_size_t(0)
    _check(_lib.tmotif_tuner_export(None, 0, C.byref(n)))
    buf = C.create_string_buffer(n.value + 1)
    _check(_lib.tmotif_tuner_export(buf, n.value + 1, C.byref(n)))
    return buf.value.decode()


def tmotif_tuner_import(text: str):
    _check(_lib.tmotif_tuner_import(text.encode()))


def tmotif_checked_build() -> bool:
    """True when the loaded library is the checked build (device bounds checks)."""
    return bool(_lib.tmotif_checked_build())


def tmotif_debug_stage_timeout(on: bool):
    """Checked build only: force the staged layer form's bounded waits to run
    out (the test of the timeout path)."""
    _check(_lib.tmotif_debug_stage_timeout(int(bool(on))))


def tmotif_last_error() -> str:
    return _lib.tmotif_last_error().decode()


# ---------------------------------------------------------------------------
# Serving (tmotif_server_*)
# ---------------------------------------------------------------------------
class Server:
    def __init__(self, handle):
        self._h = handle
        self._npts = {}  # ticket -> (number of per-point sums, their buffer) of a decide request

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            _lib.tmotif_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tmotif_server_create(hbm_budget_bytes: int) -> Server:
    h = C.c_void_p()
    _check(_lib.tmotif_server_create(hbm_budget_bytes, C.byref(h)))
    return Server(h.value)


def tmotif_submit(s: Server, g: Graph, k, multiset, *, is_extract=False, start=TMOTIF_ANY, end=TMOTIF_ANY,
                  t_min=0, t_max=0, seed=1, repeats=1, method="localized", timestamps=None,
                  preprocess=False, point_begin=0, point_end=0) -> int:
    flags = (TMOTIF_EXTRACT_HALVING if method == "halving" else 0) | (TMOTIF_PREPROCESS_STATIC if preprocess else 0)
    q, keep = _query(k, multiset, start, end, t_min, t_max, seed, repeats, point_begin, point_end, flags,
                     timestamps)
    t = C.c_uint64(0)
    _check(_lib.tmotif_submit(s.handle, g.handle, C.byref(q), int(bool(is_extract)), C.byref(t)))
    if not is_extract:
        npts = (1 << k) if point_end == 0 else max(point_end - point_begin, 0)
        s._npts[int(t.value)] = (npts, np.zeros(max(npts, 1), np.uint64))
    return int(t.value)


def _poll_buffers(s: Server, ticket: int, k: int):
    npts, pp = s._npts.get(ticket, (None, None))
    d = _Decision(0, 0, None if pp is None else pp.ctypes.data, 0.0)
    return npts, pp, d, np.zeros(max(k, 1), np.uint32), np.zeros(max(k, 1), np.uint32)


def tmotif_poll(s: Server, ticket: int, k: int):
    """None while the request runs; then (Decision, verts, times).  A decide
    request's Decision carries its per-point sums (first repeat)."""
    npts, pp, d, verts, times = _poll_buffers(s, ticket, k)
    done = C.c_int(0)
    rc = _lib.tmotif_poll(s.handle, ticket, C.byref(d), verts.ctypes.data, times.ctypes.data, C.byref(done))
    if rc == 0 and not done.value:
        return None
    s._npts.pop(ticket, None)
    _check(rc)
    return (Decision(bool(d.found), int(d.sieve_sum), None if pp is None else pp[:npts], float(d.ms)), verts[:k],
            times[:k - 1])


def tmotif_wait(s: Server, ticket: int, k: int, timeout_ms: int):
    """Block until the request finishes (raises TmotifError TIMEOUT = 4 after
    timeout_ms, the request staying pending); returns what tmotif_poll does."""
    npts, pp, d, verts, times = _poll_buffers(s, ticket, k)
    rc = _lib.tmotif_wait(s.handle, ticket, int(timeout_ms), C.byref(d), verts.ctypes.data, times.ctypes.data)
    if rc != 4:  # TIMEOUT leaves the request pending
        s._npts.pop(ticket, None)
    _check(rc)
    return (Decision(bool(d.found), int(d.sieve_sum), None if pp is None else pp[:npts], float(d.ms)), verts[:k],
            times[:k - 1])


def tmotif_cancel(s: Server, ticket: int):
    """Cancel a request (it then completes with TmotifError CANCELLED = 8,
    unless it had already finished)."""
    _check(_lib.tmotif_cancel(s.handle, ticket))


def tmotif_server_destroy(s: Server):
    s.close()
