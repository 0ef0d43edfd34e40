"""The checked build: device bounds checks that set a status word and never
trap.

libtmotif_checked.so is the same library compiled with -DTMOTIF_CHECKED: every
kernel tests the indices it derives from its inputs (vertex ids of arcs,
in-segment offsets, checkpoint numbers, lane indices, colour slots) before it
uses them; a failed test skips the access and sets a bit of the device status
word, which every call reads after its work and turns into an error.  Here
the tiny configuration, a suite of random graphs (directed and undirected,
start/end vertices, windows), every layer launch shape including the staged
form, a packed batch and the server run under it in a child process: each
call must succeed (the status word stays clear) and every per-point sum and
path must equal the oracle's or the normal build's.  The child also forces the
staged form's bounded waits to run out once (tmotif_debug_stage_timeout): that
call must report TIMEOUT, and the next one on the same context must run clean.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import random, sys, time
import numpy as np
sys.path.insert(0, ".")
import oracle, synth
import paper_2001_07158_gb300 as tm

assert tm.tmotif_checked_build(), "the checked build is not the one loaded"
args = lambda g: (g.n, g.src, g.dst, g.time, g.color, g.num_colors)

# the tiny configuration, four seeds, every point
g, q = synth.config1_tiny()
G = tm.tmotif_create_graph(*args(g))
for s in range(4):
    d = tm.tmotif_decide(G, q.k, q.multiset, seed=q.seed + s)
    _, _, pp = oracle.decide(*args(g), q.k, q.multiset, seed=q.seed + s)
    assert np.array_equal(d.per_point, pp), s
G.close()

# random graphs: directed and undirected, start/end vertices, windows
rng = random.Random(5)
for i in range(60):
    n = rng.randint(3, 60)
    m = rng.randint(0, 4 * n)
    nc = rng.randint(1, 5)
    und = i % 3 == 0
    src = np.array([rng.randrange(n) for _ in range(m)], np.uint32)
    dst = np.array([rng.randrange(n) for _ in range(m)], np.uint32)
    tim = np.array([rng.randint(1, 12) for _ in range(m)], np.uint32)
    col = np.array([rng.randrange(nc) for _ in range(n)], np.uint32)
    G = tm.tmotif_create_graph(n, src, dst, tim, col, nc, undirected=und)
    k = rng.randint(2, 6)
    ms = [rng.randrange(nc) for _ in range(k)]
    kw = {"seed": rng.getrandbits(40)}
    if i % 4 == 1:
        kw["start"] = rng.randrange(n)
    if i % 4 == 2:
        kw["end"] = rng.randrange(n)
    if i % 5 == 3:
        kw["t_min"], kw["t_max"] = 3, 9
    d = tm.tmotif_decide(G, k, ms, **kw)
    _, _, pp = oracle.decide(n, src, dst, tim, col, nc, k, ms, undirected=und, **kw)
    assert np.array_equal(d.per_point, pp), i
    f, v, t = tm.tmotif_extract(G, k, ms, **kw)
    fo, vo, to = oracle.extract_localized(n, src, dst, tim, col, nc, k, ms, undirected=und, **kw)
    assert f == fo and (not f or (np.array_equal(v, vo) and np.array_equal(t, to))), i
    G.close()

# every layer launch shape at 16..128 lanes, the staged form included
g = synth.powerlaw_graph(30000, 400000, 300, 4, seed=71)
for k, L, variants in ((4, 16, (0, 1, 2)), (5, 32, (0, 3, 4)), (6, 64, (0, 1, 2, 4)), (7, 128, (0, 1, 4))):
    ms = [j % 4 for j in range(k)]
    G = tm.tmotif_create_graph(*args(g))
    ref = tm.tmotif_decide(G, k, ms, seed=9)
    for c in (64, 1024):
        for v in variants:
            tm.tmotif_set_layer_shape(G, L, c, v)
            assert np.array_equal(tm.tmotif_decide(G, k, ms, seed=9).per_point, ref.per_point), (L, c, v)
            f, vv, tt = tm.tmotif_extract(G, k, ms, seed=9)
            assert f == ref.found
    if k == 7:
        _, _, pp = oracle.decide(*args(g), k, ms, seed=9, nthreads=16)
        assert np.array_equal(ref.per_point, pp)
    G.close()

# the staged form's bounded waits, forced to run out: the call reports
# TIMEOUT (4), and the next call on the same context runs clean with the same
# sums
G = tm.tmotif_create_graph(*args(g))
ms = [j % 4 for j in range(6)]
tm.tmotif_set_layer_shape(G, 64, 128, 4)
ref = tm.tmotif_decide(G, 6, ms, seed=9)
tm.tmotif_debug_stage_timeout(True)
try:
    tm.tmotif_decide(G, 6, ms, seed=9)
    raise AssertionError("the forced timeout was not reported")
except tm.TmotifError as e:
    assert e.code == 4, e
finally:
    tm.tmotif_debug_stage_timeout(False)
assert np.array_equal(tm.tmotif_decide(G, 6, ms, seed=9).per_point, ref.per_point)
G.close()

# a packed batch and the server, against the decisions alone
items = synth.config3_batch(num_graphs=40, n_hi=800)
graphs = [tm.tmotif_create_graph(*args(gg)) for gg, _ in items]
queries = [{"k": qq.k, "multiset": qq.multiset, "seed": qq.seed} for _, qq in items]
res = tm.tmotif_decide_batch(graphs, queries)
for Gb, qd, r in zip(graphs, queries, res):
    assert np.array_equal(r.per_point, tm.tmotif_decide(Gb, **qd).per_point)
srv = tm.tmotif_server_create(0)
tickets = [tm.tmotif_submit(srv, Gb, qd["k"], qd["multiset"], seed=qd["seed"]) for Gb, qd in zip(graphs, queries)]
t0 = time.time()
for Gb, qd, t in zip(graphs, queries, tickets):
    out = None
    while out is None:
        out = tm.tmotif_poll(srv, t, qd["k"])
        assert time.time() - t0 < 300
        time.sleep(0.001)
    assert np.array_equal(out[0].per_point, tm.tmotif_decide(Gb, **qd).per_point)
srv.close()
print("CHECKED_OK")
'''


def test_checked_build_runs_clean():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    sys.path.insert(0, ROOT)
    import importlib.util

    spec = importlib.util.spec_from_file_location("_tmotif_build", os.path.join(ROOT, "paper_2001_07158_gb300",
                                                                                "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    lib = b.build(checked=True)
    import oracle

    oracle.build()
    env = dict(os.environ, TMOTIF_LIB=lib)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0 and "CHECKED_OK" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
