"""The allocation-free decision (tmotif_decide_noalloc) against tmotif_decide.

Callers that cannot allocate device memory -- their own allocator owns the
device, or an allocation would synchronise a latency-bound loop -- hand the
library their device arrays and get the per-point sieve sums back in a device
buffer they own, with every intermediate in the library's fixed scratch array.
The results must equal the ordinary entry point's bit for bit, call after call
(the shared array keeps the previous call's contents).

This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2001_07158_gb300 as tm

    return tm


def device_graph(g):
    """Canonical arcs (self-loops dropped, duplicates merged) sorted by
    (dst, time, src), as device tensors."""
    import torch

    keep = g.src != g.dst
    s, d, t = g.src[keep], g.dst[keep], g.time[keep]
    order = np.lexsort((s, t, d))
    s, d, t = s[order], d[order], t[order]
    uniq = np.ones(len(s), bool)
    uniq[1:] = (s[1:] != s[:-1]) | (d[1:] != d[:-1]) | (t[1:] != t[:-1])
    s, d, t = s[uniq], d[uniq], t[uniq]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()
    return dev(s), dev(d), dev(t), dev(g.color), len(s)


def test_noalloc_equals_decide_on_consecutive_calls(tm):
    import torch

    stream = torch.cuda.current_stream()
    g, q = synth.config1_tiny()
    G = tm.tmotif_create_graph(g.n, g.src, g.dst, g.time, g.color, g.num_colors, stream=stream)
    src, dst, time, color, m = device_graph(g)
    g2 = synth.uniform_graph(300, 2500, 40, 5, seed=21)
    G2 = tm.tmotif_create_graph(g2.n, g2.src, g2.dst, g2.time, g2.color, g2.num_colors, stream=stream)
    src2, dst2, time2, color2, m2 = device_graph(g2)
    calls = [
        (G, (src, dst, time, m, color, g.n, g.num_colors), q.k, q.multiset, {"seed": q.seed}),
        (G, (src, dst, time, m, color, g.n, g.num_colors), q.k, q.multiset, {"seed": q.seed + 1}),
        (G2, (src2, dst2, time2, m2, color2, g2.n, g2.num_colors), 6, [0, 0, 1, 2, 3, 4], {"seed": 9, "t_max": 30}),
        (G, (src, dst, time, m, color, g.n, g.num_colors), q.k, q.multiset,
         {"seed": q.seed, "point_begin": 3, "point_end": 14}),
    ]
    for Gh, (s, d, t, mm, c, n, nc), k, ms, kw in calls:
        npts = (kw.get("point_end", 0) - kw.get("point_begin", 0)) or (1 << k)
        out = torch.full((npts,), -1, dtype=torch.int64, device="cuda")  # stale values must not survive
        tm.tmotif_decide_noalloc(s.data_ptr(), d.data_ptr(), t.data_ptr(), mm, c.data_ptr(), n, nc, k, ms,
                                 out.data_ptr(), stream=stream, **kw)
        got = out.cpu().numpy().view(np.uint64)
        want = tm.tmotif_decide(Gh, k, ms, **kw).per_point
        assert np.array_equal(got, want)
    G.close()
    G2.close()


def test_noalloc_rejects_graphs_beyond_the_fixed_scratch(tm):
    import torch

    n = 200_000  # the per-vertex coefficient table alone needs n * 64 * 8 bytes
    src = torch.zeros(1, dtype=torch.int32, device="cuda")
    dst = torch.ones(1, dtype=torch.int32, device="cuda")
    time = torch.ones(1, dtype=torch.int32, device="cuda")
    color = torch.zeros(n, dtype=torch.int32, device="cuda")
    out = torch.zeros(64, dtype=torch.int64, device="cuda")
    with pytest.raises(tm.TmotifError) as e:
        tm.tmotif_decide_noalloc(src.data_ptr(), dst.data_ptr(), time.data_ptr(), 1, color.data_ptr(), n, 1, 6,
                                 [0] * 6, out.data_ptr())
    assert e.value.code == 5 and "scratch" in str(e.value)


def hub_graph():
    """A graph with one vertex whose in-segment (300 arcs) is longer than a
    team chunk of the allocation-free layer kernel (128 arcs), plus uniform
    arcs, so that segments cross chunk boundaries."""
    rng = np.random.default_rng(31)
    g = synth.uniform_graph(400, 1500, 60, 4, seed=32)
    hub = 5
    s = rng.choice(np.setdiff1d(np.arange(400), [hub]), 300, replace=False).astype(np.uint32)
    t = rng.integers(1, 61, 300).astype(np.uint32)
    g.src = np.concatenate([g.src, s, np.full(40, hub, np.uint32)])
    g.dst = np.concatenate([g.dst, np.full(300, hub, np.uint32), rng.integers(0, 400, 40).astype(np.uint32)])
    g.time = np.concatenate([g.time, t, rng.integers(1, 61, 40).astype(np.uint32)])
    return g


def test_noalloc_start_end_k2_and_long_segments(tm):
    """Start/end vertices, k = 2 (the first layer is also the last) and an
    in-segment longer than a chunk: equal to tmotif_decide and to the oracle,
    point by point."""
    import torch

    import oracle

    stream = torch.cuda.current_stream()
    g = hub_graph()
    G = tm.tmotif_create_graph(g.n, g.src, g.dst, g.time, g.color, g.num_colors, stream=stream)
    src, dst, time, color, m = device_graph(g)
    hub = 5
    cases = [
        (2, [int(g.color[hub]), int(g.color[hub])], {"seed": 3}),
        (2, [0, 1], {"seed": 4, "end": hub}),
        (4, [int(g.color[hub]), 0, 1, 2], {"seed": 5, "end": hub}),
        (5, [0, 1, 2, 3, int(g.color[7])], {"seed": 6, "start": 7}),
        (6, [0, 0, 1, 2, 3, 3], {"seed": 7, "start": 11, "end": hub, "t_min": 3}),
        (7, [0, 1, 2, 3, 0, 1, 2], {"seed": 8, "point_begin": 60, "point_end": 127}),
    ]
    for k, ms, kw in cases:
        npts = (kw.get("point_end", 0) - kw.get("point_begin", 0)) or (1 << k)
        out = torch.full((npts,), -1, dtype=torch.int64, device="cuda")
        tm.tmotif_decide_noalloc(src.data_ptr(), dst.data_ptr(), time.data_ptr(), m, color.data_ptr(), g.n,
                                 g.num_colors, k, ms, out.data_ptr(), stream=stream, **kw)
        got = out.cpu().numpy().view(np.uint64)
        want = tm.tmotif_decide(G, k, ms, **kw).per_point
        assert np.array_equal(got, want), (k, kw)
        okw = dict(kw)
        _, _, pp = oracle.decide(g.n, g.src, g.dst, g.time, g.color, g.num_colors, k, ms, **okw)
        assert np.array_equal(got, pp), (k, kw)
    G.close()


def test_noalloc_empty_graph_gives_zero_sums(tm):
    import torch

    color = torch.zeros(10, dtype=torch.int32, device="cuda")
    out = torch.full((16,), -1, dtype=torch.int64, device="cuda")
    tm.tmotif_decide_noalloc(0, 0, 0, 0, color.data_ptr(), 10, 2, 4, [0, 0, 1, 1], out.data_ptr())
    assert not out.cpu().numpy().any()


def test_noalloc_rejects_invalid_inputs(tm):
    """Unsorted arcs, and a colour >= num_colors on a vertex with no arcs,
    are INVALID (checked before any coefficient work)."""
    import torch

    g = synth.uniform_graph(50, 200, 20, 3, seed=41)
    src, dst, time, color, m = device_graph(g)
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    # swap two arcs of different destinations: no longer sorted by (dst, time, src)
    bad_src, bad_dst, bad_time = src.clone(), dst.clone(), time.clone()
    i, j = 0, m - 1
    for a in (bad_src, bad_dst, bad_time):
        a[i], a[j] = a[j].item(), a[i].item()
    with pytest.raises(tm.TmotifError) as e:
        tm.tmotif_decide_noalloc(bad_src.data_ptr(), bad_dst.data_ptr(), bad_time.data_ptr(), m, color.data_ptr(),
                                 g.n, g.num_colors, 4, [0, 1, 2, 0], out.data_ptr())
    assert e.value.code == 1
    # one more vertex, without arcs, whose colour is num_colors
    color2 = torch.cat([color, torch.tensor([g.num_colors], dtype=torch.int32, device="cuda")])
    with pytest.raises(tm.TmotifError) as e:
        tm.tmotif_decide_noalloc(src.data_ptr(), dst.data_ptr(), time.data_ptr(), m, color2.data_ptr(), g.n + 1,
                                 g.num_colors, 4, [0, 1, 2, 0], out.data_ptr())
    assert e.value.code == 1 and "colour" in str(e.value)
    # m beyond the 32-bit arc numbering
    with pytest.raises(tm.TmotifError) as e:
        tm.tmotif_decide_noalloc(src.data_ptr(), dst.data_ptr(), time.data_ptr(), 1 << 32, color.data_ptr(), g.n,
                                 g.num_colors, 4, [0, 1, 2, 0], out.data_ptr())
    assert e.value.code == 1
