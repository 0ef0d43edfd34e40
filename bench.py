#!/usr/bin/env python3
"""Benchmark of the temporal path-motif sieve on one GB300 (or N replicas).

Headline workload: the mid-size decision of the benchmark suite -- a power-law
out-degree temporal graph (exponent 2.1, n = 10^6, m = 10^7 edges, timestamps
uniform in [1, 1000], 16 colours Zipf(1.0)) with a k = 6 multiset query (one
colour twice), 2^6 = 64 sieve points, exact GF(2^64) arithmetic.  A step is one
full decision on the resident graph: per-query arc filter and checkpoint
build, sieve coefficients, the k-1 generating-function layers, the sieve sum.

Metric: edge-steps/s = m * k * 2^k / (time of one decision).

On one GPU the same JSON line also carries the other workloads of the suite,
each measured after the headline's timed region:
  large10  the large-sieve decision n = 10^7, m = 10^8, k = 10 (1024 points);
  large5   the large-sieve decision n = 10^7, m = 5*10^8, k = 5 (32 points);
  transit  a timetable graph (2.4e7 arcs) at k = 8, without and with the
           static preprocessing sieve;
  batch    10,000 small tour graphs in one batched call, against one
           tmotif_decide per graph, both timed by CUDA events on the stream;
  serving  4,096 requests (k in 3..10, 30 % extract) against a resident
           n = 2*10^6, m = 2*10^7 graph, Poisson arrivals at 70 % of the plain
           form's capacity: the plain form (one request at a time, in arrival
           order) and the server, both live, plus both forms saturated;
  cpu_baseline  the oracle on every host core, on a sample of the points.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--legs large10,large5,transit,batch,serving,cpu] [--workload ...]

With N > 1 it runs under torchrun, one rank per GPU; every rank decides its own
query (another seed) on its own replica of the graph -- the sieve points of
different queries are independent, so there is no data-path collective
("weak" scaling); ranks meet only at the timing barrier.  The extra workloads
run at N = 1 only.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sieve edge-steps/s (m*k*2^k per s) at k=5..10; served query p50/p99 latency"
UNIT = "edge-steps/s"
WORKLOAD = ("power-law out-degree 2.1, n=1e6, m=1e7 (+50 planted arcs), t in [1,1000], 16 colours Zipf(1.0); "
            "PathMotif k=6 with one colour twice, 64 sieve points, GF(2^64)")

# The paper's own figures (Sec. 10, Table 4 and the headline extraction), on
# its own hardware: context beside the line, not a target for this workload.
PAPER = {
    "decision": {"figure_s": 109.04, "workload": "d-regular d=200, m=10,000,070, t=100, k=8 (256 points), "
                 "4 threads", "edge_steps_per_s": 10_000_070 * 8 * 256 / 109.04,
                 "hardware": "Intel Core i5-4570 (Haswell), 3.2 GHz, 4 cores", "cite": "Sec. 10, Table 4"},
    "extraction": {"figure_s": 444.66, "workload": "optimum solution, Helsinki transport graph, n=7,959, "
                   "m=6,403,785, t=1,440, k=10", "hardware": "Intel Core i5-4570 (Haswell), 3.2 GHz, 4 cores",
                   "cite": "abstract and Sec. 10"},
}


def table_costs(rates):
    """Seconds of GPU time per unit of layer work, from the product rates of
    the register-resident probe (tmotif_gf_probe): `reg` a register product;
    `lookup` one lane's table product and `build` one shared table, solved from
    the table form's rates at 64 and 128 lanes per table
    (1/R64 = build/64 + lookup, 1/R128 = build/128 + lookup)."""
    inv64, inv128 = 1.0 / rates["table64"], 1.0 / rates["table128"]
    build = max(128.0 * (inv64 - inv128), 0.0)
    lookup = max(inv128 - build / 128.0, 0.0)
    return {"reg": 1.0 / rates["reg"], "lookup": lookup, "build": build}


def layer_bound_s(costs, reg, tab, builds):
    """Lower-bound seconds of one layer launch with `reg` register products,
    `tab` table products and `builds` table builds: each product form needs
    at least the time the GPU takes for that form's work alone, at the
    probe's measured rate, so the bound is the larger of the two."""
    t_tab = tab * costs["lookup"] + builds * costs["build"]
    t_reg = reg * costs["reg"]
    return max(t_tab, t_reg), {"table": t_tab, "register": t_reg}


def probe_rates(tm, iters=2048, repeats=3):
    """GF(2^64) products per second of each product form on this GPU, on
    register-resident data with no memory traffic (best of `repeats`)."""
    rates = {}
    for name, method in (("reg", 0), ("table64", 1), ("table128", 2)):
        best = 0.0
        for _ in range(repeats):
            ms, n = tm.tmotif_gf_probe(method, iters)
            best = max(best, n / (ms / 1e3))
        rates[name] = best
    return rates


# DRAM traffic of one layer launch from an ncu capture, valid only for the
# layer-kernel sources it was taken on (source_sha() below, first 16 hex):
# a timed-decision layer of the default workload, full size, one-pass dram
# counters
LAYER_TRAFFIC = {"source_sha": "b84d4058b4a9445d", "bytes_per_launch": 1124364288 + 399417856}


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--e2e-steps", type=int, default=5)
    p.add_argument("--legs", default="large10,large5,transit,batch,serving,cpu",
                   help="extra workloads measured after the headline at N = 1 (comma list of large10, large5, "
                        "transit, batch, serving, cpu; empty for none)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--serving-requests", type=int, default=4096)
    p.add_argument("--scale", type=float, default=1.0,
                   help="scale n and m of the workload (profiling captures of a smaller case)")
    p.add_argument("--workload", choices=sorted(WORKLOADS), default="mid",
                   help="mid: the default decision (n=1e6, m=1e7, k=6); large5 / large10: power-law "
                        "n=1e7 with m=5e8, k=5 / m=1e8, k=10; batch: 10,000 small tour graphs in one "
                        "batched call (k in 5..8); transit: a timetable graph for --preprocess")
    p.add_argument("--preprocess", action="store_true", help="static preprocessing sieve before each decision")
    p.add_argument("--layer-shape", default="",
                   help="CHUNK,VARIANT: pin the layer kernel's launch shape (tmotif_set_layer_shape) for the "
                        "workload's lane width instead of the autotuner's pick (profiling one form)")
    return p.parse_args(argv)


def legs_of(args):
    legs = {x.strip() for x in args.legs.split(",") if x.strip()}
    if args.no_cpu_baseline:
        legs.discard("cpu")
    if args.no_serving:
        legs.discard("serving")
    return legs


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def source_sha():
    """Hash of the layer kernel's device code (its team body, the GF(2^64)
    products it calls, and the kernels and launches around them), comments
    and blank lines left out so that a comment edit keeps the captured
    traffic valid."""
    h = hashlib.sha256()
    for f in ("layer.cuh", "gf64.cuh", "sieve.cu"):
        text = open(os.path.join(ROOT, "paper_2001_07158_gb300", "csrc", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        code = [line.rstrip() for line in text.splitlines() if line.strip()]
        h.update("\n".join(code).encode())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None

    def start(self):
        self.out = tempfile.NamedTemporaryFile("w+", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        self.proc.wait()
        self.out.flush()
        self.out.seek(0)
        sm, smax, reasons, power = [], [], set(), []
        for line in self.out.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            if self.uuid and parts[0] != self.uuid:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, flag in zip(self.NAMES, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(name)
        os.unlink(self.out.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


WORKLOADS = {
    "mid": WORKLOAD,
    "large5": "power-law out-degree 2.1, n=1e7, m=5e8, t in [1,1e4], 32 uniform colours; PathMotif k=5, 32 points",
    "large10": "power-law out-degree 2.1, n=1e7, m=1e8, t in [1,1e4], 32 uniform colours; PathMotif k=10, "
               "1024 points",
    "batch": "10,000 tour-style graphs, n~U[100,5000], avg out-degree 8, t in [1,288], 12 colours; "
             "k~U{5..8}; one batched call",
    "transit": "timetable graph: 100,000 stops, 10,000 routes of 10-39 stops x 100 trips (2.4e7 arcs over "
               "2.4e5 static pairs), t in [1,1440], 12 colours; PathMotif k=8, 256 points",
}


def workload(scale=1.0, name="mid"):
    import synth

    if name == "large5":
        return synth.config4_large(m=int(500_000_000 * scale), n=int(10_000_000 * scale), k=5, seed=5)
    if name == "large10":
        return synth.config4_large(m=int(100_000_000 * scale), n=int(10_000_000 * scale), k=10, seed=6)
    if name == "transit":
        return synth.config_transit(n_stops=int(100_000 * scale), routes=int(10_000 * scale))
    if scale == 1.0:
        return synth.config2_mid()
    return synth.config2_mid(n=int(1_000_000 * scale), m=int(10_000_000 * scale))


def cpu_baseline(g, q):
    """The oracle as it stands (plain C, OpenMP over sieve points) on every
    host core, on a bounded sample of the same decision: the first P of its
    2^k sieve points, P = the host's core count (one point per thread)."""
    import oracle

    cores = os.cpu_count() or 1
    P = max(1, min(cores, 1 << q.k))
    t0 = time.perf_counter()
    oracle.decide(g.n, g.src, g.dst, g.time, g.color, g.num_colors, q.k, q.multiset, seed=q.seed, point_begin=0,
                  point_end=P, nthreads=P)
    dt = time.perf_counter() - t0
    return {"value": g.m * q.k * P / dt, "unit": UNIT, "cores": P, "nproc": cores, "kind": "oracle",
            "sample": f"points [0, {P}) of the {1 << q.k} sieve points of the same decision, one per host core "
                      f"({dt:.1f} s)"}


def measure_decision(tm, stream, dev, G, q, steps, warmup, seed, preprocess=False, world=1):
    """Time `steps` decisions of query q on the resident graph G (after
    `warmup` untimed ones), L2 flushed between steps, with the library's layer
    statistics on; returns (total ms, per-step results, stats, clocks)."""
    import torch

    for i in range(warmup):
        tm.tmotif_decide(G, q.k, q.multiset, seed=seed + i, preprocess=preprocess, per_point=False)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    props = torch.cuda.get_device_properties(dev)
    uuid = str(getattr(props, "uuid", ""))
    if uuid and not uuid.startswith("GPU-"):
        uuid = "GPU-" + uuid
    sampler = ClockSampler(uuid)
    tm.tmotif_set_profiling(G, True)
    sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    found = []
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xFF)
            starts[i].record(stream)
        d = tm.tmotif_decide(G, q.k, q.multiset, seed=seed + 1000 + i, per_point=False, preprocess=preprocess)
        ends[i].record(stream)
        found.append(d.found)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    stats = tm.tmotif_get_stats(G)
    tm.tmotif_set_profiling(G, False)
    total_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    del flush
    return total_ms, found, stats, clocks


def phases_of(stats, total_ms, steps):
    """Device time per step by kernel family (the library's CUDA events;
    static = the static sieve's layer launches), and the rest of the step:
    host turnarounds, launch gaps and the launches outside those families."""
    if not steps:
        return None
    out = {f: stats[f + "_ms"] / steps for f in ("prep", "coef", "layer", "other", "static")}
    out["unprofiled"] = total_ms / steps - sum(out.values())
    return {k: round(v, 4) for k, v in out.items()}


def roofline_of(stats, total_ms, costs, rates, traffic):
    """Roofline of the dominant kernel (the layer kernel), from the library's
    CUDA events around every layer launch during the timed region: achieved
    GF(2^64) products per second against the rate at which this GPU does the
    same products with no memory traffic (the larger of the launch's
    table-form and register-form times at the probe's measured rates)."""
    nl = max(stats["layer_launches"], 1)
    layer_ms = stats["layer_ms"] / nl
    muls = stats["layer_gf_muls"] / nl
    tmuls = stats["layer_table_muls"] / nl
    builds = stats["layer_table_builds"] / nl
    t_min, forms = layer_bound_s(costs, muls - tmuls, tmuls, builds)
    achieved = muls / (layer_ms / 1e3) / 1e9
    peak = muls / t_min / 1e9 if t_min > 0 else None
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G GF(2^64) products/s",
            "frac": achieved / peak if peak else None, "traffic": traffic,
            "kernel": "k_layer (eq. gen-polynomial:3 layer)",
            "model": "product rates measured at bench start by tmotif_gf_probe (register-resident, no memory "
                     "traffic); bound = max(table-form time, register-form time); binding form: "
                     + max(forms, key=forms.get),
            "probe_products_per_s": rates, "form_ms": {k: v * 1e3 for k, v in forms.items()},
            # not a bound: the two forms' times back to back, for comparison
            # with the measured launch (equal when the forms do not overlap)
            "forms_sum_ms": sum(forms.values()) * 1e3,
            "layer_ms_per_launch": layer_ms, "gf_muls_per_launch": muls, "table_muls_per_launch": tmuls,
            "table_builds_per_launch": builds, "algorithmic_bytes_per_launch": stats["layer_bytes"] / nl,
            "achieved_hbm_gbs": stats["layer_bytes"] / nl / (layer_ms / 1e3) / 1e9,
            "layer_share_of_step": stats["layer_ms"] / total_ms if total_ms else None}


def e2e_decision(tm, stream, g, q, seed, steps, preprocess=False, warmup=1):
    """End to end through the C ABI with host buffers: upload and build the
    graph from pinned host arrays, decide, read the result back, release;
    (mean seconds per step, per-step seconds).  `warmup` untimed steps first,
    as for the device-timed value (the first graph created beside the resident
    one grows the memory pool once)."""
    import numpy as np
    import torch

    pin = {}
    for name in ("src", "dst", "time"):
        a = getattr(g, name)
        tpin = torch.empty(len(a), dtype=torch.int32, pin_memory=True)
        tpin.numpy().view(np.uint32)[:] = a
        pin[name] = tpin
    cpin = torch.empty(g.n, dtype=torch.int32, pin_memory=True)
    cpin.numpy().view(np.uint32)[:] = g.color
    times = []
    for i in range(-warmup if steps > 0 else 0, steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G2 = tm.tmotif_create_graph(g.n, pin["src"].numpy().view(np.uint32), pin["dst"].numpy().view(np.uint32),
                                    pin["time"].numpy().view(np.uint32), cpin.numpy().view(np.uint32),
                                    g.num_colors, stream=stream)
        tm.tmotif_decide(G2, q.k, q.multiset, seed=seed + 5000 + i, preprocess=preprocess)
        G2.close()
        if i >= 0:
            times.append(time.perf_counter() - t0)
    return (statistics.mean(times) if times else float("nan")), times


def large_leg(tm, stream, dev, costs, rates, steps, warmup, name="large10"):
    """A large-sieve decision: k = 10 on n = 10^7, m = 10^8 (1024 points in
    lane batches of 128), or k = 5 on m = 5*10^8 (32 points, one lane batch of
    32): its own timed steps and layer roofline."""
    g, q = workload(1.0, name)
    G = tm.tmotif_create_graph(g.n, g.src, g.dst, g.time, g.color, g.num_colors, stream=stream)
    total_ms, found, stats, clocks = measure_decision(tm, stream, dev, G, q, steps, warmup, q.seed)
    G.close()
    e2e_s, e2e_steps = e2e_decision(tm, stream, g, q, q.seed, 1)
    work = g.m * q.k * (1 << q.k)
    ms = total_ms / steps
    return {"workload": WORKLOADS[name], "n": g.n, "m": g.m, "k": int(q.k), "steps": steps, "warmup": warmup,
            "ms_per_step": ms, "value": work / (ms / 1e3), "unit": UNIT, "found_all": all(found),
            "clocks": clocks, "roofline": roofline_of(stats, total_ms, costs, rates, None),
            "phases_ms": phases_of(stats, total_ms, steps),
            "e2e": {"ms_per_step": e2e_s * 1e3, "value": work / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": 12 * g.m + 4 * g.n + 4 * q.k, "d2h_bytes_per_step": 8 * (1 << q.k) + 16,
                    "steps": len(e2e_steps), "warmup": 1},
            "gpu_launches": int(stats["launches"])}


def static_roofline(stats, costs, rates):
    """Roofline of the static preprocessing sieve's layer kernel
    (k_static_layer) from the library's events around its launches, on the
    same product-rate bound as the temporal layer kernel."""
    nl = stats["static_launches"]
    if not nl:
        return None
    ms = stats["static_ms"] / nl
    muls = stats["static_gf_muls"] / nl
    tmuls = stats["static_table_muls"] / nl
    builds = stats["static_table_builds"] / nl
    t_min, forms = layer_bound_s(costs, muls - tmuls, tmuls, builds)
    achieved = muls / (ms / 1e3) / 1e9
    peak = muls / t_min / 1e9 if t_min > 0 else None
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G GF(2^64) products/s",
            "frac": achieved / peak if peak else None, "kernel": "k_static_layer (eq. gen-polynomial:1 layer)",
            "ms_per_launch": ms, "gf_muls_per_launch": muls, "launches_per_step": None,
            "form_ms": {k: v * 1e3 for k, v in forms.items()}}


def transit_leg(tm, stream, dev, costs, rates, steps, warmup):
    """The timetable graph at k = 8 (256 points): decisions without and with
    the static preprocessing sieve (Sec. 8.1 (ii)), each with its own timed
    steps; rooflines of the temporal layer kernel in both forms and of the
    static layer kernel."""
    g, q = workload(1.0, "transit")
    G = tm.tmotif_create_graph(g.n, g.src, g.dst, g.time, g.color, g.num_colors, stream=stream)
    work = g.m * q.k * (1 << q.k)
    out = {"workload": WORKLOADS["transit"], "n": g.n, "m": g.m, "k": int(q.k), "steps": steps, "warmup": warmup}
    for name, pre in (("plain", False), ("preprocess", True)):
        total_ms, found, stats, clocks = measure_decision(tm, stream, dev, G, q, steps, warmup, q.seed, pre)
        ms = total_ms / steps
        leg = {"ms_per_step": ms, "value": work / (ms / 1e3), "unit": UNIT, "found_all": all(found),
               "clocks": clocks, "roofline": roofline_of(stats, total_ms, costs, rates, None),
               "phases_ms": phases_of(stats, total_ms, steps)}
        if pre:
            sr = static_roofline(stats, costs, rates)
            if sr:
                sr["launches_per_step"] = stats["static_launches"] / steps
                sr["share_of_step"] = stats["static_ms"] / total_ms
            leg["static_roofline"] = sr
        out[name] = leg
    G.close()
    out["speedup_of_preprocess"] = out["plain"]["ms_per_step"] / out["preprocess"]["ms_per_step"]
    return out


def batch_leg(tm, stream, dev, steps, warmup, count=10_000, seed=4):
    """10,000 small tour graphs: a step is one tmotif_decide_batch call over
    all of them (graphs resident).  The plain form, one tmotif_decide per
    graph back to back, is timed the same way: CUDA events on the shared
    stream around the whole pass."""
    import torch

    import synth

    items = synth.config3_batch(num_graphs=count, seed=seed)
    graphs = [tm.tmotif_create_graph(g.n, g.src, g.dst, g.time, g.color, g.num_colors, stream=stream)
              for g, _ in items]
    queries = [{"k": q.k, "multiset": q.multiset, "seed": q.seed} for _, q in items]
    work = sum(int(g.m) * q.k * (1 << q.k) for g, q in items)
    arcs = sum(int(g.m) for g, _ in items)
    del items
    for _ in range(warmup):
        tm.tmotif_decide_batch(graphs, queries)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    sampler = ClockSampler("")
    sampler.start()
    total_ms = 0.0
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        res = tm.tmotif_decide_batch(graphs, queries)
        b.record(stream)
        torch.cuda.synchronize()
        total_ms += a.elapsed_time(b)
    clocks = sampler.stop()
    with torch.cuda.stream(stream):
        flush.fill_(0x5A)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    plain = [tm.tmotif_decide(G, **q) for G, q in zip(graphs, queries)]
    b.record(stream)
    torch.cuda.synchronize()
    plain_ms = a.elapsed_time(b)
    import numpy as np

    same = all(p.found == r.found and np.array_equal(p.per_point, r.per_point) for p, r in zip(plain, res))
    for G in graphs:
        G.close()
    ms = total_ms / steps
    return {"workload": WORKLOADS["batch"], "graphs": count, "arcs": arcs, "steps": steps, "warmup": warmup,
            "ms_per_step": ms, "value": work / (ms / 1e3), "unit": UNIT, "found": sum(r.found for r in res),
            "clocks": clocks, "timing": "CUDA events on the shared stream around each call (batch) and around "
                                        "the whole pass (plain); L2 flushed before each",
            "plain": {"ms_per_step": plain_ms, "value": work / (plain_ms / 1e3), "results_match": bool(same),
                      "form": "one tmotif_decide per graph, back to back"},
            "speedup_over_plain": plain_ms / ms}


def serving_benchmark(tm, stream, requests=4096, load=0.7, seed=8, sample=256):
    """Config-5 serving: a stream of decide/extract requests (k in [3,10], 30 %
    extract) against one resident power-law graph (n=2e6, m=2e7, 16 colours).

    1. capacity: a seeded sample of the stream, one request at a time, sets
       the Poisson arrival rate at `load` of the plain form's capacity;
    2. plain, live: the requests one at a time in arrival order, each call
       waiting for its arrival (one query per launch sequence);
    3. served, live: the same arrival schedule submitted to the
       continuous-batching server (tmotif_submit / tmotif_poll);
    4. saturated: every request submitted to the server at once; the plain
       form's saturated rate is the requests over the sum of their service
       times in step 2 (back to back, a FIFO queue never idles).
    Every served result is checked against the plain one, point by point for
    decisions and path by path for extractions."""
    import numpy as np

    import synth

    g, reqs = synth.config5_serving(requests=requests, seed=7)
    G = tm.tmotif_create_graph(g.n, g.src, g.dst, g.time, g.color, g.num_colors, stream=stream)
    for q, _ in reqs[:64]:  # tune the launch shapes of every lane width once
        tm.tmotif_decide(G, q.k, q.multiset, seed=q.seed, per_point=False)

    def run_plain(q, ex):
        if ex:
            f, v, t = tm.tmotif_extract(G, q.k, q.multiset, seed=q.seed)
            return (f, None, v.tolist(), t.tolist())
        d = tm.tmotif_decide(G, q.k, q.multiset, seed=q.seed)
        return (d.found, d.per_point.copy(), None, None)

    rng = np.random.default_rng(seed)
    idx = rng.choice(len(reqs), min(sample, len(reqs)), replace=False)
    t0 = time.perf_counter()
    for i in idx:
        run_plain(*reqs[i])
    capacity_est = len(idx) / (time.perf_counter() - t0)
    rate = load * capacity_est
    arrivals = np.cumsum(rng.exponential(1.0 / rate, len(reqs)))
    arrivals -= arrivals[0]

    # plain, live
    plain_res, service, done_plain = [], [], []
    t_start = time.perf_counter()
    for a, (q, ex) in zip(arrivals, reqs):
        wait = a - (time.perf_counter() - t_start)
        if wait > 0:
            time.sleep(wait)
        s0 = time.perf_counter()
        plain_res.append(run_plain(q, ex))
        s1 = time.perf_counter()
        service.append(s1 - s0)
        done_plain.append(s1 - t_start)
    lat_plain = np.array(done_plain) - arrivals

    def serve(schedule):
        srv = tm.tmotif_server_create(0)
        tickets = [None] * len(reqs)
        done_at = [None] * len(reqs)
        served = [None] * len(reqs)
        outstanding = set()
        t0 = time.perf_counter()
        nxt = 0
        while nxt < len(reqs) or outstanding:
            now = time.perf_counter() - t0
            while nxt < len(reqs) and (schedule is None or schedule[nxt] <= now):
                q, ex = reqs[nxt]
                tickets[nxt] = tm.tmotif_submit(srv, G, q.k, q.multiset, is_extract=ex, seed=q.seed)
                outstanding.add(nxt)
                nxt += 1
            for i in list(outstanding):
                r = tm.tmotif_poll(srv, tickets[i], reqs[i][0].k)
                if r is not None:
                    done_at[i] = time.perf_counter() - t0
                    served[i] = r
                    outstanding.discard(i)
            time.sleep(0.0002)
        srv.close()
        return np.array(done_at), served

    done_served, served = serve(arrivals)
    lat_served = done_served - arrivals
    done_sat, served_sat = serve(None)
    G.close()

    def same(pr, sr):
        dec, v, t = sr
        if pr[1] is None:  # extraction
            return dec.found == pr[0] and (not dec.found or (v.tolist() == pr[2] and t.tolist() == pr[3]))
        return dec.found == pr[0] and np.array_equal(dec.per_point, pr[1])

    match = all(same(p, s) for p, s in zip(plain_res, served)) and all(
        same(p, s) for p, s in zip(plain_res, served_sat))

    def summary(lat, done):
        span = float(np.max(done) - arrivals[0])
        return {"queries_per_s": len(reqs) / span, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3)}

    by_k = {}
    for kk in sorted(set(int(q.k) for q, _ in reqs)):
        ix = [i for i, (q, _) in enumerate(reqs) if q.k == kk]
        by_k[kk] = {"n": len(ix), "service_ms": float(np.mean([service[i] for i in ix]) * 1e3),
                    "plain_p50_ms": float(np.percentile(lat_plain[ix], 50) * 1e3),
                    "served_p50_ms": float(np.percentile(lat_served[ix], 50) * 1e3),
                    "plain_p99_ms": float(np.percentile(lat_plain[ix], 99) * 1e3),
                    "served_p99_ms": float(np.percentile(lat_served[ix], 99) * 1e3)}
    sat_plain = len(reqs) / float(np.sum(service))
    sat_served = len(reqs) / float(np.max(done_sat))
    return {"workload": "power-law n=2e6 m=2e7 t<=1000 16 colours; requests k~U{3..10}, 30% extract",
            "requests": len(reqs), "arrival_rate_per_s": rate, "plain_capacity_estimate_per_s": capacity_est,
            "capacity_sample": len(idx), "load": load, "by_k": by_k,
            "plain": summary(lat_plain, np.array(done_plain)), "served": summary(lat_served, done_served),
            "saturated_queries_per_s": {"plain": sat_plain, "served": sat_served,
                                        "served_over_plain": sat_served / sat_plain},
            "timing": "host wall clock, both forms live on the same arrival schedule",
            "results_match": bool(match)}


def run_reference(args):
    """The reference arm: the oracle as it stands on every host core, on the
    same bounded sample of the headline decision as cpu_baseline."""
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    g, q = workload(args.scale)
    for _ in range(args.warmup):
        cpu_baseline(g, q)
    t0 = time.perf_counter()
    r = None
    for _ in range(max(args.steps, 1)):
        r = cpu_baseline(g, q)
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    P = r["cores"]
    value = g.m * q.k * P / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOADS["mid"] if args.scale == 1.0 else f"{WORKLOAD} scaled x{args.scale}",
                       "sample": r["sample"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": P, "nproc": r["nproc"], "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "paper": PAPER}
    print(json.dumps(line))
    return 0


def run_leg(line, name, fn, tm=None):
    """Run one extra workload; a failure is recorded in the line, not raised.
    With tm, the leg also reports the most device memory the library's pool
    held during it (peak_hbm_bytes)."""
    try:
        if tm is not None:
            tm.tmotif_memory_stats(reset=True)
        line[name] = fn()
        if tm is not None:
            line[name]["peak_hbm_bytes"] = tm.tmotif_memory_stats()["used_high"]
    except Exception as e:  # noqa: BLE001 -- the headline line must still print
        import traceback

        line[name] = {"error": f"{type(e).__name__}: {e}",
                      "where": traceback.format_exc(limit=4).splitlines()[-6:]}


def run_ours(args):
    import torch

    import paper_2001_07158_gb300 as tm

    rank, local, world = dist_env()
    if world > 1:
        import torch.distributed as dist

    torch.cuda.set_device(local)  # before the process group, so each rank's NCCL uses its own GPU
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    if args.workload == "batch":
        return run_batch(args, tm, stream, dev, rank, world)
    rates = probe_rates(tm)
    costs = table_costs(rates)
    g, q = workload(args.scale, args.workload)
    seed = q.seed + 7919 * rank
    work_units = g.m * q.k * (1 << q.k)

    tm.tmotif_memory_stats(reset=True)
    G = tm.tmotif_create_graph(g.n, g.src, g.dst, g.time, g.color, g.num_colors, stream=stream)
    if args.layer_shape:
        chunk, variant = (int(x) for x in args.layer_shape.split(","))
        L = 4
        while L < 128 and L < (1 << q.k):
            L *= 2
        tm.tmotif_set_layer_shape(G, L, chunk, variant)
    total_ms, found, stats, clocks = measure_decision(tm, stream, dev, G, q, args.steps, args.warmup, seed,
                                                      args.preprocess, world)
    t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * work_units * args.steps / (total_ms / 1e3)
    traffic = (LAYER_TRAFFIC["bytes_per_launch"]
               if LAYER_TRAFFIC["source_sha"] == source_sha() and args.workload == "mid" and args.scale == 1.0
               else None)
    roofline = roofline_of(stats, total_ms, costs, rates, traffic)

    e2e_s, e2e_steps = e2e_decision(tm, stream, g, q, seed, args.e2e_steps, args.preprocess)
    e2e_t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
    if world > 1:
        torch.distributed.all_reduce(e2e_t, op=torch.distributed.ReduceOp.MAX)
    e2e = {"value": world * work_units / float(e2e_t.item()), "unit": UNIT,
           "h2d_bytes_per_step": 12 * g.m + 4 * g.n + 4 * q.k,
           "d2h_bytes_per_step": 8 * (1 << q.k) + 16, "ms_per_step": float(e2e_t.item()) * 1e3,
           "steps": len(e2e_steps), "warmup": 1 if e2e_steps else 0,
           "steps_ms": [round(x * 1e3, 3) for x in e2e_steps]}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "n": g.n, "m": g.m, "k": int(q.k), "points": 1 << q.k,
                       "preprocess": bool(args.preprocess),
                       "multiset": [int(c) for c in q.multiset], "found_all": all(found),
                       "l2": "flushed between timed steps (256 MB write, outside the step events)",
                       "parallelism": f"replicas x{world} (independent queries)"},
            "clocks": clocks, "roofline": roofline, "e2e": e2e,
            "gpu_launches": int(stats["launches"]), "phases_ms": phases_of(stats, total_ms, args.steps),
            "paper": PAPER,
            "peak_hbm_bytes": tm.tmotif_memory_stats()["used_high"]}
    G.close()
    legs = legs_of(args) if (world == 1 and args.workload == "mid" and args.scale == 1.0) else set()
    if rank == 0 and "cpu" in legs:
        run_leg(line, "cpu_baseline", lambda: cpu_baseline(g, q))
    del g
    leg_steps, leg_warmup = max(3, min(args.steps, 5)), 3
    for name in ("large10", "large5"):
        if name in legs:
            run_leg(line, name, lambda: large_leg(tm, stream, dev, costs, rates, leg_steps, leg_warmup, name), tm)
    if "transit" in legs:
        run_leg(line, "transit", lambda: transit_leg(tm, stream, dev, costs, rates, leg_steps, leg_warmup), tm)
    if "batch" in legs:
        run_leg(line, "batch", lambda: batch_leg(tm, stream, dev, leg_steps, leg_warmup), tm)
    if "serving" in legs:
        run_leg(line, "serving", lambda: serving_benchmark(tm, stream, requests=args.serving_requests), tm)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_batch(args, tm, stream, dev, rank, world):
    """--workload batch: the batched call over the small graphs as the
    headline (per rank, another seed)."""
    import torch

    count = max(1, int(10_000 * args.scale))
    if world > 1:
        torch.distributed.barrier()
    leg = batch_leg(tm, stream, dev, args.steps, args.warmup, count=count, seed=4 + 1000 * rank)
    t = torch.tensor([leg["ms_per_step"]], dtype=torch.float64, device=dev)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    ms = float(t.item())
    value = world * leg["value"] * leg["ms_per_step"] / ms
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOADS["batch"], "graphs": count, "arcs": leg["arcs"], "found": leg["found"],
                       "l2": "flushed between timed steps", "parallelism": f"replicas x{world}"},
            "clocks": leg["clocks"], "plain": leg["plain"]}
    if rank == 0:
        print(json.dumps(line))
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
