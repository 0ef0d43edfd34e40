#!/usr/bin/env python3
"""Benchmark of the temporal path-motif sieve on one GB300 (or N replicas).

Workload: the mid-size decision of the benchmark suite -- a power-law
out-degree temporal graph (exponent 2.1, n = 10^6, m = 10^7 edges, timestamps
uniform in [1, 1000], 16 colours Zipf(1.0)) with a k = 6 multiset query (one
colour twice), 2^6 = 64 sieve points, exact GF(2^64) arithmetic.  A step is one
full decision on the resident graph: per-query arc filter and checkpoint
build, sieve coefficients, the k-1 generating-function layers, the sieve sum.

Metric: edge-steps/s = m * k * 2^k / (time of one decision).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 it runs under torchrun, one rank per GPU; every rank decides its own
query (another seed) on its own replica of the graph -- the sieve points of
different queries are independent, so there is no data-path collective
("weak" scaling); ranks meet only at the timing barrier.
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

# Speed of light of the layer kernel, from GB300 unit counts at the maximum SM
# clock (152 SMs, 2070 MHz) and per-product costs measured by ncu on the
# library's register-resident probe (tmotif_gf_probe methods 0-2).  A launch's
# lower-bound time is the largest of three pipe times for its work:
#   shared memory, 1 wavefront (128 B) per clock per SM: a table product
#     reads 16 eight-byte entries (1 wavefront); a table build writes 2 KB
#     (16 wavefronts);
#   ALU pipe, 64 lanes per clock per SM: 39.6 ALU instructions per table
#     product plus 1059 per table build (fitted to the probe at 64 and 128
#     lanes per table: 56.1 and 47.8 per product), 92.6 per register product
#     (probe counts less about 3-4 of probe loop work);
#   FMA pipe: 9.28 sub-partition cycles per register product (4 per SM).
SMS = 152
SM_HZ = 2.070e9
ALU_PER_REG, ALU_PER_TAB, ALU_PER_BUILD = 92.6, 39.6, 1059.0
WF_PER_TAB, WF_PER_BUILD = 1.0, 16.0
FMA_CYC_PER_REG = 9.28


def layer_bound_s(reg, tab, builds):
    """Lower-bound seconds of one layer launch with `reg` register products,
    `tab` table products and `builds` table builds."""
    t_smem = (tab * WF_PER_TAB + builds * WF_PER_BUILD) / (SMS * SM_HZ)
    t_alu = (reg * ALU_PER_REG + tab * ALU_PER_TAB + builds * ALU_PER_BUILD) / (SMS * 64 * SM_HZ)
    t_fma = reg * FMA_CYC_PER_REG / (SMS * 4 * SM_HZ)
    return max(t_smem, t_alu, t_fma), {"smem": t_smem, "alu": t_alu, "fma": t_fma}


# DRAM traffic of one layer launch from an ncu capture, valid only for the
# layer-kernel sources it was taken on (source_sha() below, first 16 hex):
# a timed-decision layer of the default workload, full size, one-pass dram
# counters
LAYER_TRAFFIC = {"source_sha": "d47a2aedf1086717", "bytes_per_launch": 1125220352 + 399725824}


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--serving-requests", type=int, default=256)
    p.add_argument("--scale", type=float, default=1.0,
                   help="scale n and m of the workload (profiling captures of a smaller case)")
    p.add_argument("--workload", choices=sorted(WORKLOADS), default="mid",
                   help="mid: the default decision (n=1e6, m=1e7, k=6); large5 / large10: power-law "
                        "n=1e7 with m=5e8, k=5 / m=1e8, k=10; batch: 10,000 small tour graphs in one "
                        "batched call (k in 5..8); transit: a timetable graph for --preprocess")
    p.add_argument("--preprocess", action="store_true", help="static preprocessing sieve before each decision")
    return p.parse_args()


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


def cpu_baseline(g, q, points=None):
    """The oracle as it stands (plain C, OpenMP over sieve points) on the host
    cores, on a bounded sample of the same decision: `points` of the 64 sieve
    points (one point per thread)."""
    import oracle

    cores = os.cpu_count() or 1
    P = points or max(1, min(cores, 16))
    t0 = time.perf_counter()
    oracle.decide(g.n, g.src, g.dst, g.time, g.color, g.num_colors, q.k, q.multiset, seed=q.seed, point_begin=0,
                  point_end=P, nthreads=min(P, cores))
    dt = time.perf_counter() - t0
    return {"value": g.m * q.k * P / dt, "unit": UNIT, "cores": min(P, cores), "kind": "oracle",
            "sample": f"{P} of the {1 << q.k} sieve points of the same decision ({dt:.1f} s)"}


def serving_benchmark(tm, stream, requests=128, load=0.7, seed=8):
    """Config-5 serving: a stream of decide/extract requests (k in [3,10], 30 %
    extract) against one resident power-law graph (n=2e6, m=2e7, 16 colours).

    plain: requests one at a time, one query per launch sequence (FIFO);
    their measured service times set the Poisson arrival rate at `load` of
    the plain form's capacity and give its latencies by replaying the queue.
    served: the same arrival schedule submitted to the continuous-batching
    server (tmotif_submit / tmotif_poll), timed live.  Every served result
    is checked against the plain one."""
    import numpy as np

    import synth

    g, reqs = synth.config5_serving(requests=requests, seed=7)
    G = tm.tmotif_create_graph(g.n, g.src, g.dst, g.time, g.color, g.num_colors, stream=stream)
    warm = reqs[0][0]
    tm.tmotif_decide(G, warm.k, warm.multiset, seed=warm.seed)
    plain_res, service = [], []
    for q, ex in reqs:
        t0 = time.perf_counter()
        if ex:
            f, v, t = tm.tmotif_extract(G, q.k, q.multiset, seed=q.seed)
            plain_res.append((f, None, v.tolist(), t.tolist()))
        else:
            d = tm.tmotif_decide(G, q.k, q.multiset, seed=q.seed, per_point=False)
            plain_res.append((d.found, d.sieve_sum, None, None))
        service.append(time.perf_counter() - t0)
    capacity = len(reqs) / sum(service)
    rate = load * capacity
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, len(reqs)))
    arrivals -= arrivals[0]
    done_plain, t_free = [], 0.0
    for a, s_ in zip(arrivals, service):
        t_free = max(a, t_free) + s_
        done_plain.append(t_free)
    lat_plain = np.array(done_plain) - arrivals

    srv = tm.tmotif_server_create(0)
    tickets = [None] * len(reqs)
    done_at = [None] * len(reqs)
    served = [None] * len(reqs)
    t_start = time.perf_counter()
    nxt = 0
    while any(d is None for d in done_at):
        now = time.perf_counter() - t_start
        while nxt < len(reqs) and arrivals[nxt] <= now:
            q, ex = reqs[nxt]
            tickets[nxt] = tm.tmotif_submit(srv, G, q.k, q.multiset, is_extract=ex, seed=q.seed)
            nxt += 1
        for i in range(nxt):
            if done_at[i] is None:
                r = tm.tmotif_poll(srv, tickets[i], reqs[i][0].k)
                if r is not None:
                    done_at[i] = time.perf_counter() - t_start
                    served[i] = r
        time.sleep(0.0002)
    srv.close()
    lat_served = np.array(done_at) - arrivals

    # saturated: every request submitted at once
    srv = tm.tmotif_server_create(0)
    t0 = time.perf_counter()
    sat = [tm.tmotif_submit(srv, G, q.k, q.multiset, is_extract=ex, seed=q.seed) for q, ex in reqs]
    pending = set(range(len(reqs)))
    while pending:
        for i in list(pending):
            if tm.tmotif_poll(srv, sat[i], reqs[i][0].k) is not None:
                pending.discard(i)
        time.sleep(0.0002)
    t_sat = time.perf_counter() - t0
    srv.close()
    G.close()
    match = True
    for (q, ex), pr, sr in zip(reqs, plain_res, served):
        dec, v, t = sr
        if ex:
            match &= dec.found == pr[0] and (not dec.found or (v.tolist() == pr[2] and t.tolist() == pr[3]))
        else:
            match &= dec.found == pr[0] and dec.sieve_sum == pr[1]

    def summary(lat, done):
        span = max(done) - arrivals[0]
        return {"queries_per_s": len(reqs) / span, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3)}

    by_k = {}
    for kk in sorted(set(int(q.k) for q, _ in reqs)):
        idx = [i for i, (q, _) in enumerate(reqs) if q.k == kk]
        by_k[kk] = {"n": len(idx), "service_ms": float(np.mean([service[i] for i in idx]) * 1e3),
                    "plain_p50_ms": float(np.percentile(lat_plain[idx], 50) * 1e3),
                    "served_p50_ms": float(np.percentile(lat_served[idx], 50) * 1e3),
                    "plain_max_ms": float(np.max(lat_plain[idx]) * 1e3),
                    "served_max_ms": float(np.max(lat_served[idx]) * 1e3)}
    return {"workload": "power-law n=2e6 m=2e7 t<=1000 16 colours; requests k~U{3..10}, 30% extract",
            "requests": len(reqs), "arrival_rate_per_s": rate, "plain_capacity_per_s": capacity,
            "by_k": by_k,
            "plain": summary(lat_plain, done_plain), "served": summary(lat_served, done_at),
            "saturated_queries_per_s": {"plain": capacity, "served": len(reqs) / t_sat},
            "results_match": bool(match)}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    g, q = workload(args.scale)
    cores = os.cpu_count() or 1
    P = max(1, min(cores, 8))
    for _ in range(args.warmup):
        cpu_baseline(g, q, P)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = cpu_baseline(g, q, P)
    dt = (time.perf_counter() - t0) / args.steps
    value = g.m * q.k * P / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": r["sample"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ours(args):
    import numpy as np
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
    g, q = workload(args.scale, args.workload)
    seed = q.seed + 7919 * rank
    work_units = g.m * q.k * (1 << q.k)

    G = tm.tmotif_create_graph(g.n, g.src, g.dst, g.time, g.color, g.num_colors, stream=stream)
    for i in range(args.warmup):
        tm.tmotif_decide(G, q.k, q.multiset, seed=seed + i, preprocess=args.preprocess)

    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
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
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xFF)
            starts[i].record(stream)
        d = tm.tmotif_decide(G, q.k, q.multiset, seed=seed + 1000 + i, per_point=False,
                             preprocess=args.preprocess)
        ends[i].record(stream)
        found.append(d.found)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    stats = tm.tmotif_get_stats(G)
    tm.tmotif_set_profiling(G, False)
    total_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * work_units * args.steps / (total_ms / 1e3)

    # roofline of the dominant kernel (the layer kernel), from the library's
    # CUDA events around every layer launch during the timed region: achieved
    # GF(2^64) products per second against the speed-of-light rate of the
    # same product mix (layer_bound_s)
    nl = max(stats["layer_launches"], 1)
    layer_ms = stats["layer_ms"] / nl
    muls = stats["layer_gf_muls"] / nl
    tmuls = stats["layer_table_muls"] / nl
    builds = stats["layer_table_builds"] / nl
    t_min, pipes = layer_bound_s(muls - tmuls, tmuls, builds)
    achieved = muls / (layer_ms / 1e3) / 1e9
    peak = muls / t_min / 1e9
    sha = source_sha()
    traffic = (LAYER_TRAFFIC["bytes_per_launch"]
               if LAYER_TRAFFIC["source_sha"] == sha and args.workload == "mid" and args.scale == 1.0 else None)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G GF(2^64) products/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "k_layer (eq. gen-polynomial:3 layer)",
                "model": "integer/shared-memory pipes from unit counts at 2070 MHz; binding pipe: "
                         + max(pipes, key=pipes.get),
                "pipe_ms": {k: v * 1e3 for k, v in pipes.items()}, "layer_ms_per_launch": layer_ms,
                "gf_muls_per_launch": muls, "table_muls_per_launch": tmuls, "table_builds_per_launch": builds,
                "algorithmic_bytes_per_launch": stats["layer_bytes"] / nl,
                "achieved_hbm_gbs": stats["layer_bytes"] / nl / (layer_ms / 1e3) / 1e9,
                "layer_share_of_step": stats["layer_ms"] / total_ms if total_ms else None}

    # end to end through the C ABI with host buffers: upload + build the graph,
    # decide, read the result back, release
    pin = {}
    for name in ("src", "dst", "time"):
        a = getattr(g, name)
        tpin = torch.empty(len(a), dtype=torch.int32, pin_memory=True)
        tpin.numpy().view(np.uint32)[:] = a
        pin[name] = tpin
    cpin = torch.empty(g.n, dtype=torch.int32, pin_memory=True)
    cpin.numpy().view(np.uint32)[:] = g.color
    e2e_times = []
    for i in range(args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G2 = tm.tmotif_create_graph(g.n, pin["src"].numpy().view(np.uint32), pin["dst"].numpy().view(np.uint32),
                                    pin["time"].numpy().view(np.uint32), cpin.numpy().view(np.uint32),
                                    g.num_colors, stream=stream)
        d2 = tm.tmotif_decide(G2, q.k, q.multiset, seed=seed + 5000 + i, preprocess=args.preprocess)
        G2.close()
        e2e_times.append(time.perf_counter() - t0)
    e2e_t = torch.tensor([statistics.mean(e2e_times) if e2e_times else float("nan")], dtype=torch.float64,
                         device=dev)
    if world > 1:
        torch.distributed.all_reduce(e2e_t, op=torch.distributed.ReduceOp.MAX)
    e2e = {"value": world * work_units / float(e2e_t.item()), "unit": UNIT,
           "h2d_bytes_per_step": 12 * g.m + 4 * g.n + 4 * q.k,
           "d2h_bytes_per_step": 8 * (1 << q.k) + 16, "ms_per_step": float(e2e_t.item()) * 1e3}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "n": g.n, "m": g.m, "k": int(q.k), "points": 1 << q.k,
                       "preprocess": bool(args.preprocess),
                       "multiset": [int(c) for c in q.multiset], "found_all": all(found),
                       "l2": "flushed between timed steps (256 MB write, outside the step events)",
                       "parallelism": f"replicas x{world} (independent queries)"},
            "clocks": clocks, "roofline": roofline, "e2e": e2e,
            "gpu_launches": int(stats["launches"])}
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "mid":
        line["cpu_baseline"] = cpu_baseline(g, q)
    if rank == 0 and not args.no_serving and args.workload == "mid":
        line["serving"] = serving_benchmark(tm, stream, requests=args.serving_requests)
    if rank == 0:
        print(json.dumps(line))
    G.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_batch(args, tm, stream, dev, rank, world):
    """Batched decisions over many small graphs: a step is one
    tmotif_decide_batch call over all of them (the graphs resident)."""
    import torch

    import synth

    count = max(1, int(10_000 * args.scale))
    items = synth.config3_batch(num_graphs=count, seed=4 + 1000 * rank)
    graphs = [tm.tmotif_create_graph(g.n, g.src, g.dst, g.time, g.color, g.num_colors, stream=stream)
              for g, _ in items]
    queries = [{"k": q.k, "multiset": q.multiset, "seed": q.seed} for _, q in items]
    work = sum(int(g.m) * q.k * (1 << q.k) for g, q in items)
    arcs = sum(int(g.m) for g, _ in items)
    for _ in range(args.warmup):
        tm.tmotif_decide_batch(graphs, queries)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    sampler = ClockSampler("")
    sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    total_ms = 0.0
    found = 0
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        res = tm.tmotif_decide_batch(graphs, queries)
        total_ms += res[0].ms  # device time of the call (events on the shared stream)
        found = sum(r.found for r in res)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    # the plain form: one tmotif_decide per graph, back to back (same results)
    t0 = time.perf_counter()
    plain = [tm.tmotif_decide(G, per_point=False, **q) for G, q in zip(graphs, queries)]
    torch.cuda.synchronize()
    plain_ms = (time.perf_counter() - t0) * 1e3
    same = all(p.found == r.found and p.sieve_sum == r.sieve_sum for p, r in zip(plain, res))
    t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    total_ms = float(t.item())
    value = world * work * args.steps / (total_ms / 1e3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOADS["batch"], "graphs": count, "arcs": arcs, "found": found,
                       "l2": "flushed between timed steps", "parallelism": f"replicas x{world}"},
            "clocks": clocks,
            "plain": {"ms_per_step": plain_ms, "value": world * work / (plain_ms / 1e3), "results_match": same,
                      "form": "one tmotif_decide per graph, sequential"}}
    if rank == 0:
        print(json.dumps(line))
    for G in graphs:
        G.close()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
