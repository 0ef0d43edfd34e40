"""Host-side parts of the benchmark (CPU only): the reference arm's JSON line,
rank handling under a launcher, the speed-of-light model and the source hash
that guards the committed DRAM traffic figure."""
import json
import os
import shutil
import subprocess
import sys
import time
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _run(args, env_extra=None):
    env = dict(os.environ)
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    env.pop("LOCAL_RANK", None)
    if env_extra:
        env.update(env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                          env=env, cwd=ROOT, timeout=600)


def test_reference_arm_line():
    r = _run(["--impl", "reference", "--scale", "0.01", "--steps", "1", "--warmup", "0"])
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "paper"):
        assert key in d, key
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["cores"] == min(os.cpu_count(), 64) and d["cpu_baseline"]["nproc"] == os.cpu_count()
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_reference_arm_other_ranks_exit_quietly():
    r = _run(["--impl", "reference", "--scale", "0.01", "--steps", "1", "--warmup", "0"],
             {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_speed_of_light_model():
    # costs solved from the probe's rates reproduce them: a round of the table
    # probe (one build, 64 or 128 lookups) takes 64 / R64 or 128 / R128
    rates = {"reg": 1.2e11, "table64": 2.5e11, "table128": 2.8e11}
    c = bench.table_costs(rates)
    assert c["build"] / 64 + c["lookup"] == pytest.approx(1 / rates["table64"])
    assert c["build"] / 128 + c["lookup"] == pytest.approx(1 / rates["table128"])
    assert c["reg"] == pytest.approx(1 / rates["reg"])
    # the bound is the larger form time, and each form time scales with its work
    t, forms = bench.layer_bound_s(c, reg=1e6, tab=1e8, builds=1e6)
    assert t == max(forms.values()) and all(v > 0 for v in forms.values())
    t2, forms2 = bench.layer_bound_s(c, reg=2e6, tab=2e8, builds=2e6)
    for k in forms:
        assert forms2[k] == pytest.approx(2 * forms[k])
    _, only_reg = bench.layer_bound_s(c, reg=rates["reg"], tab=0, builds=0)
    assert only_reg["register"] == pytest.approx(1.0) and only_reg["table"] == 0
    # a table rate that does not fall with fewer lanes per table cannot give a
    # negative build cost
    c2 = bench.table_costs({"reg": 1e11, "table64": 3e11, "table128": 2.9e11})
    assert c2["build"] == 0 and c2["lookup"] > 0


def test_default_legs_and_switches():
    a = bench.parse_args([])
    assert bench.legs_of(a) == {"large10", "large5", "transit", "batch", "serving", "cpu"} and a.serving_requests == 4096
    a = bench.parse_args(["--no-serving", "--no-cpu-baseline"])
    assert bench.legs_of(a) == {"large10", "large5", "transit", "batch"}
    assert bench.legs_of(bench.parse_args(["--legs", ""])) == set()


def test_source_hash_ignores_comments_only(tmp_path, monkeypatch):
    src = os.path.join(ROOT, "paper_2001_07158_gb300", "csrc")
    dst = tmp_path / "paper_2001_07158_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in ("layer.cuh", "gf64.cuh", "sieve.cu"):
        shutil.copy(os.path.join(src, f), dst / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    base = bench.source_sha()
    assert base == bench.source_sha()
    p = dst / "layer.cuh"
    text = p.read_text()
    p.write_text("// an added comment line\n" + text.replace("namespace tmo {", "namespace tmo {  /* note */", 1))
    assert bench.source_sha() == base
    p.write_text(text.replace("namespace tmo {", "namespace tmo {\nstatic const int added_code = 1;", 1))
    assert bench.source_sha() != base


class _FakeDecision:
    def __init__(self, found, per_point):
        self.found = found
        self.per_point = per_point
        self.sieve_sum = int(np.bitwise_xor.reduce(per_point)) if len(per_point) else 0
        self.ms = 0.0


class _FakeLibrary:
    """Stands in for the binding in the serving leg: every request's result
    is a function of its query, and a request takes 0.1 ms per point of k
    (the server completes it that long after submission)."""

    def __init__(self, corrupt_ticket=None):
        self.corrupt = corrupt_ticket
        self.next = 1
        self.subs = {}

    @staticmethod
    def _result(k, ms, seed):
        rng = np.random.default_rng([int(seed) % (2**32), int(k)] + [int(c) for c in ms])
        return rng.integers(0, 2**63, 1 << k, dtype=np.uint64)

    def tmotif_create_graph(self, *a, **kw):
        return types.SimpleNamespace(close=lambda: None)

    def tmotif_decide(self, G, k, ms, seed=1, per_point=True):
        time.sleep(1e-4 * k)
        return _FakeDecision(True, self._result(k, ms, seed))

    def tmotif_extract(self, G, k, ms, seed=1):
        time.sleep(1e-4 * k)
        v = self._result(k, ms, seed)[:k].astype(np.uint32)
        return True, v, v[:k - 1]

    def tmotif_server_create(self, budget):
        return types.SimpleNamespace(close=lambda: None)

    def tmotif_submit(self, srv, G, k, ms, is_extract=False, seed=1):
        t = self.next
        self.next += 1
        self.subs[t] = (time.perf_counter() + 1e-4 * k, k, list(ms), seed, is_extract)
        return t

    def tmotif_poll(self, srv, t, k):
        due, k, ms, seed, ex = self.subs[t]
        if time.perf_counter() < due:
            return None
        pp = self._result(k, ms, seed)
        if t == self.corrupt:
            pp = pp ^ np.uint64(1)
        v = pp[:k].astype(np.uint32)
        return _FakeDecision(True, pp), v, v[:k - 1]


def _small_serving(monkeypatch):
    import synth

    real = synth.config5_serving
    monkeypatch.setattr(synth, "config5_serving", lambda requests, seed: real(n=2000, m=20000, requests=requests,
                                                                                seed=seed))


def test_serving_leg_summary_on_a_fake_library(monkeypatch):
    _small_serving(monkeypatch)
    out = bench.serving_benchmark(_FakeLibrary(), None, requests=48, sample=16)
    assert out["requests"] == 48 and out["results_match"]
    assert out["arrival_rate_per_s"] == pytest.approx(out["load"] * out["plain_capacity_estimate_per_s"])
    for form in ("plain", "served"):
        s = out[form]
        assert s["queries_per_s"] > 0 and 0 <= s["p50_ms"] <= s["p99_ms"]
    sat = out["saturated_queries_per_s"]
    assert sat["plain"] > 0 and sat["served"] > 0
    assert sat["served_over_plain"] == pytest.approx(sat["served"] / sat["plain"])
    assert sum(v["n"] for v in out["by_k"].values()) == 48


def test_serving_leg_detects_a_wrong_served_result(monkeypatch):
    _small_serving(monkeypatch)
    out = bench.serving_benchmark(_FakeLibrary(corrupt_ticket=5), None, requests=24, sample=8)
    assert not out["results_match"]


def test_failed_leg_is_recorded_not_raised():
    line = {}

    def boom():
        raise ValueError("no such workload")

    bench.run_leg(line, "leg", boom)
    assert line["leg"]["error"].startswith("ValueError") and line["leg"]["where"]
    bench.run_leg(line, "ok", lambda: {"value": 1})
    assert line["ok"] == {"value": 1}


def test_phases_split_the_step():
    import bench

    stats = {"prep_ms": 2.0, "coef_ms": 1.0, "layer_ms": 10.0, "other_ms": 0.5, "static_ms": 0.4}
    ph = bench.phases_of(stats, 14.0, 2)
    assert ph == {"prep": 1.0, "coef": 0.5, "layer": 5.0, "other": 0.25, "static": 0.2, "unprofiled": 0.05}
    assert abs(sum(ph.values()) - 7.0) < 1e-9
    assert bench.phases_of(stats, 14.0, 0) is None
