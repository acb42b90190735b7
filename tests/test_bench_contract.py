"""The JSON line of `bench.py --impl reference` (the FP64 oracle timed on the
host cores): one line with the keys every bench line carries, on a small
workload so that it runs on the CPU in seconds."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--N", "1500", "--n", "64",
           "--w", "6", "--Q", "12", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["N"] == 1500 and d["config"]["n"] == 64 and "workload" in d["config"]


def test_latency_summary():
    sys.path.insert(0, ROOT)
    import bench

    # 1,000 requests arriving 1 ms apart, each done 2 ms after arrival (the
    # last one 12 ms), admitted 0.5 ms after arrival
    comp = [{"arrival_ns": i * 1_000_000, "admit_ns": i * 1_000_000 + 500_000,
             "done_ns": i * 1_000_000 + (12_000_000 if i == 999 else 2_000_000), "status": 0} for i in range(1000)]
    s = bench.latency_summary(comp)
    assert s["completed"] == 1000 and s["failed"] == 0 and s["all_ok"]
    assert s["p50_ms"] == 2.0 and s["p99_ms"] == 2.0 and 2.0 < s["p999_ms"] < 12.0
    assert s["queue_p50_ms"] == 0.5
    assert abs(s["throughput_qps"] - 1000 / 1.011) < 1e-6
    # a timed-out request (status 4) and a failed one (status 2) enter neither
    # the throughput nor the latencies; the last request (12 ms) times out
    comp[3]["status"] = 2
    comp[999]["status"] = 4
    s = bench.latency_summary(comp)
    assert s["completed"] == 1000 and s["succeeded"] == 998 and s["failed"] == 2 and s["timed_out"] == 1
    assert not s["all_ok"]
    assert s["p999_ms"] == 2.0
    assert abs(s["throughput_qps"] - 998 / 1.000) < 1e-6
    none = bench.latency_summary([dict(comp[0], status=4)])
    assert none["succeeded"] == 0 and none["throughput_qps"] == 0.0 and none["p50_ms"] is None


def test_candidate_mode_config_and_prefix_accounting(monkeypatch):
    # the line's parallelism names the sharding; in candidate mode the bound
    # tile and the seeds run twice per step (once for the thresholds), and the
    # rates count that work twice over the shard's own candidates
    import argparse

    sys.path.insert(0, ROOT)
    import bench

    a = argparse.Namespace(data="random_walk", k=1, N=100_000, n=256, w=25, Q=1000, p=1, seed=2, dtw_path=0,
                           shard="candidates")
    assert "candidates sharded over 4 GPU(s)" in bench.workload_config(a, 4)["parallelism"]
    a.shard = "queries"
    assert "queries sharded over 4 GPU(s)" in bench.workload_config(a, 4)["parallelism"]
    monkeypatch.setattr(bench, "alu_peak_tops", lambda peaks: (40.0, "derived"))
    stages = ("lb_keogh", "lb_improved", "dtw", "seed_dtw")
    prof = {s: {"ms": 0.0, "launches": 0} for s in stages}
    prof["lb_keogh"] = {"ms": 2.0, "launches": 4}  # 2 steps x 2 runs, 0.5 ms each
    prof["seed_dtw"] = {"ms": 0.2, "launches": 4}
    stats = {"seed_cells": 1e9}
    one = bench.stage_rates(prof, a, 2, {}, stats, prefix_runs=1)
    two = bench.stage_rates(prof, a, 2, {}, stats, prefix_runs=2)
    assert abs(two["lb_keogh_tile"]["Top_s"] - 2 * one["lb_keogh_tile"]["Top_s"]) < 1e-9
    assert abs(two["seed_dtw"]["cells_per_s"] - 2 * one["seed_dtw"]["cells_per_s"]) < 1e-3
    roof = bench.roofline(prof, a, 2, {}, stats, prefix_runs=2)
    # per launch: Q N d terms of 3 ops (d = n / 8) in 0.5 ms
    assert roof["kernel"] == "k_lbk_tile"
    assert abs(roof["achieved"] - 1000 * 100_000 * 32 * 3 / 1e12 / 0.5e-3) < 1e-6


def test_no_gc_pauses_and_restores_the_collector():
    import gc

    sys.path.insert(0, ROOT)
    import bench

    assert gc.isenabled()
    with bench.no_gc():
        assert not gc.isenabled()
    assert gc.isenabled()
