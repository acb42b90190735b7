#!/usr/bin/env python3
"""Benchmark of the exact k-NN DTW retrieval cascade (LB_Keogh -> LB_Improved
-> band DTW_p with early abandoning) on one or more GB300s.

Workload (default): 100,000 seeded random walks x_1 = 0, x_t = x_{t-1} + N(0,1)
of length n = 256 (fp32, resident in HBM), band w = 25 (10 %), 1,000 fresh
queries per step from a distinct seed stream, 1-NN under DTW_1 (the measure
of the paper's experiments, Sec. 10).  A step is one knn_search call over the
whole query batch: envelopes, LB_Keogh of every pair, seed DTWs,
LB_Improved of the LB_Keogh survivors, DTW of the LB_Improved survivors and
the ordered top-k.  The same step under DTW_2 is reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --data shapes --N 50000 --n 1024 --Q 500 --w 102   # shape-like series
  python bench.py --workload batched   # mixed-length batches through the index
  python bench.py --workload serve     # Poisson arrivals through the request server
  python bench.py --workload triangle  # App. B: triangle-inequality violations
  python bench.py --workload classify  # App. C: 1-NN classification, DTW_1/2/4/inf

Under torchrun each rank holds the whole database and runs its own batch of
queries (weak scaling; the only collectives are the timing barrier and the
max-over-ranks of the elapsed time).  `--impl reference` times the FP64 CPU
oracle (the paper's Algorithm 3 scan, in C, on all host cores) on a bounded
sample of the same workload.
"""

from __future__ import annotations

import argparse
import contextlib
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "exact 1-NN DTW queries/s (LB_Improved cascade)"
L2_BYTES = 129 * 2**20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--N", type=int, default=100_000)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--w", type=int, default=25)
    ap.add_argument("--Q", type=int, default=1000)
    ap.add_argument("--k", type=int, default=1)
    ap.add_argument("--p", type=int, default=1)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--data", choices=["random_walk", "shapes"], default="random_walk",
                    help="retrieval: database and query generator (shapes: z-normalised shape-like series)")
    ap.add_argument("--seeds", type=int, default=0, help="seed DTWs per query (0: library default)")
    ap.add_argument("--parts", type=int, default=0, help="piecewise-sum parts (0: default n/8, -1: off)")
    ap.add_argument("--dtw-path", type=int, default=0, help="DTW kernel: 0 auto, 1 thread per pair, 2 warp per pair, "
                    "3 main stage on two 16-lane groups per warp, 4 thread per pair in row phases of 64 rows")
    ap.add_argument("--filter-path", type=int, default=0,
                    help="LB_Keogh/LB_Improved filter kernel: 0 auto, 1 one warp per pair, 2 batches of eight pairs")
    ap.add_argument("--lb-abandon", type=int, default=0,
                    help="1: early abandoning inside the LB sums (streamed rows of series longer than 256)")
    ap.add_argument("--no-p2", action="store_true", help="skip the DTW_2 side measurement")
    ap.add_argument("--shard", choices=["queries", "candidates"], default="queries",
                    help="N > 1: every GPU holds the database and searches its own queries (weak scaling), "
                         "or holds a candidate range and searches every query, with the seeds' thresholds "
                         "exchanged and the top-k lists merged (strong scaling)")
    ap.add_argument("--no-extra", action="store_true",
                    help="default workload only: skip the bounded batched and serving runs added to its line")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the CPU baseline sample")
    ap.add_argument("--workload", choices=["retrieval", "batched", "serve", "triangle", "classify"],
                    default="retrieval",
                    help="retrieval: one length, one knn_search per step (default); batched: mixed-length "
                         "batches against length buckets through the index")
    ap.add_argument("--bucket-N", type=int, default=20_000, help="batched: series per length bucket")
    ap.add_argument("--batch-Q", type=int, default=4096, help="batched: queries per batch")
    ap.add_argument("--batch-ks", default="1,10", help="batched: neighbour counts, one run each")
    ap.add_argument("--batch-arms", default="graph,persistent,streams,serial,per_query",
                    help="batched: execution arms to time")
    ap.add_argument("--serve-rates", default="1000,5000,20000", help="serve: Poisson arrival rates (queries/s)")
    ap.add_argument("--serve-seconds", type=float, default=2.0, help="serve: arrival window per rate")
    ap.add_argument("--serve-scale", type=float, default=1.0,
                    help="serve: database size factor (1.0: 1,000,000 x 256 + 200,000 x 1024)")
    ap.add_argument("--serve-no-tune", action="store_true",
                    help="serve: skip tuning each (n, w, k) of the index on sample queries before serving")
    ap.add_argument("--serve-secondary", action="store_true",
                    help="serve: also run with small buckets for lengths 128, 512 and 2048")
    ap.add_argument("--classify-dbs", type=int, default=50, help="classify: databases per instance count")
    return ap.parse_args()


DATA = {  # workload label, short description, description for the config
    "random_walk": ("random-walk", "seeded random walks", "seeded synthetic random walks (fp32)"),
    "shapes": ("shape-like", "seeded shape-like series",
               "seeded synthetic shape-like series (plateaus, ramps, sinusoid sums; noise, time shift, "
               "z-normalised; fp32)"),
}


def make_series(a, count, stream):
    gen = synth.shapes if a.data == "shapes" else synth.random_walks
    return gen(count, a.n, seed=a.seed, stream=stream)


@contextlib.contextmanager
def no_gc():
    """Host-timed loops run with Python's garbage collector paused, so that a
    collection does not land inside one step's wall time."""
    was = gc.isenabled()
    gc.collect()
    gc.disable()
    try:
        yield
    finally:
        if was:
            gc.enable()


def workload_config(a, world):
    return {
        "workload": "%s %d-NN retrieval: N=%d series, n=%d, w=%d, %d queries/step/GPU, DTW_%d"
        % (DATA[a.data][0], a.k, a.N, a.n, a.w, a.Q, a.p),
        "N": a.N, "n": a.n, "w": a.w, "queries_per_step_per_gpu": a.Q, "p": a.p, "k": a.k,
        "data": DATA[a.data][2], "seed": a.seed,
        "l2": "flushed between timed steps (256 MiB write)",
        "parallelism": ("candidates sharded over %d GPU(s) (thresholds all-reduced after the seeds, top-k "
                        "lists all-gathered and merged), every query on every GPU" % world
                        if getattr(a, "shard", "queries") == "candidates" else
                        "queries sharded over %d GPU(s), database replicated" % world),
    }


def cpu_info():
    model = ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if not model:
        try:  # Arm hosts name the core in lscpu only
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith(("model name", "vendor id")):
                    model = (model + " " + line.split(":", 1)[1].strip()).strip()
        except (OSError, subprocess.SubprocessError):
            pass
    return os.cpu_count() or 1, model


def oracle_rate(db, queries, w, p, k, budget_s):
    """Oracle (Algorithm 3 scan, fp64 C) on all host cores over a bounded query sample."""
    import oracle

    cores, model = cpu_info()
    # calibrate on one query per core, then size the sample to the budget
    t0 = time.perf_counter()
    oracle.knn_cascade(db, queries[:cores], w, p, k, mode=1, threads=cores)
    t1 = time.perf_counter() - t0
    per_q = max(t1 / cores, 1e-6)
    m = int(min(len(queries), max(cores, budget_s / per_q)))
    t0 = time.perf_counter()
    oracle.knn_cascade(db, queries[:m], w, p, k, mode=1, threads=cores)
    dt = time.perf_counter() - t0
    # the same scan on one thread, over a few queries
    m1 = max(1, min(len(queries), int(budget_s / 8 / per_q / cores) or 1, 8))
    t0 = time.perf_counter()
    oracle.knn_cascade(db, queries[:m1], w, p, k, mode=1, threads=1)
    dt1 = time.perf_counter() - t0
    return {"value": m / dt, "unit": "queries/s", "cores": cores, "cpu": model, "kind": "oracle",
            "sample": "%d of the step's queries against the full database, Algorithm 3 scan in fp64 C, "
                      "one query per thread" % m, "seconds": dt,
            "single_thread_value": m1 / dt1, "single_thread_sample": "%d queries on one thread" % m1}


class ClockSampler:
    """nvidia-smi clock / throttle samples, tagged with host time on arrival."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.samples = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                self.samples.append((time.time(), parts))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        win = [s for t, s in self.samples if t0 <= t <= t1]
        note = "timed region"
        if len(win) < 3:
            win = [s for _, s in self.samples]
            note = "whole run (timed region shorter than the sampling interval)"

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(s[0]) for s in win if num(s[0]) is not None]
        mx = [num(s[1]) for s in win if num(s[1]) is not None]
        pw = [num(s[2]) for s in win if num(s[2]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in win:
            for name, v in zip(names, s[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "reasons": sorted(reasons), "samples": len(win),
                "window": note}


# Algorithmic operation counts per unit of work (the paper's comparisons,
# counted as fp32 lane operations):
#  - a bound term d(v, [lo, hi])^p: two comparisons and an add, plus a
#    multiply for p = 2 (LB_Keogh per index; the piecewise-sum bound per part);
#  - LB_Improved's second sum: about five per index (the paper's 5n
#    comparisons per candidate that reaches it), plus a multiply for p = 2;
#  - a DTW band cell: a subtraction, an absolute value (or a multiply), two
#    minima and an add: five;
#  - the filter's test of a stored bound against the threshold: one.
def term_ops(p):
    return 3.0 if p == 1 else 4.0


def second_ops(p):
    return 5.0 if p == 1 else 6.0


DTW_CELL_OPS = 5.0


def alu_peak_tops(peaks):
    """Derived fp32 lane-op peak (T ops/s): SMs x 128 fp32 lanes x max SM clock."""
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    clock = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    return sms * 128 * clock / 1e12, "%d SMs x 128 fp32 lanes x %.0f MHz (max SM clock); derived, not measured" % (
        sms, clock / 1e6)


def filter_work(a, stats):
    """Per call of the default cascade: bounds scanned by the filter, pairs
    reaching LB_Keogh (piecewise-sum survivors) and pairs reaching the second
    sum (LB_Keogh survivors)."""
    scanned = stats.get("candidates", 0) - stats.get("seeds", 0)
    pd_surv = scanned - stats.get("pruned_summary", 0)
    lbk_surv = pd_surv - stats.get("pruned_keogh", 0)
    return scanned, pd_surv, lbk_surv


def stage_rates(prof, a, steps, peaks, stats, prefix_runs=1):
    """Achieved rate of each timed stage against the derived fp32 ALU peak, in
    the operation counts above: the piecewise-sum / LB_Keogh tile, the filter
    and the DTW stages (cells are the in-band cells evaluated).  prefix_runs:
    runs of the bound tile and the seeds per step (2 when the seeds'
    thresholds are exchanged before the search)."""
    alu_peak, _ = alu_peak_tops(peaks)
    out = {}

    def ms(stage):
        return prof[stage]["ms"] / max(1, steps)

    d = a.n // 8 if a.n >= 64 else a.n
    if prof["lb_keogh"]["launches"]:
        t = prefix_runs * a.Q * a.N * d * term_ops(a.p) / 1e12 / (ms("lb_keogh") / 1e3)
        out["lb_keogh_tile"] = {"ms": ms("lb_keogh"), "Top_s": t, "frac_alu": t / alu_peak}
    if prof["lb_improved"]["launches"] and stats.get("candidates"):
        scanned, pd_surv, lbk_surv = filter_work(a, stats)
        ops = scanned + pd_surv * a.n * term_ops(a.p) + lbk_surv * a.n * second_ops(a.p)
        t = ops / 1e12 / (ms("lb_improved") / 1e3)
        out["filter"] = {"ms": ms("lb_improved"), "Top_s": t, "frac_alu": t / alu_peak,
                         "lb_keogh_pairs": pd_surv, "second_sum_pairs": lbk_surv}
    if prof["dtw"]["launches"] and stats.get("dtw_cells"):
        cells = stats["dtw_cells"] / (ms("dtw") / 1e3)
        out["dtw"] = {"ms": ms("dtw"), "cells_per_s": cells, "frac_alu": cells * DTW_CELL_OPS / 1e12 / alu_peak}
        if stats.get("dtw_lane_rows"):
            # thread-per-pair kernel: share of the rows its warps stepped that
            # belonged to a live pair (a warp steps until its longest pair ends)
            out["dtw"]["lane_use"] = stats["dtw_rows"] / stats["dtw_lane_rows"]
    if prof["seed_dtw"]["launches"] and stats.get("seed_cells"):
        cells = prefix_runs * stats["seed_cells"] / (ms("seed_dtw") / 1e3)
        out["seed_dtw"] = {"ms": ms("seed_dtw"), "cells_per_s": cells,
                           "frac_alu": cells * DTW_CELL_OPS / 1e12 / alu_peak}
    return out


def roofline(prof, a, steps, peaks, stats, prefix_runs=1):
    """Roofline of the dominant stage (largest device time in the timed
    region), in the operation counts above; `instruction_mix` gives the same
    rate counted as the kernel's own fp32 instructions."""
    alu_peak, note = alu_peak_tops(peaks)
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    stages = {k: v for k, v in prof.items() if v["launches"] > 0}
    total = sum(v["ms"] for v in stages.values())
    dom = max(stages, key=lambda k: stages[k]["ms"])
    ms = stages[dom]["ms"] / max(1, stages[dom]["launches"])
    per_call = max(1, stages[dom]["launches"] // max(1, steps))  # launches of the stage per step
    share = {k: round(v["ms"] / total, 4) for k, v in stages.items()}
    base = {"bound": "alu", "peak": alu_peak, "unit": "Top/s", "traffic": None, "ms_per_launch": ms,
            "stage_share": share, "peak_note": note,
            "traffic_note": "no DRAM counter is read in the timed run; per-kernel DRAM bytes are in the ncu summaries"}
    if dom == "lb_keogh":
        d = a.n // 8 if a.n >= 64 else a.n
        ops = prefix_runs * a.Q * a.N * d * term_ops(a.p) / per_call
        achieved = ops / 1e12 / (ms / 1e3)
        return dict(base, kernel="k_lbk_tile", achieved=achieved, frac=achieved / alu_peak,
                    instruction_mix={"ops_per_term": 4, "Top_s": achieved * 4 / term_ops(a.p)})
    if dom in ("dtw", "seed_dtw"):
        cells = stats.get("dtw_cells" if dom == "dtw" else "seed_cells", 0) / per_call
        if dom == "seed_dtw":
            cells *= prefix_runs
        achieved = cells * DTW_CELL_OPS / 1e12 / (ms / 1e3) if cells else None
        band = 2 * min(a.w, a.n - 1) + 1
        lanes = a.dtw_path == 2 or (a.dtw_path == 0 and band > 208)
        name = "k_dtw_lanes" if lanes else ("k_dtw_reg4" if band <= 64 else "k_dtw_reg")
        if name == "k_dtw_reg4" and dom == "dtw" and per_call > 1:
            name = "k_dtw_reg4p"  # the main stage in row phases, one launch per phase
        return dict(base, kernel=name, achieved=achieved, frac=(achieved / alu_peak) if achieved else None,
                    cells_per_launch=cells,
                    instruction_mix={"ops_per_cell": 3, "Top_s": (achieved * 3 / DTW_CELL_OPS) if achieved else None})
    if dom == "lb_improved":
        scanned, pd_surv, lbk_surv = filter_work(a, stats)
        ops = (scanned + pd_surv * a.n * term_ops(a.p) + lbk_surv * a.n * second_ops(a.p)) / per_call
        achieved = ops / 1e12 / (ms / 1e3) if scanned > 0 else None
        mix = (scanned + pd_surv * a.n * 4.0 + lbk_surv * a.n * 6.0) / per_call / 1e12 / (ms / 1e3)
        # algorithmic DRAM bytes: the bound matrix once, and the database rows
        # and their envelope rows once each
        alg_bytes = (a.Q * a.N * 4.0 + a.N * a.n * 4.0 * 3) / per_call
        return dict(base, kernel="k_lbi_filter", achieved=achieved, frac=(achieved / alu_peak) if achieved else None,
                    algorithmic_bytes=alg_bytes, hbm_gbs_algorithmic=alg_bytes / 1e9 / (ms / 1e3),
                    hbm_frac_algorithmic=alg_bytes / 1e9 / (ms / 1e3) / hbm_peak,
                    lb_keogh_pairs=pd_surv, second_sum_pairs=lbk_surv,
                    instruction_mix={"ops_per_lb_keogh_index": 4, "ops_per_second_sum_index": 6, "Top_s": mix})
    return dict(base, kernel=dom, achieved=None, frac=None)


def run_ours(a):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_0811_3301_gb300 import build

    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    from paper_0811_3301_gb300 import _native as N
    from paper_0811_3301_gb300 import api

    from paper_0811_3301_gb300 import shard

    cand = a.shard == "candidates"
    db_h = make_series(a, a.N, synth.STREAM_DB)
    # query sharding: each GPU its own queries; candidate sharding: every GPU
    # the same queries against its own candidate range
    q_h = make_series(a, a.Q, synth.STREAM_QUERY + (0 if cand else 16 * rank))
    c0, c1 = shard.candidate_range(a.N, world, rank) if cand else (0, a.N)
    db = torch.from_numpy(np.ascontiguousarray(db_h[c0:c1])).to(dev)
    qs = torch.from_numpy(q_h).to(dev)
    flush = torch.empty(256 * 2**20 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
            torch.cuda.synchronize()

    kw = {"seeds": a.seeds, "parts": a.parts, "dtw_path": a.dtw_path, "filter_path": a.filter_path,
          "lb_abandon": a.lb_abandon}

    skw = {key: kw[key] for key in ("seeds", "parts", "dtw_path", "filter_path")}

    def step(p, queries=None):
        queries = qs if queries is None else queries
        if cand:
            return shard.sharded_knn_search(db, c0, queries, a.w, p, a.k, **kw)
        return api.knn_search(db, queries, a.w, p, a.k, **kw)

    per_step_queries = a.Q if cand else world * a.Q  # whole-job queries per step

    # pruning report (untimed): LB_Keogh alone vs LB_Keogh + LB_Improved
    pruning = {}
    for mode in ("keogh", "improved"):
        _, _, st = api.knn_search(db, qs, a.w, a.p, a.k, mode=mode, return_stats=True, **kw)
        tot = max(1, st["candidates"])
        # pruning power (Sec. 10): the share of candidates whose full DTW is
        # not computed, whichever bound (or the threshold) removed them
        dtw_fraction = (st["dtw_computed"] + st["seeds"]) / tot
        pruning[mode] = dict(st, pruning_power=round(1.0 - dtw_fraction, 6), dtw_fraction=round(dtw_fraction, 6))

    for _ in range(a.warmup):
        step(a.p)
    barrier()

    sampler = ClockSampler(local) if rank == 0 else None
    N.profile_read(reset=True)
    N.profile_enable(True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    barrier()
    t_wall0 = time.time()
    for i in range(a.steps):
        flush.fill_(float(i))  # evict the database and the previous step's buffers from L2
        evs[i][0].record(stream)
        step(a.p)
        evs[i][1].record(stream)
    barrier()
    t_wall1 = time.time()
    N.profile_enable(False)
    prof = N.profile_read(reset=True)
    ms_steps = [s.elapsed_time(e) for s, e in evs]
    ms_total = sum(ms_steps)
    t = torch.tensor([ms_total], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = per_step_queries * a.steps / (ms_max / 1e3)
    clocks = sampler.summary(t_wall0, t_wall1) if sampler else None

    # DTW rows evaluated per step (for the DTW roofline): one extra stats run
    if cand:
        thr = shard.exchange_thresholds(api.knn_seed_thresholds(db, qs, a.w, a.p, a.k, **skw))
        _, _, st_main = api.knn_search_bounded(db, qs, a.w, a.p, a.k, thr, return_stats=True, **kw)
    else:
        _, _, st_main = api.knn_search(db, qs, a.w, a.p, a.k, return_stats=True, **kw)

    # DTW_2 side measurement (same workload, same timing method)
    p2 = None
    if not a.no_p2:
        other = 2 if a.p == 1 else 1
        for _ in range(a.warmup):
            step(other)
        barrier()
        ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
        for i in range(a.steps):
            flush.fill_(float(i))
            ev2[i][0].record(stream)
            step(other)
            ev2[i][1].record(stream)
        barrier()
        ms2 = sum(s.elapsed_time(e) for s, e in ev2)
        t2 = torch.tensor([ms2], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(t2, op=dist.ReduceOp.MAX)
        p2 = {"p": other, "value": per_step_queries * a.steps / (float(t2.item()) / 1e3), "unit": "queries/s",
              "ms_per_step": float(t2.item()) / a.steps}

    # end to end through the public API: queries from pinned host memory,
    # results read back to pinned host memory, every step
    q_pin = torch.from_numpy(q_h).pin_memory()
    oi = torch.empty((a.Q, a.k), dtype=torch.int64).pin_memory()
    od = torch.empty((a.Q, a.k), dtype=torch.float32).pin_memory()
    def e2e_step():
        if cand:
            # the collectives take device tensors: queries in, merged lists out
            mi, md = step(a.p, q_pin.to(dev, non_blocking=True))
            oi.copy_(mi)
            od.copy_(md)
            torch.cuda.synchronize()
        else:
            api.knn_search(db, q_pin, a.w, a.p, a.k, out_idx=oi, out_dist=od, **kw)  # synchronous (host outputs)

    for _ in range(a.warmup):
        e2e_step()
    barrier()
    e2e_s = 0.0
    e2e_steps = []
    with no_gc():
        for i in range(a.steps):
            flush.fill_(float(i))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_step()
            e2e_steps.append(time.perf_counter() - t0)
            e2e_s += e2e_steps[-1]
    te = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e = {"value": per_step_queries * a.steps / float(te.item()), "unit": "queries/s",
           "h2d_bytes_per_step": a.Q * a.n * 4, "d2h_bytes_per_step": a.Q * a.k * (8 + 4),
           "step_ms_median": float(np.median(e2e_steps)) * 1e3, "step_ms_max": max(e2e_steps) * 1e3}

    if sampler:
        sampler.stop()

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    launches = sum(v["launches"] for v in prof.values())
    if cand:
        launches += a.steps  # the merge kernel, outside the stage timers
    # the shard's own size in candidate mode; the bound tile and the seeds run
    # twice per step there (once for the thresholds, once in the search)
    ar = argparse.Namespace(**vars(a))
    ar.N = c1 - c0
    prefix_runs = 2 if cand else 1
    roof = roofline(prof, ar, a.steps, peaks, st_main, prefix_runs)

    if rank != 0:
        return None
    cpu = None
    if world == 1:
        cpu = oracle_rate(db_h, q_h, a.w, a.p, a.k, a.cpu_seconds)
    extra = {}
    if world == 1 and not a.no_extra and a.workload == "retrieval":
        del db, qs, flush
        torch.cuda.empty_cache()
        extra = extra_workloads(a)
    out = {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True,
        "scaling": "strong" if cand else "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (%s)" % DATA[a.data][1],
        "config": workload_config(a, world), "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches, "clocks": clocks, "p2": p2, "pruning": pruning,
        "stages_ms_per_step": {k: v["ms"] / a.steps for k, v in prof.items()},
        "stage_rates": stage_rates(prof, ar, a.steps, peaks, st_main, prefix_runs),
        "stats_per_step": st_main,
    }
    out.update(extra)
    return out


def extra_workloads(a):
    """Bounded runs of the batched and serving workloads, reported beside the
    default workload in its line: the mixed-length batch (11 buckets of
    20,000 random walks, 4,096 queries, DTW_2, k = 1 and 10) through the
    index as one graph per batch against one cascade per query, and Poisson
    arrivals at 1,000, 5,000 and 20,000 queries/s through the server against
    the same server restricted to one query per launch.  Each carries its own
    clock record."""
    import copy

    import torch

    b = copy.copy(a)
    b.steps, b.warmup = min(a.steps, 5), min(max(a.warmup, 1), 2)
    b.batch_arms = "graph,persistent,per_query"
    b.per_query_steps = 1
    out = {}
    t0 = time.time()
    r = run_batched(b)
    out["batched"] = {
        "metric": r["metric"], "value": r["value"], "unit": r["unit"], "ms_per_step": r["ms_per_step"],
        "e2e": r["e2e"], "vs_per_query": r["vs_per_query"], "persistent_vs_per_query": r["persistent_vs_per_query"],
        "persistent_vs_graph": r["persistent_vs_graph"], "config": r["config"], "clocks": r["clocks"],
        "per_k": {k: {"arms": v["arms"], "e2e": v["e2e"], "autotune_seconds": v["autotune_seconds"]}
                  for k, v in r["per_k"].items()},
        "wall_s": time.time() - t0}
    torch.cuda.empty_cache()
    s = copy.copy(a)
    s.serve_rates, s.serve_seconds, s.serve_scale, s.serve_secondary = "1000,5000,20000", 1.0, 1.0, False
    t0 = time.time()
    r = run_serve(s)
    out["serve"] = {
        "metric": r["metric"], "config": r["config"], "clocks": r["clocks"],
        "runs": [{"rate_qps": x["rate_qps"], "plain_same_results": x["plain_same_results"],
                  "batched": {k: x["batched"][k] for k in ("throughput_qps", "p50_ms", "p99_ms", "p999_ms",
                                                           "succeeded", "failed", "all_ok", "mean_batch",
                                                           "max_batch")},
                  "plain": {k: x["plain"][k] for k in ("throughput_qps", "p50_ms", "p99_ms", "succeeded", "failed",
                                                       "all_ok")}}
                 for x in r["runs"]],
        "capacity": r["capacity"],
        "wall_s": time.time() - t0}
    torch.cuda.empty_cache()
    return out


def run_batched(a):
    """Mixed-length batches through the index: 11 length buckets 64 * 2^(j/2)
    (64 .. 2048) of `bucket_N` random walks each, `batch_Q` queries per batch
    with lengths log-uniform in [64, 2048] snapped to the nearest bucket in log
    space, w = floor(n / 10), DTW_2, one run per k.  Arms: the batch as one
    CUDA graph (groups on concurrent streams, autotuned parameters), the same
    without the graph, the groups serially, and one cascade per query (the
    unbatched baseline)."""
    import torch

    from paper_0811_3301_gb300 import build

    build.build()
    from paper_0811_3301_gb300 import api

    dev = torch.device("cuda", torch.cuda.current_device())
    buckets = synth.bucket_lengths(64, 2048)
    ix = api.DtwIndex(2)
    for n in buckets:
        ix.add_bucket(torch.from_numpy(synth.random_walks(a.bucket_N, n, seed=a.seed + 1000 + n)).to(dev))
    lens = synth.snap_to_buckets(synth.log_uniform_lengths(a.batch_Q, 64, 2048, seed=a.seed), buckets)
    qs = synth.mixed_queries(lens, seed=a.seed)
    ws = lens // 10
    flat_h = np.ascontiguousarray(np.concatenate(qs), dtype=np.float32)
    flat = torch.from_numpy(flat_h).to(dev)
    flush = torch.empty(256 * 2**20 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    arms_wanted = [x for x in a.batch_arms.split(",") if x]
    arm_kw = {"graph": {"graph": True}, "streams": {}, "serial": {"serial": True}, "per_query": {"per_query": True},
              "persistent": {"graph": True, "persistent": True}}
    sampler = ClockSampler(0)
    t_wall0 = time.time()
    per_k = {}
    launches = 0
    for k in [int(x) for x in a.batch_ks.split(",") if x]:
        t0 = time.perf_counter()
        ref_i, ref_d = ix.search_flat(flat, lens, ws, k, autotune=True)
        if "persistent" in arms_wanted:  # the persistent arm's chunk length
            ix.search_flat(flat, lens, ws, k, autotune=True, persistent=True)
        torch.cuda.synchronize()
        tune_s = time.perf_counter() - t0
        arms = {}
        for arm in arms_wanted:
            kw = arm_kw[arm]
            steps = a.steps if arm != "per_query" else max(1, min(a.steps, getattr(a, "per_query_steps", 3)))
            for _ in range(a.warmup):
                ix.search_flat(flat, lens, ws, k, **kw)
            torch.cuda.synchronize()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for i in range(steps):
                flush.fill_(float(i))
                evs[i][0].record(stream)
                oi, od = ix.search_flat(flat, lens, ws, k, **kw)
                evs[i][1].record(stream)
            torch.cuda.synchronize()
            ms = sum(x.elapsed_time(y) for x, y in evs)
            same = bool(torch.equal(oi, ref_i) and torch.equal(od, ref_d))
            arms[arm] = {"value": a.batch_Q * steps / (ms / 1e3), "unit": "queries/s", "ms_per_step": ms / steps,
                         "steps": steps, "same_result_as_first_run": same}
        # end to end: queries from pinned host memory, results to pinned host memory
        fpin = torch.from_numpy(flat_h).pin_memory()
        oi_h = torch.empty((a.batch_Q, k), dtype=torch.int64).pin_memory()
        od_h = torch.empty((a.batch_Q, k), dtype=torch.float32).pin_memory()
        for _ in range(a.warmup):
            ix.search_flat(fpin, lens, ws, k, graph=True, out_idx=oi_h, out_dist=od_h)
        e2e_s = 0.0
        with no_gc():
            for i in range(a.steps):
                flush.fill_(float(i))
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ix.search_flat(fpin, lens, ws, k, graph=True, out_idx=oi_h, out_dist=od_h)
                e2e_s += time.perf_counter() - t0
        _, _, st = ix.search_flat(flat, lens, ws, k, return_stats=True)
        tuning = {int(n): ix.get_tuning(int(n), int(n) // 10, k) for n in buckets}
        per_k[k] = {"arms": arms, "autotune_seconds": tune_s, "tuning": tuning, "stats": st,
                    "e2e": {"value": a.batch_Q * a.steps / e2e_s, "unit": "queries/s",
                            "h2d_bytes_per_step": int(flat_h.nbytes) + a.batch_Q * 12,
                            "d2h_bytes_per_step": a.batch_Q * k * 12}}
    t_wall1 = time.time()
    clocks = sampler.summary(t_wall0, t_wall1)
    sampler.stop()
    info = ix.info()
    ks = sorted(per_k)
    tot_q = sum(a.batch_Q * per_k[k]["arms"]["graph"]["steps"] for k in ks) if "graph" in arms_wanted else 0
    tot_s = sum(per_k[k]["arms"]["graph"]["ms_per_step"] * per_k[k]["arms"]["graph"]["steps"] / 1e3 for k in ks) \
        if "graph" in arms_wanted else 0
    value = tot_q / tot_s if tot_s else None
    e2e_v = len(ks) / sum(1.0 / per_k[k]["e2e"]["value"] for k in ks)
    out = {
        "metric": "exact k-NN DTW queries/s, mixed-length batches (LB_Improved cascade, one graph per batch)",
        "value": value, "unit": "queries/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": (tot_s * 1e3 / sum(per_k[k]["arms"]["graph"]["steps"] for k in ks)) if tot_s else None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded random walks)",
        "config": {"workload": "batched mixed-length k-NN: %d queries/batch, lengths log-uniform in [64, 2048] "
                               "snapped to 11 buckets of %d random walks, w = floor(n/10), DTW_2, k in %s"
                               % (a.batch_Q, a.bucket_N, ks),
                   "buckets": buckets, "queries_per_bucket": {int(n): int((lens == n).sum()) for n in buckets},
                   "l2": "flushed between timed steps (256 MiB write)"},
        "e2e": {"value": e2e_v, "unit": "queries/s",
                "h2d_bytes_per_step": per_k[ks[0]]["e2e"]["h2d_bytes_per_step"],
                "d2h_bytes_per_step": per_k[ks[0]]["e2e"]["d2h_bytes_per_step"]},
        "vs_per_query": {k: (per_k[k]["arms"]["graph"]["value"] / per_k[k]["arms"]["per_query"]["value"])
                         for k in ks if "graph" in per_k[k]["arms"] and "per_query" in per_k[k]["arms"]},
        "persistent_vs_per_query": {k: (per_k[k]["arms"]["persistent"]["value"] /
                                        per_k[k]["arms"]["per_query"]["value"])
                                    for k in ks if "persistent" in per_k[k]["arms"] and "per_query" in per_k[k]["arms"]},
        "persistent_vs_graph": {k: (per_k[k]["arms"]["persistent"]["value"] / per_k[k]["arms"]["graph"]["value"])
                                for k in ks if "persistent" in per_k[k]["arms"] and "graph" in per_k[k]["arms"]},
        "per_k": per_k, "index": info, "clocks": clocks,
    }
    return out


def serve_run(api, ix, lens, queries, ks, arrivals, **cfg):
    """Submits requests at their arrival times (seconds from start) to a new
    server and collects completions; returns latency and throughput figures."""
    import threading as th

    srv = api.DtwServer(ix, **cfg)
    Q = len(lens)
    tickets = [0] * Q
    got = {}
    done_flag = th.Event()

    def poller():
        while not done_flag.is_set() or len(got) < Q:
            for c in srv.poll(wait_ms=20):
                got[c["ticket"]] = c
            if done_flag.is_set() and len(got) >= Q:
                break

    pt = th.Thread(target=poller, daemon=True)
    pt.start()
    t0 = api.monotonic_ns() + 20_000_000
    sched = t0 + (np.asarray(arrivals) * 1e9).astype(np.int64)
    for i in range(Q):
        while api.monotonic_ns() < sched[i]:
            pass
        tickets[i] = srv.submit(queries[i], int(lens[i]) // 10, int(ks[i]), arrival_ns=int(sched[i]))
    deadline = time.time() + 600
    while len(got) < Q and time.time() < deadline:
        time.sleep(0.005)
    done_flag.set()
    pt.join(timeout=5)
    info = srv.info()
    srv.close()
    comp = [got[t] for t in tickets if t in got]
    out = latency_summary(comp)
    out.update({"offered_qps": Q / float(arrivals[-1]) if Q > 1 else None, "requests": Q,
                "batches": info["batches"], "mean_batch": len(comp) / max(1, info["batches"]),
                "max_batch": info["max_batch_seen"], "max_inflight_batches": info["max_inflight_batches"]})
    return out, comp


def latency_summary(comp):
    """Latency (completion - arrival) and queueing delay (admission - arrival)
    percentiles in ms, and throughput over the span from the first arrival to
    the last completion, of the server completions (dicts with arrival_ns,
    admit_ns, done_ns and status) that succeeded (status 0).  Failed requests
    (a timeout, status 4, or any other error) are counted apart and enter
    neither the latencies nor the throughput; `all_ok` says whether there
    were none."""
    ok = [c for c in comp if c["status"] == 0]
    failed = len(comp) - len(ok)
    out = {"completed": len(comp), "succeeded": len(ok), "failed": failed,
           "timed_out": sum(1 for c in comp if c["status"] == 4), "all_ok": failed == 0}
    if not ok:
        return dict(out, throughput_qps=0.0, p50_ms=None, p99_ms=None, p999_ms=None, mean_ms=None,
                    queue_p50_ms=None, queue_p99_ms=None)
    lat = np.array([(c["done_ns"] - c["arrival_ns"]) / 1e6 for c in ok])
    wait = np.array([(c["admit_ns"] - c["arrival_ns"]) / 1e6 for c in ok])
    first = min(c["arrival_ns"] for c in ok)
    last = max(c["done_ns"] for c in ok)
    out.update({"throughput_qps": len(ok) / ((last - first) / 1e9),
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "p999_ms": float(np.percentile(lat, 99.9)), "mean_ms": float(lat.mean()),
                "queue_p50_ms": float(np.percentile(wait, 50)), "queue_p99_ms": float(np.percentile(wait, 99))})
    return out


def bucket_capacity(api, N, ix, lengths, seed, count=256):
    """Throughput of each (bucket, k) alone through the index (one batch of
    `count` queries, no graph), with the device time of each cascade stage
    per query, and the capacity of the serving mix (lengths and k = 1 / 10
    in equal shares) that these rates allow."""
    import torch

    out = {}
    inv = []
    for n in lengths:
        qs = synth.random_walks(count, n, seed=seed + 7000 + n, stream=synth.STREAM_QUERY)
        flat = torch.from_numpy(np.ascontiguousarray(qs.reshape(-1))).cuda()
        lens = np.full(count, n)
        for k in (1, 10):
            ix.search_flat(flat, lens, n // 10, k)
            torch.cuda.synchronize()
            N.profile_read(reset=True)
            N.profile_enable(True)
            t0 = time.perf_counter()
            reps = 3
            for _ in range(reps):
                ix.search_flat(flat, lens, n // 10, k)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            N.profile_enable(False)
            prof = N.profile_read(reset=True)
            qps = count * reps / dt
            per_q = {st: round(v["ms"] / (count * reps) * 1e3, 3) for st, v in prof.items() if v["launches"]}
            tot = sum(per_q.values())
            out["n%d_k%d" % (n, k)] = {"qps": qps, "stage_us_per_query": per_q,
                                       "dominant_stage": max(per_q, key=per_q.get) if per_q else None,
                                       "dominant_share": (max(per_q.values()) / tot) if tot else None}
            inv.append(1.0 / qps)
    return {"buckets": out, "mix_capacity_qps": len(inv) / sum(inv),
            "note": "each (length, k) alone, %d queries per batch; the mix capacity is the harmonic mean over the "
                    "equally likely (length, k) combinations" % count}


def run_serve(a):
    """Poisson arrivals of single k-NN queries (DTW_1, half 1-NN and half
    10-NN, w = floor(n/10)) against a resident database of 1,000,000 random
    walks of length 256 and 200,000 of length 1024; query lengths drawn from
    {256, 1024} (the lengths with a bucket).  The continuous-batching server
    (4 slots, admission by a per-slot workspace of 8 GiB) is compared with the
    same server restricted to one query per launch, one at a time."""
    import torch

    from paper_0811_3301_gb300 import build

    build.build()
    from paper_0811_3301_gb300 import api

    from paper_0811_3301_gb300 import _native as N

    dev = torch.device("cuda", torch.cuda.current_device())
    sizes = {256: int(1_000_000 * a.serve_scale), 1024: int(200_000 * a.serve_scale)}
    lengths = [256, 1024]
    if a.serve_secondary:
        for n in (128, 512, 2048):
            sizes[n] = int(100_000 * a.serve_scale)
        lengths = [128, 256, 512, 1024, 2048]
    ix = api.DtwIndex(1)
    for n in sorted(sizes):
        ix.add_bucket(torch.from_numpy(synth.random_walks(sizes[n], n, seed=a.seed + 5000 + n)).to(dev))
    torch.cuda.synchronize()
    # the index's parameters for each (n, w, k) the stream will ask for, timed
    # on sample queries of that length (the server uses the index's tuning)
    tuning = {}
    t0 = time.perf_counter()
    if not a.serve_no_tune:
        for n in lengths:
            sample = torch.from_numpy(synth.random_walks(256, n, seed=a.seed + 9000 + n,
                                                         stream=synth.STREAM_QUERY)).to(dev)
            for k in (1, 10):
                tuning["n%d_k%d" % (n, k)] = ix.tune(sample, n // 10, k)
    tune_s = time.perf_counter() - t0
    sampler = ClockSampler(0)
    t_wall0 = time.time()
    runs = []
    for rate in [float(x) for x in a.serve_rates.split(",") if x]:
        Q = max(50, int(rate * a.serve_seconds))
        g = np.random.default_rng([a.seed, int(rate)])
        lens = g.choice(lengths, size=Q)
        ks = g.choice([1, 10], size=Q)
        qs = [np.ascontiguousarray(x) for x in synth.mixed_queries(lens, seed=a.seed + int(rate))]
        arr = synth.poisson_arrivals(Q, rate, seed=a.seed + int(rate))
        # warm-up: a few requests through a throwaway server
        serve_run(api, ix, lens[:64], qs[:64], ks[:64], np.linspace(0.0, 0.01, 64), slots=4, max_batch=512,
                  slot_bytes=8 << 30)
        res, comp = serve_run(api, ix, lens, qs, ks, arr, slots=4, max_batch=512, slot_bytes=8 << 30)
        # the plain arm: one query per launch of each stage, one query at a time,
        # on a bounded prefix of the same stream (it saturates far below these rates)
        Qp = min(Q, max(50, int(2.0 * 300)))
        plain, pcomp = serve_run(api, ix, lens[:Qp], qs[:Qp], ks[:Qp], arr[:Qp], slots=1, max_batch=1,
                                 per_query=True, slot_bytes=8 << 30)
        same = all(np.array_equal(x["idx"], y["idx"]) and np.array_equal(x["dist"], y["dist"])
                   for x, y in zip(comp[:Qp], pcomp))
        runs.append({"rate_qps": rate, "batched": res, "plain": plain, "plain_same_results": bool(same)})
    t_wall1 = time.time()
    clocks = sampler.summary(t_wall0, t_wall1)
    sampler.stop()
    capacity = bucket_capacity(api, N, ix, lengths, a.seed)
    best = max(runs, key=lambda r: r["batched"]["throughput_qps"])
    return {
        "metric": "exact k-NN DTW queries/s and p50/p99/p99.9 latency, Poisson arrivals, continuous batching",
        "value": best["batched"]["throughput_qps"], "unit": "queries/s", "n_gpus": 1,
        "p50_ms": best["batched"]["p50_ms"], "p99_ms": best["batched"]["p99_ms"],
        "p999_ms": best["batched"]["p999_ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded random walks)",
        "config": {"workload": "serving: Poisson arrivals at %s q/s, query lengths from %s, resident random walks %s, "
                               "w = floor(n/10), DTW_1, 1-NN/10-NN mixed 50/50"
                               % (a.serve_rates, lengths, {int(k): v for k, v in sizes.items()}),
                   "server": {"slots": 4, "max_batch": 512, "slot_bytes": 8 << 30}},
        "runs": runs, "capacity": capacity, "tuning": tuning, "tune_seconds": tune_s, "index": ix.info(),
        "clocks": clocks,
    }


def run_triangle(a):
    """App. B: DTW_p(x,z) / (DTW_p(x,y) + DTW_p(y,z)) over 100,000 triples of
    100-sample series (white noise, random walks, shape-like series standing
    in for Cylinder-Bell-Funnel), no time constraint, p = 1 and 2: the share of
    triples that violate the triangle inequality, and the DTW rate."""
    import torch

    from paper_0811_3301_gb300 import build

    build.build()
    from paper_0811_3301_gb300 import api

    N, n = 100_000, 100
    w = n - 1
    gens = {"white_noise": synth.white_noise, "random_walk": synth.random_walks, "shapes": synth.shapes}
    flush = torch.empty(256 * 2**20 // 4, dtype=torch.float32, device="cuda")
    cells_per_pair = n * (2 * w + 1) - w * (w + 1)
    res = {}
    total_ms = 0.0
    total_pairs = 0
    for kind, g in gens.items():
        x, y, z = (torch.from_numpy(g(N, n, seed=a.seed + 90 + s)).cuda() for s in range(3))
        for p in (1, 2):
            for _ in range(a.warmup):
                api.dtw_triangle(x, y, z, w, p)
            torch.cuda.synchronize()
            ms = 0.0
            for i in range(a.steps):
                flush.fill_(float(i))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                r = api.dtw_triangle(x, y, z, w, p)
                e1.record()
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
            rc = r.cpu().numpy()
            hist, edges = np.histogram(rc, bins=30, range=(0.0, 1.5))
            res["%s_p%d" % (kind, p)] = {"violations": float((rc > 1.0).mean()), "max_ratio": float(rc.max()),
                                         "ms_per_call": ms / a.steps,
                                         "histogram": {"edges": edges.tolist(), "counts": hist.tolist()}}
            total_ms += ms
            total_pairs += 3 * N * a.steps
    return {
        "metric": "DTW pairs/s, App. B triangle-inequality experiment (dense batched DTW, no band)",
        "value": total_pairs / (total_ms / 1e3), "unit": "DTW pairs/s", "n_gpus": 1, "steps": a.steps,
        "warmup": a.warmup, "cells_per_s": total_pairs * cells_per_pair / (total_ms / 1e3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded white noise, random walks, shape-like series)",
        "config": {"workload": "App. B: %d triples of n = %d, w = %d (no constraint), p in {1, 2}" % (N, n, w),
                   "paper": "no violation for white noise and Cylinder-Bell-Funnel; 20 %% (DTW_1) and 15 %% "
                            "(DTW_2) of random-walk triples violate the triangle inequality"},
        "results": res,
    }


def classify_labels(a, m, db_i, tests):
    """Database labels (m per class) and test labels (uniform) of database db_i."""
    g = np.random.default_rng([a.seed, 7000 + m, db_i])
    return np.repeat(np.arange(synth.SHAPE_CLASSES), m), g.integers(0, synth.SHAPE_CLASSES, size=tests)


def run_classify(a):
    """App. C: 1-NN classification accuracy under DTW_p, p in {1, 2, 4,
    infinity}, w = n/10, on the shape-like classes (plateau, rising ramp,
    falling ramp, sum of sinusoids; n = 128, the length of the paper's first
    data set) standing in for the paper's synthetic data sets: for m instances
    per class, `classify_dbs` databases of 4 m series, each with 500 new test
    series of random class; a test succeeds when its nearest neighbour (lowest
    index on ties) has its class.  All (test, database series) pairs of all
    databases go through dtw_band in one launch per (m, p); the oracle's 1-NN
    labels are checked on a sample."""
    import torch

    from paper_0811_3301_gb300 import build

    build.build()
    import oracle

    from paper_0811_3301_gb300 import api

    n, tests, ms_list = 128, 500, (1, 2, 3, 5, 9)
    w = n // 10
    D = a.classify_dbs
    ps = (1, 2, 4, math.inf)
    acc = {}
    rate_pairs, rate_ms = 0, 0.0
    agree, checked = 0, 0
    for m in ms_list:
        k = synth.SHAPE_CLASSES * m
        dbs, tsts, dlab, tlab = [], [], [], []
        for i in range(D):
            ld, lt = classify_labels(a, m, i, tests)
            dbs.append(synth.shape_classes(ld, n, seed=a.seed + 100 * m + i))
            tsts.append(synth.shape_classes(lt, n, seed=a.seed + 100 * m + i, stream=synth.STREAM_QUERY))
            dlab.append(ld)
            tlab.append(lt)
        db = torch.from_numpy(np.stack(dbs)).cuda()     # [D][k][n]
        ts = torch.from_numpy(np.stack(tsts)).cuda()    # [D][tests][n]
        X = db[:, None, :, :].expand(D, tests, k, n).reshape(-1, n).contiguous()
        Y = ts[:, :, None, :].expand(D, tests, k, n).reshape(-1, n).contiguous()
        dl = np.stack(dlab)
        tl = np.stack(tlab)
        for p in ps:
            api.dtw_band(X, Y, w, p)  # warm-up
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            d = api.dtw_band(X, Y, w, p)
            e1.record()
            torch.cuda.synchronize()
            rate_ms += e0.elapsed_time(e1)
            rate_pairs += X.shape[0]
            nn = torch.argmin(d.view(D, tests, k), dim=2).cpu().numpy()  # first index on ties
            pred = np.take_along_axis(dl, nn, axis=1)
            acc.setdefault(str(m), {})["inf" if p == math.inf else str(p)] = float((pred == tl).mean())
            # the oracle's nearest neighbour on a sample of tests of database 0
            op = 0 if p == math.inf else p
            for t in range(0, tests, 50):
                oi, _ = oracle.knn_bruteforce(dbs[0], tsts[0][t][None, :], w, op, 1)
                agree += int(oi[0, 0] == nn[0, t])
                checked += 1
    return {
        "metric": "1-NN classification accuracy under DTW_p (App. C), with the DTW pair rate",
        "value": rate_pairs / (rate_ms / 1e3), "unit": "DTW pairs/s", "n_gpus": 1, "steps": 1, "warmup": 1,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded shape-like series, 4 classes)",
        "config": {"workload": "App. C: n = %d, w = %d, %d databases per m, %d tests each, m in %s instances "
                               "per class, p in {1, 2, 4, inf}" % (n, w, D, tests, list(ms_list)),
                   "paper": "DTW_1 classifies best, DTW_2 a close second, DTW_4 lower; DTW_inf is competitive "
                            "only with one or two instances per class"},
        "accuracy": acc,
        "oracle_agreement": {"checked": checked, "equal": agree},
    }


def run_reference(a):
    """The reference arm: the FP64 oracle (Algorithm 3 scan in C) on all host
    cores, one query per thread.  A step is a bounded sample of the step's
    query batch against the full database, sized once from a calibration run
    so that the whole --warmup W --steps K run takes about two minutes;
    consecutive steps take consecutive slices of the batch.  ms_per_step and
    value are the measured time and rate of exactly those queries."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    import oracle

    oracle.build()
    db_h = make_series(a, a.N, synth.STREAM_DB)
    q_h = make_series(a, a.Q, synth.STREAM_QUERY)
    cores, model = cpu_info()
    t0 = time.perf_counter()
    oracle.knn_cascade(db_h, q_h[:cores], a.w, a.p, a.k, mode=1, threads=cores)
    rate0 = min(cores, a.Q) / max(time.perf_counter() - t0, 1e-6)
    budget = max(1.0, 110.0 / max(1, a.warmup + a.steps))  # seconds per step
    m = int(min(a.Q, max(min(cores, a.Q), budget * rate0)))
    times = []
    for i in range(a.warmup + a.steps):
        idx = (np.arange(m) + i * m) % a.Q
        t0 = time.perf_counter()
        oracle.knn_cascade(db_h, q_h[idx], a.w, a.p, a.k, mode=1, threads=cores)
        if i >= a.warmup:
            times.append(time.perf_counter() - t0)
    total = sum(times)
    v = m * len(times) / total
    sample = ("%d of the step's %d queries per step (consecutive slices of the batch) against the full database, "
              "Algorithm 3 scan in fp64 C, one query per thread" % (m, a.Q))
    return {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "queries/s", "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (%s)" % DATA[a.data][1],
        "config": dict(workload_config(a, world), queries_per_step_timed=m),
        "cpu_baseline": {"value": v, "unit": "queries/s", "cores": cores, "cpu": model, "kind": "oracle",
                         "sample": sample, "seconds": total},
        "e2e": {"value": v, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    a = parse()
    if a.impl == "reference":
        out = run_reference(a)
    elif a.workload == "batched":
        out = run_batched(a)
    elif a.workload == "serve":
        out = run_serve(a)
    elif a.workload == "triangle":
        out = run_triangle(a)
    elif a.workload == "classify":
        out = run_classify(a)
    else:
        out = run_ours(a)
    if out is not None:
        print(json.dumps(out))
    if int(os.environ.get("WORLD_SIZE", "1")) > 1 and a.impl == "ours":
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
