#!/usr/bin/env python
"""Benchmark: exact k-NN scan (DTW and DK), learned + batched, on the d = 16,
500,000 x 512 workload.

One step = one batched scan of the step's 1,000 queries (per GPU) against the
500,000-series database (AR(1) correlated channels, d = 16, length 512), for
DTW and for DK (k = 50, Sakoe-Chiba band 10%), with learned seeding, through
the library's public C-ABI, inputs already resident in HBM.  The timed scans
are the production path (no per-stage events); the stage split comes from one
extra profiled scan per distance after the timed region.  Prints one JSON
line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
                    [--workload NAME]

Under torchrun (N > 1) every rank scans its own 1,000 queries against a
replica of the database (independent problems, no data-path collective);
value = all ranks' queries / the slowest rank's time.

The line also carries: the plain GPU scan (batched, LB_Box-ordered seeding,
no encoder) and the paper's greedy pre-pass timed the same way on the same
queries; a parity check (the oracle's exact result on a slice of the
database against the GPU's on the same slice, and the oracle's distances for
a sample of the full-size results); the oracle's CPU rate.

--impl reference times the FP64 oracle (the paper's pruned scan, CPU) on a
bounded sample of the same workload on the host cores: a fixed prefix of the
database (the workload's first `oracle_series` series) and one query per
core, extrapolated linearly to the whole database.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact k-NN queries/sec and DP GCUPS (DTW & DK), learned+batched vs plain GPU scan"
# Workloads this harness measures: generator name in synthdata.WORKLOADS, k,
# band, queries per GPU, whether the timed scans replay a CUDA graph, and the
# database prefix the oracle scans for the CPU rate and the exact parity check.
BENCH = {
    "highdim_d16_n500k_L512": dict(k=50, band=0.1, queries=1000, graph=False,
                                   oracle_series=4000),
    "scale_d3_n100k_L256": dict(k=10, band=0.1, queries=1000, graph=False,
                                oracle_series=100_000),
    **{f"uneven_d{d}_n200k_L50_1000": dict(k=5, band=0.1, queries=256, graph=True,
                                           oracle_series=20_000)
       for d in range(3, 9)},
    "learned_d3_n1M_L128": dict(k=10, band=0.1, queries=1000, graph=False,
                                oracle_series=50_000),
}
WORKLOAD = "highdim_d16_n500k_L512"
N_SERIES, LENGTH, D, N_QUERIES = 500_000, 512, 16, 1000
K, BAND = 50, 0.1
ORACLE_SERIES = 4000
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
SEED_DESC = {"greedy": "greedy upper-bound pre-pass over every series (Section 4.3)",
             "lb": "LB_Box-ordered proposals scored exactly first, then filter",
             "learned": "learned proposals (BF16 conv encoder trained on 200k pairs of the "
                        "database's own DTW/DK distances) scored exactly first, then the "
                        "LB_Box stream with early abandoning",
             "none": "no seeding"}
TRAIN_PAIRS = 200_000
# sampled full-size parity: queries checked, random other series per query
PARITY_QUERIES, PARITY_OTHERS = 8, 192
TOL = {0: 1e-5, 1: 1e-6}     # relative distance tolerance, DTW / DK


# DRAM bytes (read + write) of the dominant kernels on the bench workloads,
# from one `ncu` capture of the current kernel on a reduced case of the same
# workload, per unit of algorithmic work (a DP band cell): the roofline's
# `traffic` is that figure times the units of the region `achieved` covers.
# A kernel changed since its capture has no entry (traffic null).
TRAFFIC_PER_UNIT = {
    # dp_kernel<16, 4, 0, WIN> on the first 50,000 series and 64 queries:
    # 1,000.1 MB of DRAM traffic for 1,494.7 M band cells (each pair streams
    # its series once, so the traffic follows the cells it sweeps)
    ("dp_kernel", "highdim_d16_n500k_L512"): (
        0.669, "ncu dram__bytes_read.sum + dram__bytes_write.sum of one DTW launch, "
               "50,000 series x 64 queries, per band cell, scaled by the cells counted here"),
}


def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, 2070.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        except FileNotFoundError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def select_workload(name: str):
    """Set the module-level workload parameters from the BENCH table."""
    global WORKLOAD, N_SERIES, LENGTH, D, N_QUERIES, K, BAND, ORACLE_SERIES
    from synthdata import WORKLOADS
    g, b = WORKLOADS[name], BENCH[name]
    WORKLOAD = name
    N_SERIES, D, N_QUERIES = g["n_series"], g["d"], b["queries"]
    LENGTH = g.get("length", 0) if "length_range" not in g else 0
    K, BAND = b["k"], b["band"]
    ORACLE_SERIES = b["oracle_series"]


def workload(world: int, n_series: int = 0):
    """The workload (all ranks' queries); n_series > 0 draws only that prefix
    of the database (the queries do not depend on it)."""
    from synthdata import WORKLOADS, make_workload
    kw = dict(WORKLOADS[WORKLOAD])
    kw["n_queries"] = N_QUERIES * world
    kw["n_series"] = n_series or N_SERIES
    return make_workload(**kw)


def db_prefix(w, n: int):
    """The first n series of a workload's database (points, offsets)."""
    n = min(n, int(w.db_off.shape[0] - 1))
    return w.db[: w.db_off[n]], w.db_off[: n + 1].copy()


def oracle_sample(w, n_sample: int, threads: int) -> dict:
    """The FP64 oracle (the paper's pruned scan) on the first n_sample queries
    against the first ORACLE_SERIES series, DTW and DK; returns the time, its
    results and the extrapolation to the whole database."""
    import oracle
    oracle.lib()
    db, off = db_prefix(w, ORACLE_SERIES)
    n_slice = int(off.shape[0] - 1)
    q_off = w.q_off[: n_sample + 1]
    q = w.q[: q_off[-1]]
    band = float(np.float32(BAND))
    res, cells = {}, 0
    t0 = time.perf_counter()
    for kind in (0, 1):
        ids, dist, st = oracle.knn(db, off, q, q_off, band=band, kind=kind, k=K, method=True,
                                   threads=threads, with_stats=True)
        res[kind] = (ids, dist)
        cells += int(st[:, 3].sum())
    dt = time.perf_counter() - t0
    scale = N_SERIES / n_slice
    return {"seconds": dt, "results": res, "n_slice": n_slice, "dp_cells": cells,
            "value": 2 * n_sample / (dt * scale)}


def cpu_baseline(w, n_sample: int = 0) -> dict:
    """The oracle as it stands, one query per host core, on the database
    prefix, extrapolated linearly to all N_SERIES series; plus a single-core
    figure (one query, one thread) as the paper reports one core."""
    cores = os.cpu_count() or 1
    n_sample = min(n_sample or cores, int(w.q_off.shape[0] - 1))
    threads = min(cores, n_sample)
    r = oracle_sample(w, n_sample, threads)
    one = oracle_sample(w, 1, 1)
    return {"value": r["value"], "unit": "queries/s", "cores": threads, "kind": "oracle",
            "sample": f"{n_sample} queries x the first {r['n_slice']} of {N_SERIES} series, "
                      f"DTW and DK, k={K}, band {BAND:g}, FP64 pruned scan (LB_Box, GDK, sparse "
                      f"DK, early abandoning), {threads} threads, {r['seconds']:.1f} s; "
                      f"queries/s extrapolated linearly in the number of series "
                      f"(x{N_SERIES / r['n_slice']:.4g})",
            "seconds": r["seconds"], "dp_cells": r["dp_cells"],
            "single_core": {"value": one["value"], "unit": "queries/s", "cores": 1,
                            "seconds": one["seconds"],
                            "sample": f"1 query x {r['n_slice']} series, DTW and DK, "
                                      f"extrapolated to {N_SERIES} series"},
            "_results": r["results"], "_n_sample": n_sample}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    # only the database prefix the oracle scans is drawn (series i depends on
    # the seed and i alone, the queries on neither)
    w = workload(1, ORACLE_SERIES)
    cores = os.cpu_count() or 1
    n_sample = min(args.cpu_sample or cores, N_QUERIES)
    threads = min(cores, n_sample)
    for _ in range(args.warmup):
        oracle_sample(w, n_sample, threads)
    secs = 0.0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        secs += oracle_sample(w, n_sample, threads)["seconds"]
    dt = time.perf_counter() - t0
    n_slice = min(ORACLE_SERIES, N_SERIES)
    scale = N_SERIES / n_slice
    value = 2 * n_sample * args.steps / (secs * scale)
    sample = (f"{n_sample} queries x the first {n_slice} of {N_SERIES} series per step, DTW and "
              f"DK, k={K}, band {BAND:g}, FP64 pruned scan, {threads} threads; queries/s "
              f"extrapolated linearly in the number of series (x{scale:.4g})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_series": N_SERIES,
                       "length": LENGTH or "50-1000", "d": D, "k": K, "band": BAND,
                       "sample_queries_per_step": n_sample, "oracle_series": n_slice},
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": threads,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def check_knn(ids, dist, oids, odist, kind) -> dict:
    """GPU k-NN rows against the oracle's: identical ids in order, distances
    within the relative tolerance of the distance."""
    ids, dist = np.asarray(ids), np.asarray(dist, dtype=np.float64)
    same_ids = bool(np.array_equal(ids, oids))
    fin = np.isfinite(odist)
    rel = np.abs(dist[fin] - odist[fin]) / np.maximum(np.abs(odist[fin]), 1e-30)
    worst = float(rel.max()) if rel.size else 0.0
    return {"ids_identical": same_ids, "max_rel_err": worst, "tol": TOL[kind],
            "pass": same_ids and worst <= TOL[kind] and
            bool(np.array_equal(np.isfinite(dist), fin))}


def sampled_eps_parity(w, kind, eps, ids, dist, counts, nq: int, n_others: int,
                       seed: int = 0) -> dict:
    """Full-size eps-NN check on sampled outputs: for each of the first nq
    queries the oracle computes (FP64) every returned series' distance and
    n_others random other series'; passes if the returned ones are within
    eps and agree within the tolerance, and no sampled other series is
    within eps (up to the tolerance at eps itself)."""
    import oracle
    rng = np.random.default_rng(seed)
    N = int(w.db_off.shape[0] - 1)
    band = float(np.float32(BAND))
    worst, ok = 0.0, True
    for qi in range(nq):
        got = [int(x) for x in ids[qi][: int(counts[qi])]]
        gs = set(got)
        others = [int(x) for x in rng.choice(N, size=min(n_others, N), replace=False)
                  if int(x) not in gs]
        sel = got + others
        pts = [w.series(i) for i in sel]
        b_off = np.zeros(len(sel) + 1, dtype=np.int64)
        np.cumsum([len(p) for p in pts], out=b_off[1:])
        q = w.query(qi)
        od = oracle.pairwise(q, np.array([0, q.shape[0]], dtype=np.int64), np.concatenate(pts),
                             b_off, np.zeros(len(sel), dtype=np.int64),
                             np.arange(len(sel), dtype=np.int64), band=band, kind=kind)
        gd = np.asarray(dist[qi][: len(got)], dtype=np.float64)
        rel = np.abs(gd - od[: len(got)]) / np.maximum(np.abs(od[: len(got)]), 1e-30)
        worst = max(worst, float(rel.max()) if rel.size else 0.0)
        ok &= bool(np.all(od[: len(got)] <= eps * (1 + TOL[kind])))
        ok &= bool(np.all(od[len(got):] > eps * (1 - TOL[kind])))
    return {"queries": nq, "others_per_query": n_others, "max_rel_err": worst,
            "tol": TOL[kind], "pass": bool(ok and worst <= TOL[kind])}


def sampled_parity(w, kind, ids, dist, nq: int, n_others: int, seed: int = 0) -> dict:
    """Full-size check on sampled outputs: for each of the first nq queries
    the oracle computes (FP64) the distance of every returned series and of
    n_others random other series.  Passes if the returned distances agree
    within the tolerance, the rows are ordered by (distance, id), and no
    sampled series is closer than the k-th result (ties by id)."""
    import oracle
    rng = np.random.default_rng(seed)
    N = int(w.db_off.shape[0] - 1)
    band = float(np.float32(BAND))
    worst, ok = 0.0, True
    for qi in range(nq):
        got = [int(x) for x in ids[qi] if x >= 0]
        others = [int(x) for x in rng.choice(N, size=min(n_others, N), replace=False)
                  if int(x) not in set(got)]
        sel = got + others
        pts = [w.series(i) for i in sel]
        b_off = np.zeros(len(sel) + 1, dtype=np.int64)
        np.cumsum([len(p) for p in pts], out=b_off[1:])
        b = np.concatenate(pts)
        q = w.query(qi)
        a_off = np.array([0, q.shape[0]], dtype=np.int64)
        pa = np.zeros(len(sel), dtype=np.int64)
        pb = np.arange(len(sel), dtype=np.int64)
        od = oracle.pairwise(q, a_off, b, b_off, pa, pb, band=band, kind=kind)
        gd = np.asarray(dist[qi][: len(got)], dtype=np.float64)
        rel = np.abs(gd - od[: len(got)]) / np.maximum(np.abs(od[: len(got)]), 1e-30)
        worst = max(worst, float(rel.max()) if rel.size else 0.0)
        keys = list(zip(gd.tolist(), got))
        ok &= keys == sorted(keys)
        if len(got) == ids.shape[1]:
            # a series outside the result is not closer than the k-th (equal
            # distances are ordered by id, so only "clearly closer" fails)
            kth = float(od[len(got) - 1])
            ok &= bool(np.all(od[len(got):] >= kth * (1 - TOL[kind])))
        else:
            # fewer than k finite results: every sampled series is infinite
            ok &= bool(np.all(~np.isfinite(od[len(got):])))
    return {"queries": nq, "others_per_query": n_others, "max_rel_err": worst,
            "tol": TOL[kind], "pass": bool(ok and worst <= TOL[kind])}


def run_gpu(args):
    import torch
    import torch.distributed as dist
    import paper_1811_11076_gb300 as kw
    from paper_1811_11076_gb300.shard import max_over_ranks, query_shard

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    kw.lib()

    t_setup = time.perf_counter()
    w = workload(world)
    nq = N_QUERIES
    (q0, q1), q_off = query_shard(w.q_off, rank, world, nq)
    q_host = np.ascontiguousarray(w.q[q0:q1])
    db_dev = torch.from_numpy(w.db).cuda()
    kinds = {"both": (kw.DTW, kw.DK), "dtw": (kw.DTW,), "dk": (kw.DK,)}[args.only]
    kname = {kw.DTW: "DTW", kw.DK: "DK"}
    seed_mode = {"greedy": kw.SEED_GREEDY, "lb": kw.SEED_LB, "none": kw.SEED_NONE,
                 "learned": kw.SEED_LEARNED}[args.seed]
    # one database handle per distance: each carries the encoder trained on
    # that distance (set-up, outside the timed region)
    dbs, train_info, encoders = {}, {}, {}
    for kind in kinds:
        dbs[kind] = kw.KnnDB(db_dev, w.db_off)
        if args.seed == "learned":
            enc = kw.Encoder(D, seed=11 + kind)
            if args.train_pairs > 0:
                train_info[kname[kind]] = enc.train(
                    dbs[kind], args.train_pairs, epochs=3, batch_pairs=2048, lr=2e-3,
                    distance=kind, band=BAND, seed=5 + kind)
            enc.attach(dbs[kind])
            encoders[kind] = enc
    del db_dev
    q_dev = torch.from_numpy(q_host).cuda()
    q_off_t = torch.from_numpy(q_off)
    out = {kind: (torch.empty((nq, K), dtype=torch.int64, device="cuda"),
                  torch.empty((nq, K), dtype=torch.float32, device="cuda"),
                  torch.empty(nq, dtype=torch.int64, device="cuda")) for kind in kinds}
    graph = BENCH[WORKLOAD]["graph"] and not args.no_graph

    def scan(kind, mode=seed_mode, profile=False, o=None):
        return dbs[kind].scan(q_dev, q_off_t, k=K, band=BAND, distance=kind, seed=mode,
                              out=o or out[kind], stats=True, profile=profile,
                              use_graph=graph and not profile)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # autotuner (set-up, outside the timed region): DP shape per distance
    shapes = {}
    r = int(np.float64(np.float32(BAND)) * LENGTH)
    for kind in kinds:
        if args.lb_compaction or args.lb_qtile:
            dbs[kind].set_lb_tile(kind, args.lb_qtile, 0, args.lb_compaction)
        if args.shape:
            P, G = (int(v) for v in args.shape.split(","))
            dbs[kind].set_dp_shape(kind, r, LENGTH, P, G)
        elif not args.no_autotune:
            nt = min(nq, 128)
            dbs[kind].autotune(q_dev[: int(q_off[nt])], q_off_t[: nt + 1], k=K, band=BAND,
                               distance=kind, seed=seed_mode)
        if LENGTH:
            shapes[kname[kind]] = dict(zip(("P", "G"), dbs[kind].get_dp_shape(kind, r, LENGTH)))
    setup_s = time.perf_counter() - t_setup

    # warm-up, then the timed steps: the production path (no stage events;
    # the counters come back with the status word every scan reads anyway)
    warmup = max(args.warmup, 3)
    for _ in range(warmup):
        for kind in kinds:
            scan(kind)
    collected = []
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            for kind in kinds:
                collected.append((kind, scan(kind)[2]))
        e1.record(stream)
        barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), device="cuda")
    total_queries = nq * len(kinds) * args.steps * world
    value = total_queries / (ms / 1000.0)
    headline = {kind: (out[kind][0].clone(), out[kind][1].clone()) for kind in kinds}

    # stage split: one profiled eager scan per distance, outside the timed region
    prof = {kind: scan(kind, profile=True)[2] for kind in kinds}
    detail = {}
    for kind in kinds:
        sts = [s for k_, s in collected if k_ == kind]
        agg = {key: sum(s[key] for s in sts) for key in sts[0]}
        p = prof[kind]
        ms_scan = agg["ms_total"] / len(sts)
        detail[kname[kind]] = {
            "queries_per_s": nq * len(sts) / (agg["ms_total"] / 1000.0),
            "ms_per_scan": ms_scan,
            "dp_gcups": p["dp_cells"] / (p["ms_dp"] / 1000.0) / 1e9 if p["ms_dp"] else None,
            "profiled_scan": {key: p[key] for key in ("ms_total", "ms_seed", "ms_lb", "ms_dp",
                                                      "ms_finalize")},
            "dp_calls_per_query": agg["dp_calls"] / (nq * len(sts)),
            "dp_abandoned_frac": agg["dp_abandoned"] / max(agg["dp_calls"], 1),
            "lb_pruned_frac": (agg["lb_pruned"] + agg["lb_pruned_late"]) / max(agg["pairs"], 1),
            "coarse_pruned_frac": agg["lb_coarse_pruned"] / max(agg["pairs"], 1),
            "lb_points_per_query": agg["lb_points"] / (nq * len(sts)),
            "coarse_segments_per_query": agg["lb_segments"] / (nq * len(sts)),
            "dp_cells_per_query": agg["dp_cells"] / (nq * len(sts)),
            "seed_cells_per_query": agg["seed_cells"] / (nq * len(sts)),
            "reranked": agg["reranked"] // len(sts),
        }
    launches = sum(s["launches"] for _, s in collected)

    # roofline of the dominant kernel (largest share of the profiled scans'
    # stage time).  Both stages are plain FP32-ALU work: the LB_Box stream with
    # a tile of queries per pass does 4 lane operations per (query, element)
    # it evaluates (two subtractions, a max, an FMA; the DK max form adds one
    # max per point), the DP 2d+3 per band cell.  Peak = SMs x 128 FP32 lanes
    # x the maximum SM clock.
    hbm_gbs, sm_max_mhz, peak_src = peaks()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak = n_sm * 128 * sm_max_mhz * 1e6 / 1e12
    stage = {"seed": 0.0, "lb": 0.0, "dp": 0.0, "finalize": 0.0}
    dp_ops = lb_ops = dp_units = 0.0
    for kind, s in prof.items():
        for k_ in stage:
            stage[k_] += s[f"ms_{k_}"]
        dp_ops += s["dp_cells"] * (2 * D + 3)
        dp_units += s["dp_cells"]
        # exact LB_Box points and coarse segments cost the same per element
        lb_ops += (s["lb_points"] + s["lb_segments"]) * (4 * D + (1 if kind == kw.DK else 0))
    clocks = clk.summary()
    share = {k_: v / max(sum(stage.values()), 1e-12) for k_, v in stage.items()}

    def alu_roof(kernel, ops, ms_, units=0.0):
        achieved = ops / (ms_ / 1000.0) / 1e12 if ms_ else 0.0
        per_unit = TRAFFIC_PER_UNIT.get((kernel, WORKLOAD))
        traffic = None
        if per_unit and units:
            traffic = {"bytes": per_unit[0] * units, "bytes_per_unit": per_unit[0],
                       "units": units, "source": per_unit[1]}
        r_ = {"kernel": kernel, "bound": "alu", "achieved": achieved, "peak": alu_peak,
              "unit": "Tops/s (FP32 lane ops)", "frac": achieved / alu_peak,
              "traffic": traffic,
              "peak_source": f"{n_sm} SMs x 128 FP32 lanes x {sm_max_mhz:.0f} MHz "
                             f"(max SM clock, {peak_src})",
              "timing": "CUDA events around the stage in one profiled scan per distance"}
        if clocks.get("sm_mhz"):
            r_["frac_at_sampled_clock"] = achieved / (n_sm * 128 * clocks["sm_mhz"] * 1e6 / 1e12)
        return r_

    # which LB_Box kernels ran (the library reports a bit mask per scan)
    lb_bits = 0
    for s in list(prof.values()) + [s for _, s in collected]:
        lb_bits |= int(s.get("lb_kernels", 0))
    lb_name = "+".join(n_ for b_, n_ in ((16, "lb_coarse_kernel+lb_pair_kernel"), (1, "lb_kernel"),
                                         (2, "lb_multi_kernel"), (4, "lb_win_kernel"),
                                         (8, "lb_compact_kernel"))
                       if lb_bits & b_) or "lb_multi_kernel"
    stage_roofs = {"lb": alu_roof(lb_name, lb_ops, stage["lb"]),
                   "dp": alu_roof("dp_kernel", dp_ops, stage["dp"], dp_units)}
    dominant = "lb" if stage["lb"] >= stage["dp"] else "dp"
    roof = dict(stage_roofs[dominant])
    roof["stage_share"] = share
    roof["other_stage"] = stage_roofs["dp" if dominant == "lb" else "lb"]

    # end to end through the public API with host buffers: H2D of queries and
    # D2H of results inside the timed region
    q_pin = torch.from_numpy(q_host).pin_memory()
    ids_h = torch.empty((nq, K), dtype=torch.int64).pin_memory()
    dst_h = torch.empty((nq, K), dtype=torch.float32).pin_memory()
    cnt_h = torch.empty(nq, dtype=torch.int64).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for kind in kinds:
            dbs[kind].scan(q_pin, q_off_t, k=K, band=BAND, distance=kind, seed=seed_mode,
                           out=(ids_h, dst_h, cnt_h), use_graph=graph)
    barrier()
    e2e_dt = max_over_ranks(time.perf_counter() - t0, device="cuda")
    h2d = (q_host.nbytes + q_off.nbytes) * len(kinds)
    d2h = (ids_h.numel() * 8 + dst_h.numel() * 4 + cnt_h.numel() * 8) * len(kinds)
    e2e = {"value": nq * len(kinds) * e2e_steps * world / e2e_dt, "unit": "queries/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # the comparators, timed like the headline (CUDA events around whole
    # scans on the same queries, same tuned shapes): the plain GPU scan
    # (batched, LB_Box-ordered seeding, no encoder), the paper's greedy
    # pre-pass (Section 4.3), and the same learned flow with an untrained
    # encoder (what the training itself buys)
    comparators = {}
    if rank == 0 and not args.no_variants:
        n_cmp = max(1, min(args.steps, 2))
        cmp_db = None
        if args.seed == "learned":
            cmp_db = kw.KnnDB(w.db, w.db_off)
            untrained = kw.Encoder(D, seed=99)
            untrained.attach(cmp_db)
        modes = [("plain_lb", kw.SEED_LB, None), ("greedy", kw.SEED_GREEDY, None)]
        if cmp_db is not None:
            modes.append(("learned_untrained", kw.SEED_LEARNED, cmp_db))
        modes.append(("no_coarse_stage", seed_mode, None))
        for kind in kinds:
            for mname, mode, other in modes:
                h = other or dbs[kind]
                h.set_lb_cascade(kind, 1 if mname == "no_coarse_stage" else 0)
                if other is not None:
                    h.set_lb_tile(kind, *dbs[kind].get_lb_tile(kind))
                    if LENGTH:
                        h.set_dp_shape(kind, r, LENGTH, *dbs[kind].get_dp_shape(kind, r, LENGTH))
                o = (torch.empty_like(out[kind][0]), torch.empty_like(out[kind][1]),
                     torch.empty_like(out[kind][2]))
                h.scan(q_dev, q_off_t, k=K, band=BAND, distance=kind, seed=mode, out=o)
                st_sum = None
                torch.cuda.synchronize()
                c0 = torch.cuda.Event(enable_timing=True)
                c1 = torch.cuda.Event(enable_timing=True)
                c0.record(stream)
                for _ in range(n_cmp):
                    _, _, st = h.scan(q_dev, q_off_t, k=K, band=BAND, distance=kind, seed=mode,
                                      out=o, stats=True)
                    st_sum = st if st_sum is None else {k_: st_sum[k_] + st[k_] for k_ in st}
                c1.record(stream)
                c1.synchronize()
                cms = c0.elapsed_time(c1)
                same = bool(torch.equal(o[0], headline[kind][0]) and
                            torch.equal(o[1], headline[kind][1]))
                dbs[kind].set_lb_cascade(kind, 0)
                comparators[f"{kname[kind]}/{mname}"] = {
                    "queries_per_s": nq * n_cmp / (cms / 1000.0), "scans_timed": n_cmp,
                    "identical_results": same,
                    "ub_walks": st_sum["ub_walks"] // n_cmp,
                    "lb_points": st_sum["lb_points"] // n_cmp,
                    "dp_calls": st_sum["dp_calls"] // n_cmp,
                    "dp_cells": (st_sum["dp_cells"] + st_sum["seed_cells"]) // n_cmp}
        if cmp_db is not None:
            cmp_db.close()
            untrained.close()
    headline_cmp = {}
    for kind in kinds:
        base = comparators.get(f"{kname[kind]}/plain_lb")
        if base:
            headline_cmp[kname[kind]] = detail[kname[kind]]["queries_per_s"] / base["queries_per_s"]

    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world,
            "steps": args.steps, "warmup": warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_series": N_SERIES,
                       "length": LENGTH or "50-1000", "d": D, "queries_per_gpu": nq, "k": K,
                       "band": BAND, "distances": [kname[k_] for k_ in kinds],
                       "seed": SEED_DESC[args.seed], "cuda_graph": graph, "batched": True,
                       "l2": f"inputs larger than L2 ({w.db.nbytes / 1e6:.0f} MB database)",
                       "parallelism": f"replicated database, queries sharded x{world}"},
            "roofline": roof, "clocks": clocks, "gpu_launches": launches, "e2e": e2e,
            "per_distance": detail, "vs_plain_gpu_scan": headline_cmp,
            "comparators": comparators, "dp_shape": shapes, "encoder_training": train_info,
            "setup_s": setup_s,
        }

    # the eps-NN form: eps = the 1st percentile of the FP32 distances of the
    # batch's queries to a seeded sample of 10,000 series (knn_pairwise on
    # the GPU, pooled over queries: the scan takes one eps); the result sets
    # are large (about 1 % of the database on average)
    eps_nn = {}
    if rank == 0 and not args.no_eps:
        rng = np.random.default_rng(123)
        samp = rng.choice(N_SERIES, size=min(10_000, N_SERIES), replace=False)
        s_pts = np.concatenate([w.series(int(i)) for i in samp])
        s_off = np.zeros(len(samp) + 1, dtype=np.int64)
        np.cumsum([w.series(int(i)).shape[0] for i in samp], out=s_off[1:])
        s_dev, s_off_dev = torch.from_numpy(s_pts).cuda(), torch.from_numpy(s_off).cuda()
        q_off_dev = torch.from_numpy(q_off).cuda()
        cap = 1 << 16
        for kind in kinds:
            pa = torch.arange(nq, device="cuda").repeat_interleave(len(samp))
            pb = torch.arange(len(samp), device="cuda").repeat(nq)
            dd, _ = kw.pairwise(q_dev, q_off_dev, s_dev, s_off_dev, pa, pb, band=BAND,
                                distance=kind)
            flat = dd.float().flatten()
            kth = max(1, int(0.01 * flat.numel()))
            eps_all = float(np.float32(torch.kthvalue(flat.cpu(), kth).values.item()))
            del dd, flat, pa, pb
            oi = torch.empty((nq, cap), dtype=torch.int64, device="cuda")
            od = torch.empty((nq, cap), dtype=torch.float32, device="cuda")
            oc = torch.empty(nq, dtype=torch.int64, device="cuda")
            dbs[kind].scan(q_dev, q_off_t, k=0, eps=eps_all, eps_capacity=cap, band=BAND,
                           distance=kind, out=(oi, od, oc))
            torch.cuda.synchronize()
            c0 = torch.cuda.Event(enable_timing=True)
            c1 = torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            n_eps = max(1, min(args.steps, 2))
            for _ in range(n_eps):
                _, _, _, st = dbs[kind].scan(q_dev, q_off_t, k=0, eps=eps_all, eps_capacity=cap,
                                             band=BAND, distance=kind, out=(oi, od, oc),
                                             stats=True)
            c1.record(stream)
            c1.synchronize()
            cnt = oc.cpu().numpy()
            rec = {"queries_per_s": nq * n_eps / (c0.elapsed_time(c1) / 1000.0),
                   "eps": eps_all, "eps_rule": "1st percentile of the FP32 distances of "
                   "the batch's queries to 10,000 sampled series (pooled)",
                   "mean_results": float(cnt.mean()), "max_results": int(cnt.max()),
                   "capacity": cap, "dp_calls_per_query": st["dp_calls"] / nq}
            if not args.no_parity:
                rec["parity"] = sampled_eps_parity(w, kind, eps_all, oi.cpu().numpy(),
                                                   od.cpu().numpy(), cnt, 4, 96, seed=kind)
            eps_nn[kname[kind]] = rec
        del s_dev, s_off_dev
    if rank == 0:
        line["eps_nn"] = eps_nn

    # the LB_Box stream for one query (Section 3 Eq. 1 against every series,
    # the single-query streaming kernel): database bytes / time, against HBM
    if rank == 0 and not args.no_eps:
        hbm_gbs, _, peak_src = peaks()
        db_bytes = int(w.db.nbytes)
        qi = torch.from_numpy(w.query(0)).cuda()
        dbs[kinds[0]].lb_box(qi, BAND, 0)
        torch.cuda.synchronize()
        l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0.record(stream)
        for i in range(3):
            dbs[kinds[0]].lb_box(torch.from_numpy(w.query(i)).cuda(), BAND, 0)
        l1.record(stream)
        l1.synchronize()
        ms_lb = l0.elapsed_time(l1) / 3
        gbs = db_bytes / (ms_lb / 1000.0) / 1e9
        line["lb_single_query_stream"] = {
            "kernel": "lb_kernel (knn_lb_box: envelope, stream, scatter)",
            "ms": ms_lb, "database_bytes": db_bytes, "achieved_gbs": gbs, "peak_gbs": hbm_gbs,
            "frac": gbs / hbm_gbs, "peak_source": peak_src}

    # parity of the measured configuration against the oracle
    if rank == 0 and not args.no_parity:
        par = {}
        hcpu = {kind: (headline[kind][0].cpu().numpy(), headline[kind][1].cpu().numpy())
                for kind in kinds}
        for kind in kinds:
            par[f"{kname[kind]}/full_size_sampled"] = sampled_parity(
                w, kind, *hcpu[kind], min(PARITY_QUERIES, nq), PARITY_OTHERS, seed=kind)
        line["parity"] = par
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(w, args.cpu_sample)
        res, ns = cb.pop("_results"), cb.pop("_n_sample")
        line["cpu_baseline"] = cb
        if not args.no_parity:
            # the GPU on the same database prefix and queries, same flow
            sdb_pts, sdb_off = db_prefix(w, ORACLE_SERIES)
            full = sdb_off.shape[0] - 1 >= N_SERIES
            for kind in kinds:
                if full:
                    gi, gd = (x[:ns] for x in hcpu[kind])
                else:
                    sdb = kw.KnnDB(sdb_pts, sdb_off)
                    if kind in encoders:
                        encoders[kind].attach(sdb)
                    gi, gd = sdb.scan(q_dev[: int(q_off[ns])], q_off_t[: ns + 1], k=K,
                                      band=BAND, distance=kind, seed=seed_mode)
                    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
                    sdb.close()
                c = check_knn(gi, gd, *res[kind], kind)
                c.update(queries=ns, series=int(sdb_off.shape[0] - 1))
                line["parity"][f"{kname[kind]}/database_prefix_exact"] = c
        line["parity"]["pass"] = all(v["pass"] for v in line["parity"].values()
                                     if isinstance(v, dict))
    elif rank == 0 and not args.no_parity:
        line["parity"]["pass"] = all(v["pass"] for v in line["parity"].values())
    if rank == 0:
        print(json.dumps(line), flush=True)
    for e_ in encoders.values():
        e_.close()
    for d_ in dbs.values():
        d_.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def tightness_table(kw, dims, lengths, n_pairs: int, band: float, data: str, seed: int = 0):
    """Mean LB_Box / DTW over random pairs for every (d, n) (Section 3's
    Theorem: the ratio falls as d grows).  data "iid": elements U[0, 1]
    (the Theorem's setting); "classes": random pairs of the class-structured
    synthetic series.  LB_Box(T, env(S)) and DTW(S, T) on the GPU."""
    import torch
    from synthdata import make_workload
    rng = np.random.default_rng(seed)
    rows = []
    for d in dims:
        for n in lengths:
            if data == "iid":
                S = rng.random((n_pairs, n, d), dtype=np.float32)
                T = rng.random((n_pairs, n, d), dtype=np.float32)
            else:
                w = make_workload(n_series=2 * n_pairs, n_queries=1, d=d, length=n, n_classes=10,
                                  seed=seed + d * 1000 + n)
                X = w.db.reshape(2 * n_pairs, n, d)
                S, T = X[:n_pairs], X[n_pairs:]
            off = np.arange(n_pairs + 1, dtype=np.int64) * n
            db = kw.KnnDB(torch.from_numpy(T.reshape(-1, d)).cuda(), off)
            lb = np.empty(n_pairs)
            for i in range(n_pairs):
                lb[i] = float(db.lb_box(torch.from_numpy(S[i]).cuda(), band, 0)[i])
            db.close()
            pa = torch.arange(n_pairs, dtype=torch.int64, device="cuda")
            dtw, _ = kw.pairwise(torch.from_numpy(S.reshape(-1, d)).cuda(),
                                 torch.from_numpy(off).cuda(),
                                 torch.from_numpy(T.reshape(-1, d)).cuda(),
                                 torch.from_numpy(off).cuda(), pa, pa, band=band, distance=kw.DTW)
            dtw = dtw.cpu().numpy().astype(np.float64)
            ok = dtw > 0
            rows.append({"d": d, "n": n, "mean_ratio": float(np.mean(lb[ok] / dtw[ok])),
                         "ratio_of_means": float(lb.mean() / dtw.mean()), "pairs": int(ok.sum())})
    return rows


def accuracy_table(kw, dims, lengths, n_series: int, n_queries: int, band: float,
                   seed: int = 0, noise: float = 0.1, n_classes: int = 10):
    """1-NN classification accuracy of DTW and DK (the exact scan with k = 1) on
    the class-structured synthetic data (instance noise N(0, noise^2)), for
    every (d, n)."""
    import torch
    from synthdata import make_workload
    rows = []
    for d in dims:
        for n in lengths:
            w = make_workload(n_series=n_series, n_queries=n_queries, d=d, length=n,
                              n_classes=n_classes, seed=seed + d * 1000 + n, noise_sigma=noise)
            db = kw.KnnDB(torch.from_numpy(w.db).cuda(), w.db_off)
            row = {"d": d, "n": n}
            for kind, name in ((kw.DTW, "dtw"), (kw.DK, "dk")):
                ids, _ = db.scan(torch.from_numpy(w.q).cuda(), w.q_off, k=1, band=band,
                                 distance=kind, seed=kw.SEED_LB)
                ids = ids.cpu().numpy()[:, 0]
                row["acc_" + name] = float(np.mean(w.db_labels[ids] == w.q_labels))
                row["ids_" + name] = ids.tolist() if n_queries <= 64 else None
            db.close()
            rows.append(row)
    return rows


def lb_stream(args) -> dict:
    """The LB_Box stream of one query (Section 3 Eq. 1 against every series;
    the single-query streaming kernel via knn_lb_box) on the workload's
    database: the call's time, and the database bytes it reads."""
    import torch
    import paper_1811_11076_gb300 as kw
    select_workload(args.workload)
    if args.series:
        globals()["N_SERIES"] = args.series
    w = workload(1)
    db = kw.KnnDB(torch.from_numpy(w.db).cuda(), w.db_off)
    qs = [torch.from_numpy(w.query(i)).cuda() for i in range(8)]
    for form in (0, 1):
        db.lb_box(qs[0], BAND, form)
    torch.cuda.synchronize()
    out = {}
    for form in (0, 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for q in qs:
            db.lb_box(q, BAND, form)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / len(qs)
        out[f"form{form}"] = {"ms_per_call": ms, "gbs_per_call": w.db.nbytes / ms / 1e6}
    db.close()
    hbm, _, src = peaks()
    return {"workload": WORKLOAD, "n_series": N_SERIES, "database_bytes": int(w.db.nbytes),
            "calls": out, "peak_gbs": hbm, "peak_source": src,
            "note": "call time includes the query upload, envelope and scatter kernels"}


def cascade_study(args) -> dict:
    """What a tighter second bound would prune, on the d = 16 workload's first
    series (default 20,000) and 4 queries, DTW (Section 3 Eq. 1 and the
    bounds that tighten it).  The threshold is each query's exact 50-th
    distance (the scan's result); the candidates are the series whose LB_Box
    (envelope on the query) is within it, i.e. the pairs the DP receives.
    For them: the reverse bound LB_Box(Q, env(X)) (the GPU component with the
    roles swapped: a one-series database holding the query) and the
    LB_Improved-style bound (LB_Box plus the query against the envelope of the
    series' projection onto the query's envelope, FP64 numpy).  Reports how
    many DP pairs each would remove, and the coarse segment bound's pass rate
    at the database's segment width."""
    import torch
    from scipy.ndimage import maximum_filter1d, minimum_filter1d
    import paper_1811_11076_gb300 as kw
    select_workload("highdim_d16_n500k_L512")
    n_series = args.series or 20000
    w = workload(1, n_series=n_series)
    L = LENGTH
    r = int(np.float64(np.float32(BAND)) * L)
    db = kw.KnnDB(torch.from_numpy(w.db).cuda(), w.db_off)
    _, W = db.get_lb_cascade(0)

    def env(a):
        return (minimum_filter1d(a, size=2 * r + 1, axis=0, mode="nearest"),
                maximum_filter1d(a, size=2 * r + 1, axis=0, mode="nearest"))

    def box_sum(x, lo, hi):
        e = np.maximum(np.maximum(lo - x, x - hi), 0.0)
        return float(np.sum(e * e))

    rows = []
    for qi in range(4):
        q = w.query(qi)
        qd = torch.from_numpy(q).cuda()
        _, dist = db.scan(qd, np.array([0, L]), k=K, band=BAND, distance=kw.DTW,
                          seed=kw.SEED_LB)
        thr = float(dist[0, -1])
        fwd = db.lb_box(qd, BAND, 0).cpu().numpy().astype(np.float64)
        seg = db.lb_seg(qd, BAND, 0).cpu().numpy().astype(np.float64)
        surv = np.nonzero(fwd <= thr)[0]
        qdb = kw.KnnDB(qd, np.array([0, L]))
        q64 = q.astype(np.float64)
        qlo, qhi = env(q64)
        rev = np.empty(surv.size)
        imp = np.empty(surv.size)
        for j, c in enumerate(surv):
            x = w.series(int(c))
            rev[j] = float(qdb.lb_box(torch.from_numpy(x).cuda(), BAND, 0)[0])
            h = np.clip(x.astype(np.float64), qlo, qhi)
            hlo, hhi = env(h)
            imp[j] = fwd[c] + box_sum(q64, hlo, hhi)
        qdb.close()
        rows.append({"query": qi, "threshold": thr, "dp_pairs": int(surv.size),
                     "removed_by_reverse": int(np.sum(rev > thr)),
                     "removed_by_improved": int(np.sum(imp > thr)),
                     "removed_by_either": int(np.sum((rev > thr) | (imp > thr))),
                     "coarse_pass": float(np.mean(seg <= thr)),
                     "lb_box_pass": float(np.mean(fwd <= thr))})
    db.close()
    tot = sum(x["dp_pairs"] for x in rows)
    return {"workload": WORKLOAD, "n_series": n_series, "k": K, "band": BAND,
            "segment_width": W, "queries": rows, "dp_pairs": tot,
            "removed_by_either_frac": sum(x["removed_by_either"] for x in rows) / max(tot, 1)}


def run_experiment(args):
    """Tightness sweep (the Theorem's trend) or 1-NN accuracy, one JSON line."""
    import paper_1811_11076_gb300 as kw
    kw.lib()
    t0 = time.perf_counter()
    if args.experiment == "cascade":
        line = {"experiment": "cascade", **cascade_study(args)}
        line["seconds"] = time.perf_counter() - t0
        print(json.dumps(line), flush=True)
        return 0
    if args.experiment == "lbstream":
        line = {"experiment": "lbstream", **lb_stream(args)}
        line["seconds"] = time.perf_counter() - t0
        print(json.dumps(line), flush=True)
        return 0
    if args.experiment == "tightness":
        rows = {data: tightness_table(kw, (1, 2, 4, 8, 16),
                                      (32, 64, 128, 256, 512), 128, 0.1, data)
                for data in ("iid", "classes")}
        line = {"experiment": "tightness", "quantity": "LB_Box / DTW, band 10 %",
                "pairs_per_cell": 128, "rows": rows}
    else:
        rows = {}
        for noise in (3.0, 6.0):
            rows[f"noise {noise}"] = accuracy_table(kw, (1, 2, 4, 8, 16), (64, 128, 256), 5000,
                                                    400, 0.1, noise=noise, n_classes=50)
            for r in rows[f"noise {noise}"]:
                r.pop("ids_dtw", None)
                r.pop("ids_dk", None)
        line = {"experiment": "accuracy",
                "quantity": "1-NN accuracy, 50 classes of warped random walks, band 10 %",
                "series": 5000, "queries": 400, "rows": rows}
    line["seconds"] = time.perf_counter() - t0
    print(json.dumps(line), flush=True)
    return 0


SUB_METRIC = "exact subsequence search queries/sec and GCUPS (DTW & DK, free start and end)"


def sub_cpu_baseline(w, n_sample: int) -> dict:
    """The FP64 oracle's subsequence search on a sample of queries, one query
    per thread (ctypes releases the GIL)."""
    import concurrent.futures
    import oracle
    oracle.lib()
    n_sample = min(n_sample, int(w.q_off.shape[0] - 1))
    cores = min(os.cpu_count() or 1, n_sample)
    t64 = w.t.astype(np.float64)
    jobs = [(kind, w.q[w.q_off[i]:w.q_off[i + 1]].astype(np.float64))
            for i in range(n_sample) for kind in (0, 1)]
    t0 = time.perf_counter()
    with concurrent.futures.ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(lambda j: oracle.sub_distance(j[0], j[1], t64), jobs))
    dt = time.perf_counter() - t0
    return {"value": len(jobs) / dt, "unit": "queries/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_sample} queries x {w.t.shape[0]} points, DTW and DK, FP64 "
                      f"free-start/free-end DP, {cores} threads", "seconds": dt}


def run_subseq(args):
    """Subsequence search workloads: every query against one long series."""
    from synthdata import LONG_SERIES, make_long_series
    cfg = dict(LONG_SERIES[args.workload])
    if args.queries:
        cfg["n_queries"] = args.queries
    w = make_long_series(**cfg)
    if args.impl == "reference":
        steps = []
        n_sample = args.cpu_sample or (os.cpu_count() or 1)
        for _ in range(args.warmup + args.steps):
            steps.append(sub_cpu_baseline(w, n_sample))
        vals = [x["value"] for x in steps[args.warmup:]]
        value = len(vals) / sum(1.0 / v for v in vals)
        cb = dict(steps[-1])
        cb["value"] = value
        print(json.dumps({"impl": "reference", "metric": SUB_METRIC, "value": value,
                          "unit": "queries/s", "n_gpus": args.gpus, "steps": args.steps,
                          "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": args.workload, **cfg}, "cpu_baseline": cb,
                          "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return 0
    import torch
    import paper_1811_11076_gb300 as kw
    kw.lib()
    q, qo, t = (torch.from_numpy(x).cuda() for x in (w.q, w.q_off, w.t))
    nq, m, n, d = int(qo.shape[0] - 1), int(cfg["q_length"]), int(w.t.shape[0]), w.d
    for _ in range(max(args.warmup, 3)):
        for kind in (kw.DTW, kw.DK):
            kw.subseq(q, qo, t, distance=kind)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        ms = {kw.DTW: 0.0, kw.DK: 0.0}
        for _ in range(args.steps):
            for kind in (kw.DTW, kw.DK):
                ev[0].record(stream)
                kw.subseq(q, qo, t, distance=kind)
                ev[1].record(stream)
                ev[1].synchronize()
                ms[kind] += ev[0].elapsed_time(ev[1])
    total_ms = ms[kw.DTW] + ms[kw.DK]
    value = 2 * nq * args.steps / (total_ms / 1000.0)
    # rows per warp: 32 P >= m; every cell of the 32 P x (n + m - 1 rounded) sweep is
    # computed, the algorithmic work counts the m x n cells at 2d+3 lane ops each
    cells = nq * m * n
    hbm_gbs, sm_max_mhz, peak_src = peaks()
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    alu_peak = n_sm * 128 * sm_max_mhz * 1e6 / 1e12
    achieved = cells * (2 * d + 3) * 2 * args.steps / (total_ms / 1000.0) / 1e12
    clocks = clk.summary()
    roof = {"kernel": "subseq_kernel", "bound": "alu", "achieved": achieved, "peak": alu_peak,
            "unit": "Tops/s (FP32 lane ops)", "frac": achieved / alu_peak,
            "traffic": None,
            "peak_source": f"{n_sm} SMs x 128 FP32 lanes x {sm_max_mhz:.0f} MHz (max SM clock, "
                           f"{peak_src})"}
    # end to end from host buffers (series and queries copied in every call)
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        for kind in (kw.DTW, kw.DK):
            v, e = kw.subseq(w.q, w.q_off, w.t, distance=kind)
    e2e_dt = time.perf_counter() - t0
    line = {"metric": SUB_METRIC, "value": value, "unit": "queries/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "d": d, "queries": nq, "m": m,
                       "band": "none (free start and end)",
                       "l2": f"series {w.t.nbytes / 1e6:.0f} MB, streamed once per query"},
            "per_distance": {("DTW" if k_ == kw.DTW else "DK"): {
                "ms": ms[k_] / args.steps, "queries_per_s": nq * args.steps / (ms[k_] / 1000.0),
                "gcups": cells * args.steps / (ms[k_] / 1000.0) / 1e9} for k_ in ms},
            "roofline": roof, "clocks": clocks, "gpu_launches": 5 * 2 * args.steps,
            "e2e": {"value": 2 * nq * e2e_steps / e2e_dt, "unit": "queries/s",
                    "h2d_bytes_per_step": 2 * (w.q.nbytes + w.q_off.nbytes + w.t.nbytes),
                    "d2h_bytes_per_step": 2 * nq * 12}}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = sub_cpu_baseline(w, args.cpu_sample or (os.cpu_count() or 1))
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=0,
                    help="queries of the oracle's timed sample (0: one per host core)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--seed", default="learned", choices=["greedy", "lb", "none", "learned"])
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the comparators (plain GPU scan, greedy, untrained encoder)")
    ap.add_argument("--train-pairs", type=int, default=TRAIN_PAIRS,
                    help="pairs the encoder trains on (0: untrained, for profiling captures)")
    ap.add_argument("--no-eps", action="store_true",
                    help="skip the eps-NN form and the single-query LB_Box stream")
    ap.add_argument("--no-parity", action="store_true",
                    help="skip the oracle checks of the measured results")
    from synthdata import LONG_SERIES
    ap.add_argument("--workload", default=WORKLOAD, choices=list(BENCH) + list(LONG_SERIES))
    ap.add_argument("--queries", type=int, default=0,
                    help="queries per GPU (default: the workload's; smaller only for profiling)")
    ap.add_argument("--series", type=int, default=0,
                    help="database series (default: the workload's; smaller only for profiling)")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--only", default="both", choices=["both", "dtw", "dk"])
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--shape", default="", help="P,G: fix the DP shape instead of tuning it")
    ap.add_argument("--experiment", default="",
                    choices=["", "tightness", "accuracy", "lbstream", "cascade"],
                    help="instead of the throughput line: the LB_Box tightness sweep, the "
                         "1-NN accuracy of DTW and DK, the single-query LB_Box stream alone, "
                         "or what tighter second bounds would prune")
    ap.add_argument("--lb-qtile", type=int, default=0, choices=[0, 4, 8, 16],
                    help="queries per LB_Box pass (0: 16, or tuned)")
    ap.add_argument("--lb-compaction", type=int, default=0, choices=[0, 1, 2],
                    help="LB_Box compaction: 0 automatic, 1 never, 2 always")
    args = ap.parse_args()
    if args.experiment:
        return run_experiment(args)
    if args.workload in LONG_SERIES:
        return run_subseq(args)
    select_workload(args.workload)
    if args.queries:
        globals()["N_QUERIES"] = args.queries
    if args.series:
        globals()["N_SERIES"] = args.series
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
