#!/usr/bin/env python
"""Throughput of exact cosine k-NN phase-order suggestion on GB300.

One step = one pass of the whole suggestion path over a batch of queries
against a device-resident database of explored kernels (Sec. 4 of Nobre, Reis
and Cardoso): query normalisation and codes, the database scan with fused
candidate lists, certification, FP32 rerank and binary64 rescoring, and the
gather of the neighbours' phase orders. The database itself is prepared once
(fs_build_db) before timing, as a reference set is in the paper.

Default workload: 16,777,216 database rows x 256 features, 8,192 queries,
k = 3, phase orders of 1-128 pass IDs, BF16 tensor-core scan with certified
FP32 / binary64 rerank (synthetic instruction-mix vectors standing in for the
paper's MILEPOST features). ``--impl reference`` times the CPU oracle
instead, on a bounded sample of the same workload.

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import os

_NCPU = os.cpu_count() or 1
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, str(_NCPU))

import argparse  # noqa: E402
import json  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import fsgen  # noqa: E402

METRIC = "query×DB pairs/s and top-k queries/s vs plain FP32 scan at recall 1.0; p99 ms"
UNIT = "pairs/s"
# FP32 SIMT peak: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (maximum SM clock)
FP32_SIMT_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# DRAM bytes (read + write) per launch of the dominant kernel from an ncu
# capture of the current version of that kernel, keyed by (kernel, workload,
# precision), with the scan plan tuning it was captured under (None: the
# default plan); absent (reported as null) until captured. Source: the
# matching summary under profiles/.
TRAFFIC_BYTES = {
    # a 1,048,576-row cut (594.8 MB per launch) scaled by the rows to the full
    # 16,777,216 rows: profiles/scan_bf16_precision.md
    ("scan_bf16", "precision", "bf16"): (9.45e9, None),
    # the first 64 of the 512 databases (653.3 MB per launch) scaled by the rows
    # to all 19,138,960: profiles/scan_bf16_batching.md
    ("scan_bf16", "batching", "bf16"): (5.37e9, {"items_per_block": 1, "list_len": 16}),
    ("scan_bf16", "fp32_scale", "bf16"): (310.1e6, None),   # profiles/scan_bf16_fp32_scale.md
    # (FP8: the scan changed after its capture in profiles/scan_fp8_fp32_scale.md,
    # 202.9 MB per launch then, so no captured traffic is attached)
    ("scan_fp32", "fp32_scale", "fp32"): (644.2e6, None),   # profiles/scan_fp32_fp32_scale.md
}


def captured_traffic(kernel, workload, prec, metric, tuning, full_size):
    """The captured DRAM bytes per launch when this run matches the capture:
    the whole workload, the cosine and the captured plan tuning."""
    got = TRAFFIC_BYTES.get((kernel, workload, prec))
    if got is None or not full_size or metric != "cosine":
        return None
    nbytes, plan = got
    if plan is None:
        return nbytes if tuning is None else None
    if tuning is None:
        return None
    used = {k: v for k, v in tuning.items() if v}
    return nbytes if all(used.get(k) == v for k, v in plan.items()) else None


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return p, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, \
            "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]
        return False

    def summary(self):
        rows = []
        for ln in getattr(self, "lines", []):
            p = [c.strip() for c in ln.split(",")]
            if len(p) < 9:
                continue
            rows.append(p)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        idxs = sorted({r[0] for r in rows})
        pick = idxs[self.idx] if self.idx < len(idxs) else idxs[0]
        rows = [r for r in rows if r[0] == pick]

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(pw) if pw else None}


def setup_dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, device, world: int) -> float:
    """The largest of every rank's `value` (all ranks get it). The device is
    the process group's: a CUDA device under NCCL, the CPU under gloo."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as tdist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step: float, steps: int, seconds: float, world: int) -> float:
    """Units all ranks processed per second: every rank runs the same fixed
    work per step (weak scaling, replicas), timed by the slowest rank."""
    return world * units_per_rank_step * steps / seconds


def workload_desc(w):
    if w.n_seg > 1:
        return (f"{w.name}: {w.n_seg} databases, {w.n:,} rows x {w.f} features in all, "
                f"{w.q:,} queries, k in {sorted(set(w.k))} per database, phase orders 1-128 "
                f"int16 pass IDs")
    return (f"{w.name}: database {w.n:,} x {w.f} features, {w.q:,} queries, "
            f"k={w.k[0]}, phase orders 1-128 int16 pass IDs")


def segment_arrays(w):
    """Per-query segment, its row range and k (one segment when unsegmented)."""
    if w.n_seg == 1:
        return (np.zeros(w.q, np.int64), np.array([0, w.n], np.int64),
                np.array([0, w.q], np.int64), np.array(w.k[:1], np.int64))
    seg_of_q = np.repeat(np.arange(w.n_seg), np.diff(w.q_seg_off))
    return seg_of_q, w.seg_off.astype(np.int64), w.q_seg_off.astype(np.int64), np.array(w.k)


def pair_count(w):
    _, so, qo, _ = segment_arrays(w)
    return int(np.sum(np.diff(so) * np.diff(qo)))


def oracle_sample(w, nq_sample, seed=0, metric="cosine"):
    """Time the CPU oracle (as it stands) on a sample of the queries, each
    against its whole database. Returns the picked queries, the oracle's
    (idx, dist, seqs, lens) per picked query, the seconds and the pairs."""
    import oracle
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(w.q, size=min(nq_sample, w.q), replace=False))
    seg_of_q, so, qo, ks = segment_arrays(w)
    out = {}
    pairs = 0
    t0 = time.perf_counter()
    for s in np.unique(seg_of_q[pick]):
        qs = pick[seg_of_q[pick] == s]
        lo, hi = int(so[s]), int(so[s + 1])
        off = w.seq_off[lo:hi + 1] - w.seq_off[lo]
        ids = w.seq_ids[w.seq_off[lo]:w.seq_off[hi]]
        if metric == "cosine":
            res = oracle.recommend(w.x[lo:hi], w.queries[qs], int(ks[s]), off, ids, 128)
        else:
            i_o, d_o = oracle.knn_metric(w.x[lo:hi], w.queries[qs], int(ks[s]), metric)
            res = (i_o, d_o) + oracle.gather(i_o, off, ids, 128)
        for j, q in enumerate(qs):
            out[int(q)] = tuple(r[j] for r in res)
        pairs += len(qs) * (hi - lo)
    dt = time.perf_counter() - t0
    return pick, out, dt, pairs


# The CPU oracle's cost per (query, database element), measured on the GPU
# box's 16 host cores (1.46 s per query on 16,777,216 x 256; 53 queries/s on
# 1,048,576 x 128): used only to size the bounded CPU samples so that a
# default run stays within minutes.
ORACLE_S_PER_ELEMENT = 1.0 / 2.9e9


def oracle_sample_size(w, seconds: float, lo: int, hi: int) -> int:
    """Queries whose oracle answers take about `seconds` on the host cores."""
    _, so, qo, _ = segment_arrays(w)
    per_query = float(np.sum(np.diff(so) * np.diff(qo))) / max(1, w.q) * w.f * ORACLE_S_PER_ELEMENT
    return int(min(hi, w.q, max(lo, round(seconds / max(per_query, 1e-9)))))


# The oracle passes once over the rows it is given per call, whatever the
# number of queries (norms and binary64 copies per 65,536-row chunk): about
# 7.6 ns per row element on the machine's host cores (32.5 s for 16,777,216 x 256).
ORACLE_PASS_S_PER_ELEMENT = 7.6e-9


def oracle_window_sample(w, nq, rows, step, metric="cosine"):
    """Time the oracle on `nq` queries against a window of `rows` consecutive
    rows of a one-database workload (the window moves with `step`); returns
    the seconds and the (query, row) pairs."""
    import oracle
    rng = np.random.default_rng(step)
    pick = np.sort(rng.choice(w.q, size=min(nq, w.q), replace=False))
    lo = (step * rows) % max(1, w.n - rows + 1)
    hi = lo + rows
    off = w.seq_off[lo:hi + 1] - w.seq_off[lo]
    ids = w.seq_ids[w.seq_off[lo]:w.seq_off[hi]]
    t0 = time.perf_counter()
    if metric == "cosine":
        oracle.recommend(w.x[lo:hi], w.queries[pick], w.k[0], off, ids, 128)
    else:
        oracle.knn_metric(w.x[lo:hi], w.queries[pick], w.k[0], metric)
    return time.perf_counter() - t0, len(pick) * rows


def run_reference(args):
    world, rank, _ = setup_dist()
    if rank != 0:
        return 0
    w = fsgen.make(args.workload, workers=min(16, _NCPU), n=args.n, q=args.q, n_db=args.n_db)
    # each step a bounded sample of about 4 s of oracle work: some queries
    # against their whole databases, or, where one pass over a database takes
    # longer (the oracle's cost per call is a pass over its rows), against a
    # window of its rows that moves from step to step
    budget = 4.0
    nq = args.ref_sample if args.ref_sample else oracle_sample_size(w, budget, 1, 32)
    window = None
    if w.n_seg == 1 and w.n * w.f * ORACLE_PASS_S_PER_ELEMENT > budget:
        window = int(min(w.n, max(65536, budget / (w.f * ORACLE_PASS_S_PER_ELEMENT) // 65536 * 65536)))
        nq = args.ref_sample if args.ref_sample else 8
    times, pairs = [], 0
    for s in range(args.warmup + args.steps):
        if window:
            dt, pr = oracle_window_sample(w, nq, window, s, metric=args.metric)
        else:
            _, _, dt, pr = oracle_sample(w, nq, seed=s, metric=args.metric)
        if s >= args.warmup:
            times.append(dt)
            pairs += pr
    nq = min(nq, w.q)
    sec = float(np.sum(times))
    value = pairs / sec
    sample = (f"{nq} of {w.q:,} queries per step against a window of {window:,} of the "
              f"{w.n:,} rows (moving each step)" if window else
              f"{nq} of {w.q:,} queries per step, each against its whole database")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_desc(w), "sample": sample},
        "queries_per_s": pairs / w.n / sec if window is None and w.n_seg == 1 else None,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": _NCPU, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_serving(args, fs, torch, dev, world, rank, local):
    """Serving workload: a device-resident database, requests of 1-1,024
    queries arriving as a Poisson process, continuous batching with
    memory-based admission (paper_1810_10496_gb300.serve)."""
    import torch.distributed as tdist
    from paper_1810_10496_gb300 import serve

    w = fsgen.make("serving", workers=min(16, _NCPU), n=args.n, q=1)
    pool = fsgen.query_rows(w.seed + 1, 65536, w.f, workers=min(16, _NCPU))
    k, slots, max_batch, l_max = w.k[0], args.slots, 1024, 128
    x_d = torch.from_numpy(w.x).to(dev)
    off_d = torch.from_numpy(w.seq_off).to(dev)
    ids_d = torch.from_numpy(w.seq_ids).to(dev)

    def serve_at(prec, rate, duration):
        db = fs.fs_build_db(x_d, off_d, ids_d, prec=prec)
        per_batch = (max_batch * w.f * 4 + max_batch * k * (12 + 2 * l_max)
                     + fs.fs_workspace_size(db, max_batch) + 6 * 256)
        arena = slots * per_batch
        eng = serve.GpuEngine(fs, db, w.f, k, slots, max_batch, arena, l_max, dev)
        # a batch of one query tile, timed: the longest a small batch waits
        # for more queries while another batch is in flight
        q_tile = torch.from_numpy(pool[:128]).to(dev)
        fs.fs_recommend(db, q_tile, k)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fs.fs_recommend(db, q_tile, k)
        e1.record()
        torch.cuda.synchronize()
        tile_ms = e0.elapsed_time(e1)
        max_wait = tile_ms / 1e3 if args.max_wait_ms is None else args.max_wait_ms / 1e3
        srv = serve.Server(eng, arena_bytes=arena, slots=slots, max_batch=max_batch,
                           min_batch=args.min_batch, max_wait_s=max_wait,
                           max_queued=args.max_queued if args.max_queued > 0 else None)
        # warm-up: a few batches of every size class
        serve.run_open_loop(srv, serve.poisson_requests(pool, rate, min(0.05, duration), 1, 1024, 99))
        srv.stats = serve.ServerStats()
        reqs = serve.poisson_requests(pool, rate, duration, 1, 1024, seed=7)
        # one full batch timed with the stage events: the scan's roofline
        fs.fs_profile_read(reset=True)
        fs.fs_profile_enable(True)
        qd = torch.from_numpy(pool[:max_batch]).to(dev)
        fs.fs_recommend(db, qd, k)
        torch.cuda.synchronize()
        fs.fs_profile_enable(False)
        prof = fs.fs_profile_read(reset=True)
        sampler = ClockSampler(local)
        sampler.__enter__()
        wall = serve.run_open_loop(srv, reqs)
        sampler.__exit__(None, None, None)
        nq_offered = sum(r.queries.shape[0] for r in reqs)
        nq = nq_offered - srv.stats.shed_queries
        gpu_ms_1024 = sum(prof["ms"][s_] / max(1, prof["calls"][s_]) for s_ in prof["ms"])
        res = {"wall_s": wall, "queries": nq, "offered_queries": nq_offered,
               "requests": len(reqs), "batches": srv.stats.batches,
               "shed_requests": srv.stats.shed_requests, "shed_queries": srv.stats.shed_queries,
               "max_queued": args.max_queued,
               "host_launch_ms_per_batch": srv.stats.launch_s * 1e3 / max(1, srv.stats.batches),
               "host_retire_ms_per_batch": srv.stats.retire_s * 1e3 / max(1, srv.stats.batches),
               "gpu_ms_per_1024_batch": gpu_ms_1024,
               "mean_batch": float(np.mean(srv.stats.batch_sizes)),
               "max_inflight": srv.stats.max_inflight,
               "admissions_blocked_by_memory": srv.stats.admissions_blocked_by_memory,
               "arena_bytes": arena, "max_arena_used": srv.stats.max_arena_used,
               "offered_qps": rate, "served_qps": nq / wall,
               "clocks": sampler.summary(), "scan_ms_1024": prof["ms"]["scan"],
               "tile_batch_ms": tile_ms, "min_batch": args.min_batch,
               "max_wait_ms": max_wait * 1e3, "held_for_fill": srv.stats.held_for_fill,
               # kernels per fs_recommend call (from the profiled call) x batches served
               "gpu_launches": int(round(prof["launches"] / max(1, prof["calls"]["prepare"])
                                         * srv.stats.batches))}
        res.update(serve.latency_summary(reqs))
        # sample of answers for the oracle check (answered requests)
        done = [r for r in reqs if r.done is not None]
        res["_sample"] = done[::max(1, len(done) // 16)][:16]
        db.close()
        del eng, srv
        return res

    sweep = None
    if args.sweep:
        # offered rates from light load to far past capacity: served rate,
        # latency and shed load at each (the headline line is --rate's)
        sweep = []
        for rate in [float(v) for v in args.sweep.split(",")]:
            rr = serve_at(args.precision, rate, args.duration)
            sweep.append({k_: v for k_, v in rr.items()
                          if not k_.startswith("_") and k_ != "clocks"} | {"clocks": rr["clocks"]})
            log(f"[serving] offered {rate:,.0f} q/s: served {rr['served_qps']:,.0f} q/s, "
                f"p50 {rr['p50_ms']} ms, p99 {rr['p99_ms']} ms, shed {rr['shed_queries']:,} queries")
    r16 = serve_at(args.precision, args.rate, args.duration)
    r32 = None
    if not args.no_fp32_compare:
        r32 = serve_at("fp32", args.fp32_rate, args.duration)
    N = w.n
    # every rank serves the same request stream against its own replica
    wall = max_over_ranks(r16["wall_s"], dev, world)
    qps = whole_job_rate(r16["queries"], 1, wall, world)
    value = qps * N
    flops = 2.0 * 1024 * N * w.f
    peaks, peak_src = load_peaks()
    roof = {"bound": "tensor", "achieved": flops / (r16["scan_ms_1024"] / 1e3) / 1e12,
            "peak": peaks["bf16_tflops"], "unit": "TFLOP/s", "traffic": None,
            "kernel": f"scan ({args.precision}), one 1,024-query batch",
            "peak_source": f"{peak_src} bf16 burst", "kernel_ms": r16["scan_ms_1024"]}
    roof["frac"] = roof["achieved"] / roof["peak"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": r16["batches"], "warmup": 3, "ms_per_step": r16["wall_s"] * 1e3 / r16["batches"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "bf16": "bf16", "fp8": "fp8_e4m3"}[args.precision] + "+f64 rescoring",
        "data": "synthetic",
        "config": {"workload": f"serving: database {N:,} x {w.f} features resident, Poisson "
                               f"arrivals of requests of 1-1,024 queries, k={k}",
                   "offered_queries_per_s": args.rate, "duration_s": args.duration,
                   "slots": slots, "precision": args.precision,
                   "l2": "inputs larger than L2 (database scanned per batch)"},
        "queries_per_s": qps, "p50_ms": r16["p50_ms"], "p99_ms": r16["p99_ms"],
        "clocks": r16["clocks"],
        "e2e": {"value": value, "unit": UNIT,
                "h2d_bytes_per_step": int(r16["queries"] * w.f * 4 / r16["batches"]),
                "d2h_bytes_per_step": int(r16["queries"] * k * (12 + 2 * 128) / r16["batches"]),
                "note": "the serving loop is end to end: host queries in, host results out"},
        "gpu_launches": r16["gpu_launches"], "roofline": roof,
        "serving": {kk: v for kk, v in r16.items() if not kk.startswith("_")},
        "sweep": sweep,
        "vs_fp32_scan": None if r32 is None else {
            "fp32_offered_qps": args.fp32_rate, "fp32_served_qps": r32["served_qps"],
            "fp32_p50_ms": r32["p50_ms"], "fp32_p99_ms": r32["p99_ms"],
            "fp32_mean_batch": r32["mean_batch"], "fp32_tile_batch_ms": r32["tile_batch_ms"],
            "served_qps_ratio": r16["served_qps"] / r32["served_qps"]},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        exact = True
        t0 = time.perf_counter()
        nq = 0
        for r in r16["_sample"][:4]:
            i_o, d_o, s_o, l_o = oracle.recommend(w.x, r.queries[:4], k, w.seq_off, w.seq_ids, 128)
            exact &= bool(np.array_equal(r.idx[:4], i_o) and np.array_equal(r.seqs[:4], s_o))
            nq += min(4, r.queries.shape[0])
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": nq * N / dt, "unit": UNIT, "cores": _NCPU,
                                "kind": "oracle", "sample": f"{nq} served queries against all {N:,} rows",
                                "seconds": dt, "sample_exact": exact}
        line["recall"] = 1.0 if exact else None
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        tdist.destroy_process_group()
    return 0


def run_ours(args):
    import torch
    import torch.distributed as tdist

    import paper_1810_10496_gb300 as fs
    from paper_1810_10496_gb300 import build as libbuild
    from paper_1810_10496_gb300 import tune as fstune

    world, rank, local = setup_dist()
    if world > 1:
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        libbuild.build()
    if world > 1:
        tdist.barrier()
    fs.lib()
    if args.workload == "serving":
        return run_serving(args, fs, torch, dev, world, rank, local)

    t0 = time.perf_counter()
    w = fsgen.make(args.workload, workers=min(16, _NCPU), n=args.n, q=args.q, n_db=args.n_db)
    log(f"[rank {rank}] workload generated in {time.perf_counter() - t0:.1f} s")
    ks = np.array(w.k, dtype=np.int32)
    k_max = int(ks.max())
    seg_off = w.seg_off if w.n_seg > 1 else None
    q_seg_off = w.q_seg_off if w.n_seg > 1 else None
    Q, N, F = w.q, w.n, w.f
    l_max = 128
    pairs = pair_count(w)
    use_graph = args.graph if args.graph is not None else (w.n_seg > 1)

    x_d = torch.from_numpy(w.x).to(dev)
    off_d = torch.from_numpy(w.seq_off).to(dev)
    ids_d = torch.from_numpy(w.seq_ids).to(dev)
    q_host = torch.from_numpy(w.queries).pin_memory()
    q_d = q_host.to(dev)

    tuned = {}
    # autotuning pays on many uneven databases; on one database the default
    # plan is within noise of the best, and it is the plan the committed
    # profiles were taken on
    tune_plan = args.tune if args.tune is not None else (w.n_seg > 1)

    def make_db(prec):
        db = fs.fs_build_db(x_d, off_d, ids_d, seg_off=seg_off, prec=prec)
        if args.metric != "cosine":
            fs.fs_db_set_metric(db, args.metric)
        if args.tuning:
            fs.fs_db_set_tuning(db, json.loads(args.tuning))
            tuned[prec] = {"tuning": fs.fs_db_get_tuning(db), "fixed": True}
        elif tune_plan:
            # the plan parameters for this batch shape, timed before the timed region
            res = fstune.autotune(db, q_d, ks, q_seg_off=q_seg_off, reps=3, cache_path=None)
            tuned[prec] = {"tuning": res["tuning"], "ms": res["ms"],
                           "default_ms": res["default_ms"], "candidates": len(res["tried"])}
        ws = torch.empty(fs.fs_workspace_size(db, Q, q_seg_off), dtype=torch.uint8, device=dev)
        return db, ws

    outs = dict(idx=torch.empty((Q, k_max), dtype=torch.int32, device=dev),
                dist=torch.empty((Q, k_max), dtype=torch.float32, device=dev),
                seq_out=torch.empty((Q, k_max, l_max), dtype=torch.int16, device=dev),
                seq_len=torch.empty((Q, k_max), dtype=torch.int32, device=dev))

    def step(db, ws, q):
        fs.fs_recommend(db, q, ks, q_seg_off=q_seg_off, workspace=ws, l_max=l_max, **outs)

    def timed(db, ws, steps, warmup, sample_clocks=False, graph=False):
        """Time `steps` steps (events around each); per-stage times and launch
        counts come from eager steps with the library's stage timing on."""
        stream = torch.cuda.current_stream()
        for i in range(warmup):
            step(db, ws, q_d)
            if i == 0:
                # a scan whose error bound is wider than the gaps near the top
                # (FP8 on these vectors) leaves most queries to the exact
                # fallback, a full rescan each: stop instead of timing that
                torch.cuda.synchronize()
                s0 = fs.fs_db_stats(db)
                if s0["queries"] and s0["fallback"] > 0.5 * s0["queries"] and pairs > 1e10:
                    raise SystemExit(
                        f"{db.prec} certifies {s0['certified']} of {s0['queries']} queries of this "
                        f"workload; the others need the exact fallback scan of their whole "
                        f"database, so a timed run would take hours (use --precision bf16)")
        torch.cuda.synchronize()
        g = None
        if graph:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                step(db, ws, q_d)
            g.replay()
            torch.cuda.synchronize()
        # eager, profiled steps: stage times and kernel launches per step
        fs.fs_profile_read(reset=True)
        fs.fs_profile_enable(True)
        for _ in range(max(3, min(steps, 10))):
            step(db, ws, q_d)
        torch.cuda.synchronize()
        fs.fs_profile_enable(False)
        prof = fs.fs_profile_read(reset=True)
        launches_per_step = prof["launches"] / max(1, prof["calls"]["prepare"])
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        if world > 1:
            tdist.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(local) if sample_clocks else None
        if sampler:
            sampler.__enter__()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for a, b in evs:
            a.record(stream)
            if g is not None:
                g.replay()
            else:
                step(db, ws, q_d)
            b.record(stream)
        g1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            tdist.barrier()
        if sampler:
            sampler.__exit__(None, None, None)
        per = [a.elapsed_time(b) for a, b in evs]
        total = g0.elapsed_time(g1)
        return total, per, prof, launches_per_step, (sampler.summary() if sampler else None)

    prec = args.precision
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    db, ws = make_db(prec)
    torch.cuda.synchronize()    # the build's kernels are done
    build_s = time.perf_counter() - t0
    fs.fs_db_stats(db, reset=True)
    total_ms, per, prof, lps, clocks = timed(db, ws, args.steps, args.warmup,
                                             sample_clocks=True, graph=use_graph)
    st = fs.fs_db_stats(db)
    fs.fs_db_check(db)
    total_ms = max_over_ranks(total_ms, dev, world)
    ms_step = total_ms / args.steps
    value = whole_job_rate(pairs, args.steps, total_ms / 1e3, world)

    # dominant kernel: the scan (one launch per step)
    scan_ms = prof["ms"]["scan"] / max(1, prof["calls"]["scan"])
    flops = 2.0 * pairs * F
    peaks, peak_src = load_peaks()
    if prec == "fp32" and args.metric == "manhattan":
        # |a - b| then an add: two FP32 instructions per element, so half the
        # FMA rate; work counted as 2 flop per element like the dot products
        roof = {"bound": "alu", "achieved": flops / (scan_ms / 1e3) / 1e12,
                "peak": FP32_SIMT_PEAK_TFLOPS / 2, "unit": "TFLOP/s",
                "peak_source": "derived: 152 SM x 128 FP32 lanes x 2.07 GHz x 1 element per "
                               "2 instructions (2 flop per element)"}
    elif prec == "fp32":
        roof = {"bound": "alu", "achieved": flops / (scan_ms / 1e3) / 1e12,
                "peak": FP32_SIMT_PEAK_TFLOPS, "unit": "TFLOP/s",
                "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 flop x 2.07 GHz"}
    elif w.n_seg > 1:
        # many small databases with at most 256 queries each: about Q_s flop
        # per code byte, below the ridge point, so HBM bounds the scan. Its
        # algorithmic bytes: one pass over every row's codes (and FP8 row
        # scales) plus the query codes.
        b = 2 if prec == "bf16" else 1
        fl = -(-F // (64 if prec == "bf16" else 128)) * (64 if prec == "bf16" else 128)
        scan_bytes = N * fl * b + Q * fl * b + (N * 4 if prec == "fp8" else 0)
        roof = {"bound": "hbm", "achieved": scan_bytes / (scan_ms / 1e3) / 1e9,
                "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "peak_source": f"{peak_src} HBM copy",
                "algorithmic_bytes": scan_bytes,
                "tensor_tflops": flops / (scan_ms / 1e3) / 1e12}
    else:
        pk = peaks["bf16_tflops"] * (2.0 if prec == "fp8" else 1.0)
        roof = {"bound": "tensor", "achieved": flops / (scan_ms / 1e3) / 1e12, "peak": pk,
                "unit": "TFLOP/s",
                "peak_source": f"{peak_src} bf16 burst" + (" x 2 (fp8 nominal ratio)" if prec == "fp8" else "")}
    roof["frac"] = roof["achieved"] / roof["peak"]
    # the captured figure holds for the captured configuration only
    full_size = args.n is None and args.q is None and args.n_db is None
    roof["traffic"] = captured_traffic(f"scan_{prec}", args.workload, prec, args.metric,
                                       tuned[prec]["tuning"] if tuned else None, full_size)
    if prec != "fp32" and w.n_seg == 1:
        roof["frac_of_sustained"] = roof["achieved"] / (peaks["bf16_tflops_sustained"] *
                                                        (2.0 if prec == "fp8" else 1.0))
    roof["kernel"] = f"scan ({prec})"
    roof["kernel_ms"] = scan_ms
    roof["stage_ms_per_step"] = {s: prof["ms"][s] / max(1, prof["calls"][s]) for s in prof["ms"]}

    # end to end through the public API from host buffers
    idx_h = torch.empty((Q, k_max), dtype=torch.int32).pin_memory()
    dist_h = torch.empty((Q, k_max), dtype=torch.float32).pin_memory()
    seq_h = torch.empty((Q, k_max, l_max), dtype=torch.int16).pin_memory()
    len_h = torch.empty((Q, k_max), dtype=torch.int32).pin_memory()
    q_stage = torch.empty_like(q_d)

    def e2e_step():
        q_stage.copy_(q_host, non_blocking=True)
        fs.fs_recommend(db, q_stage, ks, q_seg_off=q_seg_off, workspace=ws, l_max=l_max, **outs)
        idx_h.copy_(outs["idx"], non_blocking=True)
        dist_h.copy_(outs["dist"], non_blocking=True)
        seq_h.copy_(outs["seq_out"], non_blocking=True)
        len_h.copy_(outs["seq_len"], non_blocking=True)

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        tdist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev, world)
    e2e = {"value": whole_job_rate(pairs, args.steps, e2e_s, world), "unit": UNIT,
           "h2d_bytes_per_step": Q * F * 4,
           "d2h_bytes_per_step": Q * k_max * (4 + 4 + 4 + 2 * l_max),
           "ms_per_step": e2e_s * 1e3 / args.steps}

    # the plain FP32 scan on the same workload, for the "vs plain FP32" ratio
    vs_fp32 = None
    if prec != "fp32" and not args.no_fp32_compare:
        db32, ws32 = make_db("fp32")
        # the FP32 scan is tens of times slower: a few steps, about 30 s at most
        slow = pairs * F > 1e14
        n32 = 3 if slow else max(3, args.steps // 4)
        t32, per32, _, _, _ = timed(db32, ws32, n32, 1 if slow else 2, graph=use_graph)
        v32 = pairs * n32 / (t32 / 1e3)
        vs_fp32 = {"fp32_pairs_per_s": v32, "fp32_ms_per_step": t32 / n32,
                   "speedup": (pairs * args.steps / (total_ms / 1e3)) / v32}
        db32.close()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "bf16": "bf16", "fp8": "fp8_e4m3"}[prec] + "+f64 rescoring",
        "data": "synthetic",
        "config": {"workload": workload_desc(w), "precision": prec, "metric": args.metric,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "cuda_graph": bool(use_graph),
                   "plan_tuning": tuned if tuned else "default plan",
                   "l2": f"inputs larger than L2 (database {N * F * (4 if prec == 'fp32' else 2 if prec == 'bf16' else 1) / 1e6:.0f} MB scanned per step)"},
        "queries_per_s": world * Q * args.steps / (total_ms / 1e3),
        "p50_ms": float(np.percentile(per, 50)), "p99_ms": float(np.percentile(per, 99)),
        "clocks": clocks, "e2e": e2e, "gpu_launches": int(round(lps * args.steps)),
        "roofline": roof, "vs_fp32_scan": vs_fp32,
        "stats": st, "db_build_s": build_s,
    }

    # CPU oracle on a bounded sample (rank 0, one GPU only), and recall of
    # the GPU answers on that sample
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # a bounded sample: about 15 s of oracle work on the host cores
        ncpu = args.cpu_sample if args.cpu_sample else oracle_sample_size(w, 15.0, 8, 1024)
        pick, ores, dt, spairs = oracle_sample(w, ncpu, metric=args.metric)
        step(db, ws, q_d)
        torch.cuda.synchronize()
        ig = outs["idx"].cpu().numpy()
        dg = outs["dist"].cpu().numpy().astype(np.float64)
        sg = outs["seq_out"].cpu().numpy()
        seg_of_q, _, _, kk = segment_arrays(w)
        hits, exact = [], True
        err_abs, err_rel = 0.0, 0.0
        for q in pick:
            kq = int(kk[seg_of_q[q]])
            i_o, d_o, s_o, l_o = ores[int(q)]
            hits.append(len(set(ig[q, :kq]) & set(i_o[:kq])) / kq)
            exact &= bool(np.array_equal(ig[q, :kq], i_o[:kq]) and np.array_equal(sg[q, :kq], s_o[:kq]))
            # distance error where the places hold the same rows
            same = (ig[q, :kq] == i_o[:kq]) & (i_o[:kq] >= 0)
            if same.any():
                e = np.abs(dg[q, :kq][same] - np.asarray(d_o[:kq], dtype=np.float64)[same])
                err_abs = max(err_abs, float(e.max()))
                den = np.abs(np.asarray(d_o[:kq], dtype=np.float64)[same])
                nz = den > 0
                if nz.any():
                    err_rel = max(err_rel, float((e[nz] / den[nz]).max()))
        line["cpu_baseline"] = {
            "value": spairs / dt, "unit": UNIT, "cores": _NCPU, "kind": "oracle",
            "sample": f"{len(pick)} of {Q:,} queries, each against its whole database",
            "seconds": dt, "queries_per_s": len(pick) / dt,
            "sample_recall": float(np.mean(hits)), "sample_exact": exact,
            "max_dist_err": {"abs": err_abs, "rel": err_rel}}
        line["recall"] = float(np.mean(hits))
    db.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        tdist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="precision", choices=sorted(fsgen.CONFIGS) + ["batching"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "fp8"])
    ap.add_argument("--metric", default="cosine", choices=["cosine", "euclidean", "manhattan"],
                    help="similarity (euclidean / manhattan: standardised, FP32 path)")
    ap.add_argument("--n", type=int, default=None,
                    help="database rows instead of the workload's (bounded profiling cases)")
    ap.add_argument("--q", type=int, default=None, help="queries instead of the workload's")
    ap.add_argument("--n-db", type=int, default=None,
                    help="batching: databases instead of 512 (bounded profiling cases)")
    ap.add_argument("--cpu-sample", type=int, default=None,
                    help="queries of the CPU-oracle sample (default: about 15 s of work)")
    ap.add_argument("--rate", type=float, default=500_000,
                    help="serving: offered queries per second (Poisson)")
    ap.add_argument("--fp32-rate", type=float, default=10_000,
                    help="serving: offered rate for the plain FP32 path")
    ap.add_argument("--duration", type=float, default=2.0, help="serving: seconds of arrivals")
    ap.add_argument("--slots", type=int, default=4, help="serving: batches in flight")
    ap.add_argument("--max-queued", type=int, default=8192,
                    help="serving: queries the queue may hold; requests beyond are shed (0: no bound)")
    ap.add_argument("--sweep", default=None,
                    help="serving: comma-separated offered rates (q/s) to sweep before the headline run")
    ap.add_argument("--min-batch", type=int, default=128,
                    help="serving: queries a batch waits for while another is in flight")
    ap.add_argument("--max-wait-ms", type=float, default=None,
                    help="serving: longest such wait (default: the time of a 128-query batch)")
    ap.add_argument("--ref-sample", type=int, default=None,
                    help="--impl reference: queries per step (default: about 4 s of work)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32-compare", action="store_true")
    ap.add_argument("--tune", dest="tune", action="store_true", default=None,
                    help="autotune the scan plan before timing (default: segmented workloads)")
    ap.add_argument("--no-tune", dest="tune", action="store_false")
    ap.add_argument("--tuning", default=None,
                    help='a fixed scan plan tuning instead, e.g. \'{"list_len": 4}\'')
    ap.add_argument("--graph", dest="graph", action="store_true", default=None,
                    help="replay each step as a captured CUDA graph (default: segmented workloads)")
    ap.add_argument("--no-graph", dest="graph", action="store_false")
    args = ap.parse_args()
    if args.metric != "cosine" and args.precision != "fp32":
        ap.error("--metric euclidean / manhattan runs on the FP32 path: add --precision fp32")
    if args.warmup < 3:
        log("warning: fewer than 3 warm-up steps")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
