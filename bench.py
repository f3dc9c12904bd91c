#!/usr/bin/env python
"""Throughput of exact cosine k-NN phase-order suggestion on GB300.

One step = one pass of the whole suggestion path over a batch of queries
against a device-resident database of explored kernels (Sec. 4 of Nobre, Reis
and Cardoso): query normalisation and codes, the database scan with fused
candidate lists, certification, FP32 rerank and binary64 rescoring, and the
gather of the neighbours' phase orders. The database itself is prepared once
(fs_build_db) before timing, as a reference set is in the paper.

Default workload: 1,048,576 database rows x 128 features, 4,096 queries,
k = 3, phase orders of 1-128 pass IDs (synthetic instruction-mix vectors
standing in for the paper's MILEPOST features). ``--impl reference`` times
the CPU oracle instead, on a bounded sample of the same workload.

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
# precision); absent (reported as null) until captured. Source: the matching
# summary under profiles/.
TRAFFIC_BYTES = {
    ("scan_fp32", "fp32_scale", "fp32"): 650.46e6,   # profiles/scan_fp32_fp32_scale.md
}


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


def workload_desc(w):
    return (f"{w.name}: database {w.n:,} x {w.f} features, {w.q:,} queries, "
            f"k={w.k[0] if w.n_seg == 1 else 'per segment'}, phase orders 1-128 int16 pass IDs")


def oracle_sample(w, nq_sample, seed=0):
    """Time the CPU oracle on a sample of the queries against the whole
    database (the oracle as it stands)."""
    import oracle
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(w.q, size=min(nq_sample, w.q), replace=False))
    t0 = time.perf_counter()
    i_o, d_o, s_o, l_o = oracle.recommend(w.x, w.queries[pick], w.k[0], w.seq_off, w.seq_ids, 128)
    dt = time.perf_counter() - t0
    return pick, (i_o, d_o, s_o, l_o), dt


def run_reference(args):
    world, rank, _ = setup_dist()
    if rank != 0:
        return 0
    w = fsgen.make(args.workload, workers=min(16, _NCPU))
    times = []
    for s in range(args.warmup + args.steps):
        _, _, dt = oracle_sample(w, args.ref_sample, seed=s)
        if s >= args.warmup:
            times.append(dt)
    nq = min(args.ref_sample, w.q)
    sec = float(np.mean(times))
    value = nq * w.n / sec
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_desc(w), "sample": f"{nq} queries per step"},
        "queries_per_s": nq / sec,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": _NCPU, "kind": "oracle",
                         "sample": f"{nq} of {w.q:,} queries against all {w.n:,} rows per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as tdist

    import paper_1810_10496_gb300 as fs
    from paper_1810_10496_gb300 import build as libbuild

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

    t0 = time.perf_counter()
    w = fsgen.make(args.workload, workers=min(16, _NCPU))
    log(f"[rank {rank}] workload generated in {time.perf_counter() - t0:.1f} s")
    k = w.k[0]
    Q, N, F = w.q, w.n, w.f
    l_max = 128

    x_d = torch.from_numpy(w.x).to(dev)
    off_d = torch.from_numpy(w.seq_off).to(dev)
    ids_d = torch.from_numpy(w.seq_ids).to(dev)
    q_host = torch.from_numpy(w.queries).pin_memory()
    q_d = q_host.to(dev)

    def make_db(prec):
        db = fs.fs_build_db(x_d, off_d, ids_d, prec=prec)
        ws = torch.empty(fs.fs_workspace_size(db, Q), dtype=torch.uint8, device=dev)
        return db, ws

    outs = dict(idx=torch.empty((Q, k), dtype=torch.int32, device=dev),
                dist=torch.empty((Q, k), dtype=torch.float32, device=dev),
                seq_out=torch.empty((Q, k, l_max), dtype=torch.int16, device=dev),
                seq_len=torch.empty((Q, k), dtype=torch.int32, device=dev))

    def step(db, ws, q):
        fs.fs_recommend(db, q, k, workspace=ws, l_max=l_max, **outs)

    def timed(db, ws, steps, warmup, sample_clocks=False):
        stream = torch.cuda.current_stream()
        for _ in range(warmup):
            step(db, ws, q_d)
        torch.cuda.synchronize()
        fs.fs_profile_read(reset=True)
        fs.fs_profile_enable(True)
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
            step(db, ws, q_d)
            b.record(stream)
        g1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            tdist.barrier()
        if sampler:
            sampler.__exit__(None, None, None)
        fs.fs_profile_enable(False)
        prof = fs.fs_profile_read(reset=True)
        per = [a.elapsed_time(b) for a, b in evs]
        total = g0.elapsed_time(g1)
        return total, per, prof, (sampler.summary() if sampler else None)

    prec = args.precision
    db, ws = make_db(prec)
    fs.fs_db_stats(db, reset=True)
    total_ms, per, prof, clocks = timed(db, ws, args.steps, args.warmup, sample_clocks=True)
    st = fs.fs_db_stats(db)
    fs.fs_db_check(db)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_step = total_ms / args.steps
    pairs = Q * N
    value = world * pairs * args.steps / (total_ms / 1e3)

    # dominant kernel: the scan (one launch per step)
    scan_ms = prof["ms"]["scan"] / max(1, prof["calls"]["scan"])
    flops = 2.0 * Q * N * F
    peaks, peak_src = load_peaks()
    if prec == "fp32":
        roof = {"bound": "alu", "achieved": flops / (scan_ms / 1e3) / 1e12,
                "peak": FP32_SIMT_PEAK_TFLOPS, "unit": "TFLOP/s",
                "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 flop x 2.07 GHz"}
    else:
        pk = peaks["bf16_tflops"] * (2.0 if prec == "fp8" else 1.0)
        roof = {"bound": "tensor", "achieved": flops / (scan_ms / 1e3) / 1e12, "peak": pk,
                "unit": "TFLOP/s",
                "peak_source": f"{peak_src} bf16 burst" + (" x 2 (fp8 nominal ratio)" if prec == "fp8" else "")}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = TRAFFIC_BYTES.get((f"scan_{prec}", args.workload, prec))
    roof["kernel"] = f"scan ({prec})"
    roof["kernel_ms"] = scan_ms
    roof["stage_ms_per_step"] = {s: prof["ms"][s] / max(1, prof["calls"][s]) for s in prof["ms"]}

    # end to end through the public API from host buffers
    idx_h = torch.empty((Q, k), dtype=torch.int32).pin_memory()
    dist_h = torch.empty((Q, k), dtype=torch.float32).pin_memory()
    seq_h = torch.empty((Q, k, l_max), dtype=torch.int16).pin_memory()
    len_h = torch.empty((Q, k), dtype=torch.int32).pin_memory()
    q_stage = torch.empty_like(q_d)

    def e2e_step():
        q_stage.copy_(q_host, non_blocking=True)
        fs.fs_recommend(db, q_stage, k, workspace=ws, l_max=l_max, **outs)
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
    e2e_s = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": world * pairs * args.steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": Q * F * 4,
           "d2h_bytes_per_step": Q * k * (4 + 4 + 4 + 2 * l_max),
           "ms_per_step": e2e_s * 1e3 / args.steps}

    # the plain FP32 scan on the same workload, for the "vs plain FP32" ratio
    vs_fp32 = None
    if prec != "fp32" and not args.no_fp32_compare:
        db32, ws32 = make_db("fp32")
        t32, per32, _, _ = timed(db32, ws32, max(3, args.steps // 4), 2)
        v32 = pairs * len(per32) / (t32 / 1e3)
        vs_fp32 = {"fp32_pairs_per_s": v32, "speedup": (pairs * args.steps / (total_ms / 1e3)) / v32}
        db32.close()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "bf16": "bf16", "fp8": "fp8_e4m3"}[prec] + "+f64 rescoring",
        "data": "synthetic",
        "config": {"workload": workload_desc(w), "precision": prec,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": f"inputs larger than L2 (database {N * F * (4 if prec == 'fp32' else 2 if prec == 'bf16' else 1) / 1e6:.0f} MB scanned per step)"},
        "queries_per_s": world * Q * args.steps / (total_ms / 1e3),
        "p50_ms": float(np.percentile(per, 50)), "p99_ms": float(np.percentile(per, 99)),
        "clocks": clocks, "e2e": e2e, "gpu_launches": prof["launches"],
        "roofline": roof, "vs_fp32_scan": vs_fp32,
        "stats": st,
    }

    # CPU oracle on a bounded sample (rank 0, one GPU only), and recall of
    # the GPU answers on that sample
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pick, (i_o, d_o, s_o, l_o), dt = oracle_sample(w, args.cpu_sample)
        step(db, ws, q_d)
        torch.cuda.synchronize()
        ig = outs["idx"].cpu().numpy()[pick]
        sg = outs["seq_out"].cpu().numpy()[pick]
        hit = np.mean([len(set(ig[r]) & set(i_o[r])) / k for r in range(len(pick))])
        line["cpu_baseline"] = {
            "value": len(pick) * N / dt, "unit": UNIT, "cores": _NCPU, "kind": "oracle",
            "sample": f"{len(pick)} of {Q:,} queries against all {N:,} rows",
            "seconds": dt, "queries_per_s": len(pick) / dt,
            "sample_recall": float(hit),
            "sample_exact": bool(np.array_equal(ig, i_o) and np.array_equal(sg, s_o))}
        line["recall"] = float(hit)
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
    ap.add_argument("--workload", default="fp32_scale", choices=sorted(fsgen.CONFIGS))
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "fp8"])
    ap.add_argument("--cpu-sample", type=int, default=128)
    ap.add_argument("--ref-sample", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32-compare", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        log("warning: fewer than 3 warm-up steps")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
