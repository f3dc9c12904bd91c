"""Autotuner of the scan's planning parameters, with a JSON cache.

For one database and one query-batch shape, the tuner times fs_knn under
each candidate tuning (fs_db_set_tuning: work items per block, candidate
list length, the share of L2 for the row chunks in flight), checks that
every candidate returns the same answers as the defaults, and keeps the
fastest. The selection is exact, so a tuning can only change the time; a
candidate whose answers differ is a library error and raises.

Results are cached in a JSON file keyed by a schema version, the device
name, the precision, the similarity metric, the feature count and
power-of-two buckets of the rows, queries and segments, plus the largest k,
so a later process with a batch of the same shape applies the choice without
timing again. The schema version changes whenever the meaning of a tuning
parameter changes, so entries written under an older meaning are timed
again rather than applied.
"""
from __future__ import annotations

import json
import math
import os
import tempfile

DEFAULT_CACHE = os.environ.get(
    "FS_TUNE_CACHE",
    os.path.join(os.path.expanduser("~"), ".cache", "paper_1810_10496_gb300", "tuning.json"))

ITEMS_PER_BLOCK = (1, 2, 4, 8, 16)
LIST_LEN = (4, 8, 16)
L2_SHARE_PCT = (25, 50, -1)
# bumped whenever a tuning parameter changes meaning (2: scan items are
# claimed dynamically, so items_per_block sets the item length only)
SCHEMA = 2


def candidates(prec: str, n_seg: int, k_max: int) -> list[dict]:
    """The tunings worth timing for this shape: the list length (each that
    holds k) matters only for the tensor-core scans, the L2 share only for a
    single segment. The defaults come first."""
    lists = tuple(n for n in LIST_LEN if n >= k_max) if prec != "fp32" else ()
    lists = lists or (0,)
    shares = L2_SHARE_PCT if n_seg == 1 else (0,)
    out = [{"items_per_block": 0, "list_len": 0, "l2_share_pct": 0}]
    seen = {_normal(out[0], prec, k_max)}
    for i in ITEMS_PER_BLOCK:
        for ln in lists:
            for p in shares:
                c = {"items_per_block": i, "list_len": ln, "l2_share_pct": p}
                if _normal(c, prec, k_max) not in seen:
                    seen.add(_normal(c, prec, k_max))
                    out.append(c)
    return out


def _normal(c: dict, prec: str = "bf16", k_max: int = 1) -> tuple:
    """A tuning with the defaults written out and the list length the
    library will actually keep (to drop duplicates)."""
    want = c.get("list_len") or 8
    if prec == "fp32":
        ln = 16
    elif want == 4 and k_max <= 4:
        ln = 4
    elif want <= 8 and k_max <= 8:
        ln = 8
    else:
        ln = 16
    return (c.get("items_per_block") or 4, ln, c.get("l2_share_pct") or 50)


def _bucket(v: int) -> int:
    return 0 if v <= 0 else 1 << max(0, math.ceil(math.log2(v)))


def shape_key(device: str, prec: str, f: int, n_rows: int, nq: int, n_seg: int,
              k_max: int, metric: str = "cosine") -> str:
    return (f"v{SCHEMA}|{device}|{prec}|{metric}|F{f}|N{_bucket(n_rows)}|Q{_bucket(nq)}"
            f"|S{_bucket(n_seg)}|K{k_max}")


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as fh:
            d = json.load(fh)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str = DEFAULT_CACHE):
    """Writes the whole cache atomically (temporary file, then rename)."""
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(os.path.abspath(path)), suffix=".tmp")
    with os.fdopen(fd, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def choose(measure, cands: list[dict], same, finalists: int = 3) -> dict:
    """Times every candidate with measure(c) -> (ms, answers), checks its
    answers against the first candidate's with same(a, b) and returns the
    fastest with the timings of all. The fastest `finalists` and the
    defaults are then timed once more, in reverse order, and each keeps its
    better time: a first timing taken while the clocks or caches were still
    settling does not decide the choice."""
    tried = []
    base = None
    for c in cands:
        ms, ans = measure(c)
        if base is None:
            base = ans
        elif not same(ans, base):
            raise RuntimeError(f"tuning {c} changed the answers")
        tried.append({"tuning": dict(c), "ms": float(ms)})
    again = sorted(range(len(tried)), key=lambda i: tried[i]["ms"])[:max(1, finalists)]
    if 0 not in again:
        again.append(0)
    for i in sorted(again, reverse=True):
        ms, ans = measure(cands[i])
        if not same(ans, base):
            raise RuntimeError(f"tuning {cands[i]} changed the answers")
        tried[i]["ms"] = min(tried[i]["ms"], float(ms))
    best = min(tried, key=lambda t: t["ms"])
    return {"tuning": best["tuning"], "ms": best["ms"], "default_ms": tried[0]["ms"],
            "tried": tried}


def autotune(db, q, k, q_seg_off=None, reps: int = 5, cache_path: str | None = DEFAULT_CACHE,
             force: bool = False, cands: list[dict] | None = None, warm_s: float = 0.2) -> dict:
    """Picks the fastest tuning of `db` for batches shaped like (q, k,
    q_seg_off), applies it to `db` and returns {"tuning", "ms",
    "default_ms", "tried", "key", "cached"}. With a cache entry for the
    shape (and not `force`) the cached tuning is applied without timing."""
    import numpy as np
    import torch

    import paper_1810_10496_gb300 as fs

    nq = int(q.shape[0])
    kk = np.broadcast_to(np.asarray(k, dtype=np.int32), (db.n_seg,))
    k_max = int(kk.max())
    key = shape_key(torch.cuda.get_device_name(q.device), db.prec, db.f, db.n, nq, db.n_seg,
                    k_max, db.metric)
    cache = load_cache(cache_path) if cache_path else {}
    if not force and key in cache:
        fs.fs_db_set_tuning(db, cache[key]["tuning"])
        return dict(cache[key], key=key, cached=True)

    cands = cands or candidates(db.prec, db.n_seg, k_max)
    ws_bytes = 0
    for c in cands:
        fs.fs_db_set_tuning(db, c)
        ws_bytes = max(ws_bytes, fs.fs_workspace_size(db, nq, q_seg_off))
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=q.device)
    idx = torch.empty((nq, k_max), dtype=torch.int32, device=q.device)
    dist = torch.empty((nq, k_max), dtype=torch.float32, device=q.device)
    stream = torch.cuda.current_stream(q.device)

    def measure(c):
        fs.fs_db_set_tuning(db, c)
        fs.fs_knn(db, q, kk, q_seg_off=q_seg_off, workspace=ws, idx=idx, dist=dist)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
        evs[0].record(stream)
        for i in range(reps):
            fs.fs_knn(db, q, kk, q_seg_off=q_seg_off, workspace=ws, idx=idx, dist=dist)
            evs[i + 1].record(stream)
        torch.cuda.synchronize(q.device)
        times = [evs[i].elapsed_time(evs[i + 1]) for i in range(reps)]
        return float(np.median(times)), (idx.cpu().numpy(), dist.cpu().numpy())

    def same(a, b):
        # exact selection: identical rows; distances within the stated tolerance
        if not np.array_equal(a[0], b[0]):
            return False
        fin = np.isfinite(b[1])
        if not np.array_equal(np.isfinite(a[1]), fin):
            return False
        d0, d1 = a[1][fin], b[1][fin]
        return bool(np.all(np.abs(d0 - d1) <= 1e-5 * np.abs(d1) + 1e-6))

    # the first calls after a build or an idle spell run slow (clocks still
    # rising, first touches of the workspace): run the defaults for a while
    import time
    fs.fs_db_set_tuning(db, cands[0])
    t_end = time.perf_counter() + warm_s
    n = 0
    while n < 3 or time.perf_counter() < t_end:
        fs.fs_knn(db, q, kk, q_seg_off=q_seg_off, workspace=ws, idx=idx, dist=dist)
        n += 1
        if n % 8 == 0:
            torch.cuda.synchronize(q.device)
    torch.cuda.synchronize(q.device)
    res = choose(measure, cands, same)
    fs.fs_db_set_tuning(db, res["tuning"])
    fs.fs_db_check(db)
    if cache_path:
        cache = load_cache(cache_path)
        cache[key] = {"tuning": res["tuning"], "ms": res["ms"], "default_ms": res["default_ms"]}
        save_cache(cache, cache_path)
    return dict(res, key=key, cached=False)
