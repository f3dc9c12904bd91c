"""Seeded synthetic workloads: instruction-mix feature vectors and phase orders.

This module draws random inputs only. It holds none of the similarity
arithmetic (no norms, no dot products, no selection), so both the CUDA path
and the CPU oracle can take their inputs from it without sharing any part of
the method.

What the inputs stand in for (Sec. 4.1 and Table 1 of Nobre, Reis and
Cardoso, "Improving OpenCL Performance by Specializing Compiler Phase
Selection and Ordering"): each kernel is described by a vector of
non-negative static code features that are counts or averages of counts, and
each explored kernel carries its best LLVM phase order, an ordered list of
pass names in which repeats are allowed and which may be empty. The paper's
own vectors (MILEPOST GCC, 55 features) and its benchmarks are not available,
so synthetic instruction-mix vectors of the same kind replace them:

* a row's total instruction count is ``lognormal(mean=6, sigma=1)``;
* its opcode mix is ``dirichlet([0.3] * F)``;
* its features are ``rint(total * mix)`` (round half to even), stored as
  float32 (the values are small integers, so the cast is exact);
* a phase order is a run of ``uniform[1, 128]`` pass IDs, each uniform in
  ``[0, 100)``, stored as int16 in CSR form (``off[n + 1]``, ``ids[off[n]]``).

Every stream is drawn in fixed chunks of 65,536 rows from
``numpy.random.default_rng([seed, stream, chunk])`` so that any number of
worker processes produce the same bytes. Streams: 0 = database rows,
1 = query rows, 2 = phase-order lengths, 3 = pass IDs, 4 = batch layout.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

CHUNK = 65536
N_PASSES = 100          # pass-ID vocabulary
MAX_ORDER_LEN = 128     # longest synthetic phase order

STREAM_DB, STREAM_QUERY, STREAM_LEN, STREAM_IDS, STREAM_LAYOUT = 0, 1, 2, 3, 4


def _feature_chunk(args):
    seed, stream, chunk, rows, f = args
    rng = np.random.default_rng([seed, stream, chunk])
    total = rng.lognormal(mean=6.0, sigma=1.0, size=rows)
    mix = rng.dirichlet(np.full(f, 0.3), size=rows)
    return np.rint(total[:, None] * mix).astype(np.float32)


def _chunk_tasks(seed, stream, n, f):
    tasks = []
    for c in range((n + CHUNK - 1) // CHUNK):
        rows = min(CHUNK, n - c * CHUNK)
        tasks.append((seed, stream, c, rows, f))
    return tasks


def feature_rows(seed: int, stream: int, n: int, f: int, workers: int = 1,
                 out: np.ndarray | None = None) -> np.ndarray:
    """Instruction-mix rows ``[n, f]`` float32 for one stream.

    Row ``r`` depends only on ``(seed, stream, r // CHUNK)``; ``workers > 1``
    spreads chunks over a spawn-started process pool (safe after CUDA use).
    """
    if out is None:
        out = np.empty((n, f), dtype=np.float32)
    tasks = _chunk_tasks(seed, stream, n, f)
    if workers > 1 and len(tasks) > 1:
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        with ctx.Pool(min(workers, len(tasks))) as pool:
            for (s, st, c, rows, ff), block in zip(
                    tasks, pool.imap(_feature_chunk, tasks, chunksize=1)):
                out[c * CHUNK:c * CHUNK + rows] = block
    else:
        for t in tasks:
            c, rows = t[2], t[3]
            out[c * CHUNK:c * CHUNK + rows] = _feature_chunk(t)
    return out


def db_rows(seed: int, n: int, f: int, workers: int = 1) -> np.ndarray:
    return feature_rows(seed, STREAM_DB, n, f, workers)


def query_rows(seed: int, q: int, f: int, workers: int = 1) -> np.ndarray:
    return feature_rows(seed, STREAM_QUERY, q, f, workers)


def phase_orders(seed: int, n: int, min_len: int = 1,
                 max_len: int = MAX_ORDER_LEN) -> tuple[np.ndarray, np.ndarray]:
    """CSR phase orders for ``n`` database rows: ``(off int64[n+1], ids int16)``.

    Lengths are uniform in ``[min_len, max_len]`` (``min_len = 0`` admits
    empty orders, which Table 1 has for three benchmarks); IDs are uniform in
    ``[0, N_PASSES)``.
    """
    lens = np.empty(n, dtype=np.int64)
    for c in range((n + CHUNK - 1) // CHUNK):
        rows = min(CHUNK, n - c * CHUNK)
        rng = np.random.default_rng([seed, STREAM_LEN, c])
        lens[c * CHUNK:c * CHUNK + rows] = rng.integers(min_len, max_len + 1, size=rows)
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    ids = np.empty(int(off[-1]), dtype=np.int16)
    for c in range((n + CHUNK - 1) // CHUNK):
        lo, hi = off[c * CHUNK], off[min(n, (c + 1) * CHUNK)]
        rng = np.random.default_rng([seed, STREAM_IDS, c])
        ids[lo:hi] = rng.integers(0, N_PASSES, size=int(hi - lo)).astype(np.int16)
    return off, ids


@dataclass
class Workload:
    """One synthetic problem: databases, queries, phase orders and k."""
    name: str
    seed: int
    n: int                      # total database rows over all segments
    f: int
    q: int                      # total queries over all segments
    k: list[int]                # k per segment
    seg_off: np.ndarray | None = None    # int64[n_seg + 1] database row offsets
    q_seg_off: np.ndarray | None = None  # int32[n_seg + 1] query offsets
    x: np.ndarray | None = field(default=None, repr=False)
    queries: np.ndarray | None = field(default=None, repr=False)
    seq_off: np.ndarray | None = field(default=None, repr=False)
    seq_ids: np.ndarray | None = field(default=None, repr=False)

    @property
    def n_seg(self) -> int:
        return 1 if self.seg_off is None else len(self.seg_off) - 1


# name -> (n, f, q, k); every config's phase orders are 1-128 pass IDs.
CONFIGS = {
    "tiny_k1":   (64, 64, 15, 1),
    "tiny_k3":   (64, 64, 15, 3),
    "fp32_scale": (1_048_576, 128, 4096, 3),
    "precision": (16_777_216, 256, 8192, 3),
    "serving":   (8_388_608, 128, 1024, 3),
}


def batch_layout(seed: int, n_db: int = 512, lo: int = 1000, hi: int = 200_000,
                 q_max: int = 256):
    """Sizes of ``n_db`` independent databases (log-uniform in [lo, hi]),
    their query counts (uniform in [1, q_max]) and k (uniform over {1, 3})."""
    rng = np.random.default_rng([seed, STREAM_LAYOUT, 0])
    sizes = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_db))).astype(np.int64)
    nq = rng.integers(1, q_max + 1, size=n_db).astype(np.int64)
    ks = rng.choice(np.array([1, 3]), size=n_db).astype(np.int64)
    return sizes, nq, ks


def make(name: str, seed: int = 0, workers: int = 1, n: int | None = None,
         q: int | None = None, f: int | None = None, n_db: int | None = None) -> Workload:
    """Build a named workload; ``n``/``q``/``f`` override the sizes (for
    bounded samples of a large workload and for small test cases), ``n_db``
    the number of databases of the batching workload (512)."""
    if name == "batching":
        sizes, nq, ks = batch_layout(seed, n_db=n_db or 512)
        ff = f or 128
        seg_off = np.zeros(len(sizes) + 1, dtype=np.int64)
        np.cumsum(sizes, out=seg_off[1:])
        q_seg_off = np.zeros(len(sizes) + 1, dtype=np.int32)
        np.cumsum(nq, out=q_seg_off[1:])
        w = Workload(name, seed, int(seg_off[-1]), ff, int(q_seg_off[-1]),
                     [int(v) for v in ks], seg_off, q_seg_off)
    else:
        n0, f0, q0, k0 = CONFIGS[name]
        w = Workload(name, seed, n or n0, f or f0, q or q0, [k0])
    w.x = db_rows(seed, w.n, w.f, workers)
    w.queries = query_rows(seed, w.q, w.f, workers)
    w.seq_off, w.seq_ids = phase_orders(seed, w.n)
    return w


STREAM_DSE = 5


@dataclass
class DseSuite:
    """A synthetic reference set for the evaluation procedure of Sec. 4.2:
    kernels with feature vectors, each kernel's best phase order, and the
    speedup of every kernel compiled with every kernel's best order."""
    features: np.ndarray        # [n][f] float32 counts
    seq_off: np.ndarray         # [n + 1] int64 CSR offsets of the best orders
    seq_ids: np.ndarray         # int16 pass IDs
    speedup: np.ndarray         # [n][n] float64: kernel i compiled with order j
    family: np.ndarray          # [n] int64 family label of each kernel


def dse_suite(seed: int = 0, n: int = 15, f: int = 55, families: int = 5,
              duplicate_orders: int = 2) -> DseSuite:
    """Kernels drawn in `families` families (the stand-in for the paper's 15
    PolyBench/GPU kernels and Table 1): a family has an opcode mix and a best
    phase order; a member's features are ``rint(total * mix')`` with ``mix'``
    drawn close to the family mix, and its best order is the family order
    with a few passes replaced. Speedups (over compilation without phase
    ordering, the fallback) are lognormal draws: around 1.5 for an order
    from the kernel's own family, around 1.0 otherwise (below 1 is a
    slowdown), and the kernel's own order is the best of its row.
    `duplicate_orders` kernels reuse another kernel's order exactly, as
    Table 1 repeats some orders. Drawn from family labels alone: there is no
    similarity arithmetic here."""
    rng = np.random.default_rng([seed, STREAM_DSE, 0])
    fam = rng.integers(0, families, size=n).astype(np.int64)
    fam_mix = rng.dirichlet(np.full(f, 0.3), size=families)
    fam_len = rng.integers(8, 48, size=families)
    fam_order = [rng.integers(0, N_PASSES, size=int(fam_len[c])) for c in range(families)]
    feats = np.zeros((n, f), dtype=np.float32)
    orders = []
    for i in range(n):
        c = fam[i]
        mix = rng.dirichlet(200.0 * fam_mix[c] + 1e-3)
        total = rng.lognormal(mean=6.0, sigma=0.5)
        feats[i] = np.rint(total * mix).astype(np.float32)
        o = fam_order[c].copy()
        edits = rng.integers(0, o.size, size=max(1, o.size // 8))
        o[edits] = rng.integers(0, N_PASSES, size=edits.size)
        orders.append(o.astype(np.int16))
    for d in range(min(duplicate_orders, n - 1)):
        orders[n - 1 - d] = orders[d].copy()
    same = fam[:, None] == fam[None, :]
    speed = np.where(same, rng.lognormal(np.log(1.5), 0.15, size=(n, n)),
                     rng.lognormal(0.0, 0.25, size=(n, n)))
    for i in range(n):
        speed[i, i] = speed[i].max() * rng.uniform(1.0, 1.1)
    # kernels sharing an order exactly get one speedup per (kernel, order)
    for d in range(min(duplicate_orders, n - 1)):
        speed[:, n - 1 - d] = speed[:, d]
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum([o.size for o in orders], out=off[1:])
    return DseSuite(feats, off, np.concatenate(orders).astype(np.int16), speed, fam)
