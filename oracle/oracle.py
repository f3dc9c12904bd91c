"""FP64 CPU oracle for feature-based phase-order suggestion (Sec. 4).

TEST INFRASTRUCTURE ONLY. This module is the independent checker of the CUDA
library: only the test suite, the package's smoke check and the benchmark's
CPU-baseline leg may import it. The product path never calls it, and it
imports nothing from the CUDA package (the two share no code).

What it computes, step by step, from the paper:

* Sec. 4: a new kernel is compared with every kernel of the reference set
  through their code-feature vectors, the K most similar ones are selected
  (k-nearest neighbours) and their best phase orders (Table 1) are the
  suggestions.
* Sec. 4.2: similarity is the cosine distance between the two feature
  vectors.
* Sec. 4.1: features are absolute counts or averages of counts; no feature
  selection or scaling is applied, so the vectors enter the metric as given.

The paper gives no formula, precision, tie rule or zero-vector rule, so the
oracle fixes these readings (each listed in the design notes):

1. Per query ``q`` and database row ``x`` (both length F), in IEEE binary64
   with round-to-nearest-even and no fused multiply-add:
   ``D = sum_i q_i*x_i``, ``A = sum_i q_i*q_i``, ``B = sum_i x_i*x_i``, each
   summed sequentially for i = 0..F-1; the cosine similarity is
   ``s = D / sqrt(A*B)`` and the cosine distance is ``d = 1 - s``.
2. If ``A == 0`` or ``B == 0`` the cosine is undefined; the oracle sets
   ``s = 0`` (so ``d = 1``).
3. Neighbours are ranked by ``s`` descending; equal ``s`` go to the lower
   database index. Ranking by ``s`` rather than by ``d`` keeps distinct
   scores distinct where ``1 - s`` would round them together.
4. If ``k`` exceeds the number of rows, missing slots get index -1,
   distance +inf and an empty phase order.
5. A phase order is returned exactly as stored, in rank order, duplicates
   included.

When every feature is an integer and ``F * max|q| * max|x|`` stays below
2**53, every partial sum of D, A and B is an exactly representable integer,
so any summation order gives the same bits; only then does the oracle use a
BLAS matrix product for D (a library primitive standing in for the
sequential loop, checked against it by the tests).

Parity pins: closed forms, brute force against the C checker in
``naive_knn.c``, an exact rational cross-check, invariants and the Table 1
fixture (see ``tests/test_oracle.py``).
"""
from __future__ import annotations

import numpy as np

__all__ = ["norm2", "dot_seq", "cosine_scores", "knn", "recommend", "gather",
           "exact_integer_inputs", "standardize_stats", "standardize", "metric_distances",
           "knn_metric", "METRICS"]


def norm2(x: np.ndarray) -> np.ndarray:
    """``sum_i x_i*x_i`` per row, sequential in i (reading 1)."""
    x = np.asarray(x, dtype=np.float64)
    acc = np.zeros(x.shape[0], dtype=np.float64)
    for i in range(x.shape[1]):
        acc = acc + x[:, i] * x[:, i]
    return acc


def dot_seq(q: np.ndarray, x: np.ndarray) -> np.ndarray:
    """``D[a, b] = sum_i q[a, i]*x[b, i]``, sequential in i, each product
    rounded before it is added (reading 1)."""
    q = np.asarray(q, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    acc = np.zeros((q.shape[0], x.shape[0]), dtype=np.float64)
    for i in range(q.shape[1]):
        acc = acc + q[:, i:i + 1] * x[None, :, i]
    return acc


def exact_integer_inputs(q: np.ndarray, x: np.ndarray) -> bool:
    """True when D, A and B are exact in binary64 in any summation order."""
    if q.size == 0 or x.size == 0:
        return True
    q64 = np.asarray(q, dtype=np.float64)
    x64 = np.asarray(x, dtype=np.float64)
    if not (np.all(q64 == np.rint(q64)) and np.all(x64 == np.rint(x64))):
        return False
    f = q64.shape[1]
    mq, mx = float(np.abs(q64).max()), float(np.abs(x64).max())
    return f * max(mq, mx) ** 2 < 2.0 ** 53


def cosine_scores(q: np.ndarray, x: np.ndarray, a: np.ndarray | None = None,
                  b: np.ndarray | None = None, use_blas: bool | None = None) -> np.ndarray:
    """Cosine similarity ``s[a, b]`` of query rows against database rows.

    ``s = D / sqrt(A*B)`` in binary64 (Sec. 4.2, reading 1); ``s = 0`` where a
    vector is all zeros (reading 2). ``use_blas=None`` takes the BLAS product
    only when :func:`exact_integer_inputs` proves it equal to the loop.
    """
    q = np.asarray(q, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    if a is None:
        a = norm2(q)
    if b is None:
        b = norm2(x)
    if use_blas is None:
        use_blas = exact_integer_inputs(q, x)
    d = q @ x.T if use_blas else dot_seq(q, x)
    ab = a[:, None] * b[None, :]
    root = np.sqrt(ab)
    with np.errstate(divide="ignore", invalid="ignore"):
        s = d / root
    s[(a[:, None] == 0) | (b[None, :] == 0)] = 0.0
    return s


def _topk_rows(s: np.ndarray, cols: np.ndarray, k: int, exclude=None):
    """Per row of ``s``: the k best (score desc, column asc) among ``cols``,
    leaving out column ``exclude[r]`` for row r when given."""
    nq, n = s.shape
    idx = np.full((nq, k), -1, dtype=np.int64)
    sc = np.full((nq, k), -np.inf, dtype=np.float64)
    for r in range(nq):
        row = s[r]
        ccols = cols
        if exclude is not None and exclude[r] >= 0:
            keep = cols != exclude[r]
            row, ccols = row[keep], cols[keep]
        n = len(row)
        kk = min(k, n)
        if kk == 0:
            continue
        if n > 4 * kk:
            # every row scoring at least the kk-th largest score, ties included
            t = np.partition(row, n - kk)[n - kk]
            cand = np.nonzero(row >= t)[0]
        else:
            cand = np.arange(n)
        order = np.lexsort((ccols[cand], -row[cand]))[:kk]
        idx[r, :kk] = ccols[cand[order]]
        sc[r, :kk] = row[cand[order]]
    return idx, sc


def _merge(idx_a, sc_a, idx_b, sc_b, k):
    """Merge two per-row top-k lists under (score desc, index asc)."""
    idx = np.concatenate([idx_a, idx_b], axis=1)
    sc = np.concatenate([sc_a, sc_b], axis=1)
    out_i = np.full((idx.shape[0], k), -1, dtype=np.int64)
    out_s = np.full((idx.shape[0], k), -np.inf, dtype=np.float64)
    for r in range(idx.shape[0]):
        valid = idx[r] >= 0
        ii, ss = idx[r][valid], sc[r][valid]
        order = np.lexsort((ii, -ss))[:k]
        out_i[r, :len(order)] = ii[order]
        out_s[r, :len(order)] = ss[order]
    return out_i, out_s


def knn(x: np.ndarray, queries: np.ndarray, k: int, chunk: int = 65536,
        use_blas: bool | None = None, exclude=None):
    """k nearest database rows per query under cosine distance (Sec. 4).

    ``exclude[r]`` (optional) is a row that query r may not select: the
    leave-one-out protocol of Sec. 4.2, where a kernel's own entry is not part
    of its reference set. Returns ``(idx int64[nq, k], dist float64[nq, k],
    score float64[nq, k])``; padded slots hold -1, +inf and -inf (reading 4).
    """
    q = np.asarray(queries, dtype=np.float64)
    nq, n = q.shape[0], x.shape[0]
    if k < 1:
        raise ValueError("k must be >= 1")
    a = norm2(q)
    best_i = np.full((nq, k), -1, dtype=np.int64)
    best_s = np.full((nq, k), -np.inf, dtype=np.float64)
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        # one chunk in binary64 at a time (a large database need not fit
        # twice in memory); the BLAS product is taken for a chunk only when
        # it is provably equal to the sequential loop there, so the choice
        # never changes a score
        xc = np.asarray(x[lo:hi], dtype=np.float64)
        blas = exact_integer_inputs(q, xc) if use_blas is None else use_blas
        s = cosine_scores(q, xc, a=a, b=norm2(xc), use_blas=blas)
        ci, cs = _topk_rows(s, np.arange(lo, hi, dtype=np.int64), k, exclude)
        best_i, best_s = _merge(best_i, best_s, ci, cs, k)
    dist = np.where(best_i >= 0, 1.0 - best_s, np.inf)
    return best_i, dist, best_s


def gather(idx: np.ndarray, seq_off: np.ndarray, seq_ids: np.ndarray, l_max: int):
    """Phase orders of the selected rows (Sec. 4, Table 1): a ``[nq, k, l_max]``
    int16 array padded with -1 and the true lengths ``int32[nq, k]``. Orders
    longer than ``l_max`` are cut to ``l_max`` (the length still reports the
    full order)."""
    nq, k = idx.shape
    out = np.full((nq, k, l_max), -1, dtype=np.int16)
    lens = np.zeros((nq, k), dtype=np.int32)
    for r in range(nq):
        for c in range(k):
            j = int(idx[r, c])
            if j < 0:
                continue
            lo, hi = int(seq_off[j]), int(seq_off[j + 1])
            lens[r, c] = hi - lo
            m = min(hi - lo, l_max)
            out[r, c, :m] = seq_ids[lo:lo + m]
    return out, lens


def recommend(x, queries, k, seq_off, seq_ids, l_max=128, **kw):
    """k-NN then the neighbours' phase orders: the whole Sec. 4 suggestion."""
    idx, dist, score = knn(x, queries, k, **kw)
    seqs, lens = gather(idx, seq_off, seq_ids, l_max)
    return idx, dist, seqs, lens


def knn_segments(x, queries, seg_off, q_seg_off, ks, **kw):
    """Independent databases: segment ``s`` holds rows ``seg_off[s]:seg_off[s+1]``
    and queries ``q_seg_off[s]:q_seg_off[s+1]``, searched with ``ks[s]``.
    Indices are local to each segment. Returns per-segment lists."""
    out = []
    for s in range(len(seg_off) - 1):
        xs = x[seg_off[s]:seg_off[s + 1]]
        qs = queries[q_seg_off[s]:q_seg_off[s + 1]]
        out.append(knn(xs, qs, int(ks[s]), **kw))
    return out


# ---------------------------------------------------------------------------
# Other similarity metrics (Sec. 4.2 names their evaluation as future work;
# these are the readings the library implements for it): Euclidean and
# Manhattan distance between standardised feature vectors.
#
# 6. Standardisation statistics come from the reference set (one database
#    segment), per feature f, in binary64 with the row order i = 0..n-1:
#    ``mu_f = (sum_i x_if) / n`` and the population deviation
#    ``sigma_f = sqrt((sum_i (x_if - mu_f)**2) / n)``, sums sequential, no
#    fused multiply-add. ``z_f = (v_f - mu_f) / sigma_f`` for database rows
#    and queries alike; a feature with ``sigma_f == 0`` (constant over the
#    reference set) gives ``z_f = 0``.
# 7. Euclidean: ``d = sqrt(sum_f (zq_f - zx_f)**2)``; Manhattan:
#    ``d = sum_f |zq_f - zx_f|``; each sum sequential in f, binary64, no fused
#    multiply-add. Ranking: d ascending, equal d to the lower index.

METRICS = ("cosine", "euclidean", "manhattan")


def standardize_stats(x: np.ndarray):
    """Per-feature mean and population deviation of the rows of ``x``
    (reading 6): ``(mu float64[f], sigma float64[f])``."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    if n == 0:
        return np.zeros(x.shape[1]), np.zeros(x.shape[1])
    # np.cumsum adds in order, so its last element is the sequential sum
    mu = np.cumsum(x, axis=0)[-1] / n
    d = x - mu
    var = np.cumsum(d * d, axis=0)[-1] / n
    return mu, np.sqrt(var)


def standardize(v: np.ndarray, mu: np.ndarray, sigma: np.ndarray) -> np.ndarray:
    """``z = (v - mu) / sigma``, 0 where sigma is 0 (reading 6)."""
    v = np.asarray(v, dtype=np.float64)
    safe = np.where(sigma > 0, sigma, 1.0)
    return np.where(sigma > 0, (v - mu) / safe, 0.0)


def metric_distances(q: np.ndarray, x: np.ndarray, metric: str, mu, sigma) -> np.ndarray:
    """``[nq, n]`` binary64 distances under ``metric`` (reading 7)."""
    zq = standardize(q, mu, sigma)
    zx = standardize(x, mu, sigma)
    acc = np.zeros((zq.shape[0], zx.shape[0]), dtype=np.float64)
    for f in range(zq.shape[1]):
        diff = zq[:, f][:, None] - zx[:, f][None, :]
        acc = acc + (diff * diff if metric == "euclidean" else np.abs(diff))
    return np.sqrt(acc) if metric == "euclidean" else acc


def knn_metric(x: np.ndarray, queries: np.ndarray, k: int, metric: str, exclude=None,
               chunk: int = 16384):
    """k nearest rows per query under ``metric`` (cosine goes to ``knn``):
    ``(idx int64[nq, k], dist float64[nq, k])``, padded with -1 and +inf."""
    if metric == "cosine":
        i, d, _ = knn(x, queries, k, exclude=exclude)
        return i, d
    x = np.asarray(x, dtype=np.float64)
    q = np.asarray(queries, dtype=np.float64)
    mu, sigma = standardize_stats(x)
    best_i = np.full((q.shape[0], k), -1, dtype=np.int64)
    best_s = np.full((q.shape[0], k), -np.inf, dtype=np.float64)
    for lo in range(0, x.shape[0], chunk):
        hi = min(x.shape[0], lo + chunk)
        s = -metric_distances(q, x[lo:hi], metric, mu, sigma)   # larger is nearer
        ci, cs = _topk_rows(s, np.arange(lo, hi, dtype=np.int64), k, exclude)
        best_i, best_s = _merge(best_i, best_s, ci, cs, k)
    return best_i, np.where(best_i >= 0, -best_s, np.inf)
