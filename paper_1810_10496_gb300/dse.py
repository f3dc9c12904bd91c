"""Host side of the suggestion method: the evaluate-K loop and the K sweep.

Sec. 4: for a new kernel, the K reference kernels most similar to it are
found and their best phase orders (Table 1) are compiled and evaluated with
the new kernel; the best compiled code wins. Sec. 4.2 adds the rules this
module follows:

* a safe fallback (compilation without phase ordering, or a standard level
  such as -O3) always stays in the running, so a bad suggestion never makes
  the result worse than the fallback; the result says when the fallback won;
* each distinct order is compiled and evaluated once, however many of the K
  neighbours share it, and a fitness seen before for the same kernel is
  recalled, not measured again;
* exploration may stop early once the compiled code meets the requirement;
* the paper's experiment: for K = 1..14, leave-one-out over the reference
  set, the geometric mean speedup of the best evaluated order, against
  random selection of K kernels repeated 1,000 times.

The compile-and-run step itself (LLVM, OpenCL, the benchmarks) is the
caller's: it is passed in as a callback. The neighbour search is the CUDA
library (fs_recommend); `k_sweep` takes any function with fs_knn's answer so
the procedure can be checked on its own.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Sequence

import numpy as np


@dataclass
class Suggestion:
    """The K suggestions for one kernel, nearest first."""
    rows: list                  # reference rows (segment-local indices)
    distances: list             # cosine distances
    orders: list                # int16 arrays: the rows' best phase orders
    duplicate_of: list          # earlier slot with the same order, or -1


@dataclass
class Outcome:
    fitness: float              # best fitness seen (the fallback's if nothing beat it)
    order: np.ndarray | None    # the winning order (None: the fallback won)
    fallback: bool              # True when no suggested order beat the fallback
    compiled: int               # distinct orders compiled and evaluated
    recalled: int               # evaluations answered from the memo
    stopped_early: bool = False
    trace: list = field(default_factory=list)   # (slot, fitness or None for skipped)


def suggest(db, queries, k: int, exclude=None, l_max: int = 128) -> list[Suggestion]:
    """The K nearest reference kernels of each query and their orders, from
    the CUDA library (fs_recommend with duplicate marks)."""
    import torch

    import paper_1810_10496_gb300 as fs

    q = torch.as_tensor(np.ascontiguousarray(queries, dtype=np.float32)).to(db.device)
    ex = None
    if exclude is not None:
        ex = torch.as_tensor(np.asarray(exclude, dtype=np.int32)).to(db.device)
    idx, dist, seqs, lens, dup = fs.fs_recommend(db, q, k, exclude=ex, l_max=l_max, want_dup=True)
    torch.cuda.synchronize(db.device)
    idx, dist, seqs, lens, dup = (t.cpu().numpy() for t in (idx, dist, seqs, lens, dup))
    out = []
    for i in range(idx.shape[0]):
        keep = idx[i] >= 0
        out.append(Suggestion(rows=[int(r) for r in idx[i][keep]],
                              distances=[float(d) for d in dist[i][keep]],
                              orders=[seqs[i, c, :min(int(lens[i, c]), l_max)].copy()
                                      for c in range(idx.shape[1]) if keep[c]],
                              duplicate_of=[int(d) for d in dup[i][keep]]))
    return out


def evaluate(suggestion: Suggestion, fitness: Callable[[np.ndarray], float],
             fallback_fitness: float, good_enough: Callable[[float], bool] | None = None,
             memo: dict | None = None, budget: int | None = None) -> Outcome:
    """Evaluates the suggested orders in rank order (higher fitness is
    better). Duplicates are skipped, fitness values already in `memo` (keyed
    by the order's bytes, for this kernel) are recalled, at most `budget`
    orders are compiled, and the loop stops once `good_enough(best)` holds.
    The fallback's fitness is the floor of the result."""
    memo = {} if memo is None else memo
    best, best_order = float(fallback_fitness), None
    out = Outcome(best, None, True, 0, 0)
    for slot, order in enumerate(suggestion.orders):
        if suggestion.duplicate_of[slot] >= 0:
            out.trace.append((slot, None))
            continue
        key = np.asarray(order, dtype=np.int16).tobytes()
        if key in memo:
            val = memo[key]
            out.recalled += 1
        else:
            if budget is not None and out.compiled >= budget:
                break
            val = float(fitness(order))
            memo[key] = val
            out.compiled += 1
        out.trace.append((slot, val))
        if val > best:
            best, best_order = val, order
        if good_enough is not None and good_enough(best):
            out.stopped_early = True
            break
    out.fitness, out.order, out.fallback = best, best_order, best_order is None
    return out


def geomean(v) -> float:
    v = np.asarray(v, dtype=np.float64)
    return float(math.exp(np.log(v).mean()))


def k_sweep(knn: Callable[[np.ndarray, int, np.ndarray], np.ndarray], features: np.ndarray,
            speedup: np.ndarray, order_of: Sequence[int] | None = None,
            ks: Sequence[int] | None = None, n_random: int = 1000, seed: int = 0) -> dict:
    """Sec. 4.2's experiment on a reference set of n kernels, leave-one-out.

    `knn(features, k, exclude)` returns the [n][k] nearest rows of every
    kernel among the others (fs_knn's answer); `speedup[i][j]` is kernel i
    compiled with kernel j's best order, over the fallback (1.0). A kernel
    takes the best of the fallback and its selected orders. Returns, per K,
    the geometric mean over kernels for the K nearest and for random
    selection (K distinct other kernels, `n_random` draws per kernel, the
    geometric mean over all of them)."""
    n = features.shape[0]
    ks = list(ks) if ks is not None else list(range(1, n))
    exclude = np.arange(n, dtype=np.int32)
    rng = np.random.default_rng(seed)
    res = {}
    for k in ks:
        idx = np.asarray(knn(features, k, exclude))
        best_nn = [max(1.0, max(speedup[i, j] for j in idx[i, :k] if j >= 0)) for i in range(n)]
        others = [np.delete(np.arange(n), i) for i in range(n)]
        best_rand = []
        for _ in range(n_random):
            for i in range(n):
                pick = rng.choice(others[i], size=k, replace=False)
                best_rand.append(max(1.0, speedup[i, pick].max()))
        res[k] = {"nearest": geomean(best_nn), "random": geomean(best_rand)}
    return res


def gpu_knn(prec: str = "fp32"):
    """A `knn` for k_sweep backed by the CUDA library: builds the reference
    set on the current device and answers with fs_knn (leave-one-out)."""
    def knn(features, k, exclude):
        import torch

        import paper_1810_10496_gb300 as fs
        dev = torch.device("cuda")
        n = features.shape[0]
        x = torch.as_tensor(np.ascontiguousarray(features, dtype=np.float32), device=dev)
        off = torch.zeros(n + 1, dtype=torch.int64, device=dev)
        ids = torch.zeros(1, dtype=torch.int16, device=dev)
        db = fs.fs_build_db(x, off, ids[:0], prec=prec)
        try:
            idx, _ = fs.fs_knn(db, x, k, exclude=torch.as_tensor(exclude, device=dev))
            torch.cuda.synchronize()
            return idx.cpu().numpy()
        finally:
            db.close()
    return knn
