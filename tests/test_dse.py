"""The evaluate-K loop and the K sweep of Sec. 4.2, on the CPU: the neighbour
search here is the oracle's (test infrastructure); the GPU tests run the same
procedure on the CUDA library."""
import numpy as np
import pytest

import fsgen
import oracle
from paper_1810_10496_gb300 import dse


def oracle_knn(features, k, exclude):
    return oracle.knn(features, features, k, exclude=exclude)[0]


def _suggestion(orders, dup):
    return dse.Suggestion(rows=list(range(len(orders))), distances=[0.1] * len(orders),
                          orders=[np.array(o, np.int16) for o in orders], duplicate_of=dup)


def test_evaluate_dedup_memo_fallback_and_early_stop():
    calls = []

    def fitness(order):
        calls.append(tuple(order))
        return {(1, 2): 1.3, (3,): 0.8, (4, 4): 1.6}[tuple(order)]

    s = _suggestion([[1, 2], [1, 2], [3], [4, 4]], [-1, 0, -1, -1])
    memo = {}
    out = dse.evaluate(s, fitness, 1.0, memo=memo)
    assert calls == [(1, 2), (3,), (4, 4)]          # the duplicate is not compiled
    assert out.compiled == 3 and out.fitness == 1.6 and not out.fallback
    assert list(out.order) == [4, 4]
    # the same kernel again: every fitness is recalled
    out2 = dse.evaluate(s, fitness, 1.0, memo=memo)
    assert calls == [(1, 2), (3,), (4, 4)] and out2.recalled == 3 and out2.compiled == 0
    # nothing beats the fallback: the fallback is the answer
    out3 = dse.evaluate(_suggestion([[3]], [-1]), fitness, 1.0)
    assert out3.fallback and out3.order is None and out3.fitness == 1.0
    # early stop once the requirement holds, and a compile budget
    out4 = dse.evaluate(s, fitness, 1.0, good_enough=lambda f: f >= 1.2)
    assert out4.stopped_early and out4.compiled == 1
    out5 = dse.evaluate(s, fitness, 1.0, budget=2)
    assert out5.compiled == 2 and out5.fitness == 1.3


def test_k_sweep_procedure():
    suite = fsgen.dse_suite(seed=0)
    n = suite.features.shape[0]
    res = dse.k_sweep(oracle_knn, suite.features, suite.speedup, n_random=200, seed=1)
    assert sorted(res) == list(range(1, n))
    near = [res[k]["nearest"] for k in range(1, n)]
    # the K nearest sets are nested, so the best can only grow with K
    assert all(b >= a - 1e-12 for a, b in zip(near, near[1:]))
    # at K = n - 1 both methods evaluate every other kernel's order
    assert res[n - 1]["nearest"] == pytest.approx(res[n - 1]["random"], rel=1e-12)
    # every result is at least the fallback
    assert all(v["nearest"] >= 1.0 and v["random"] >= 1.0 for v in res.values())
    # on a reference set made of families, the nearest kernels beat random picks at small K
    assert res[1]["nearest"] > res[1]["random"] and res[3]["nearest"] > res[3]["random"]


def test_dse_suite_shape_and_duplicates():
    s = fsgen.dse_suite(seed=3, n=15, f=55, duplicate_orders=2)
    assert s.features.shape == (15, 55) and s.speedup.shape == (15, 15)
    assert np.all(s.features >= 0) and np.all(s.features == np.rint(s.features))
    o = [s.seq_ids[s.seq_off[i]:s.seq_off[i + 1]] for i in range(15)]
    assert np.array_equal(o[14], o[0]) and np.array_equal(o[13], o[1])
    assert np.all(s.speedup > 0)
