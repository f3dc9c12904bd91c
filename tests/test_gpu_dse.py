"""The Sec. 4.2 procedure on the CUDA library: leave-one-out neighbours,
suggested orders with duplicate marks, and the K sweep, against the oracle."""
import numpy as np
import pytest

import fsgen
import oracle
from paper_1810_10496_gb300 import dse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_10496_gb300 import build
    build.build()
    import paper_1810_10496_gb300 as m
    return m


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_k_sweep_on_gpu_matches_oracle(fs, prec):
    suite = fsgen.dse_suite(seed=0)
    gk = dse.gpu_knn(prec)
    ok = lambda f, k, e: oracle.knn(f, f, k, exclude=e)[0]  # noqa: E731
    n = suite.features.shape[0]
    ex = np.arange(n, dtype=np.int32)
    for k in (1, 3, n - 1):
        assert np.array_equal(gk(suite.features, k, ex), ok(suite.features, k, ex)), k
    a = dse.k_sweep(gk, suite.features, suite.speedup, n_random=50, seed=2)
    b = dse.k_sweep(ok, suite.features, suite.speedup, n_random=50, seed=2)
    assert a == b


def test_suggest_orders_and_duplicates(fs):
    import torch
    suite = fsgen.dse_suite(seed=0)
    n = suite.features.shape[0]
    dev = torch.device("cuda")
    db = fs.fs_build_db(torch.from_numpy(suite.features).to(dev),
                        torch.from_numpy(suite.seq_off).to(dev),
                        torch.from_numpy(suite.seq_ids).to(dev), prec="fp32")
    sug = dse.suggest(db, suite.features, n - 1, exclude=np.arange(n))
    i_o, _, _ = oracle.knn(suite.features, suite.features, n - 1, exclude=np.arange(n))
    orders = [suite.seq_ids[suite.seq_off[i]:suite.seq_off[i + 1]] for i in range(n)]
    for q in range(n):
        s = sug[q]
        assert s.rows == list(i_o[q]) and q not in s.rows
        for c, r in enumerate(s.rows):
            assert np.array_equal(s.orders[c], orders[r])
            first = next(c2 for c2 in range(c + 1) if np.array_equal(orders[s.rows[c2]], orders[r]))
            assert s.duplicate_of[c] == (first if first < c else -1)
        # every distinct order is compiled once
        seen = []
        out = dse.evaluate(s, lambda o: (seen.append(o.tobytes()), 1.0 + len(o) / 1e3)[1], 1.0)
        assert len(seen) == len(set(seen)) == out.compiled
    db.close()
