"""Standardised Euclidean and Manhattan distances on the CUDA library against
the oracle: indices and gathered orders exact, distances within
1e-5 * d + 1e-6."""
import numpy as np
import pytest

import fsgen
import oracle

pytestmark = pytest.mark.gpu

METRICS = ["euclidean", "manhattan"]
RTOL, ATOL = 1e-5, 1e-6


@pytest.fixture(scope="module")
def fs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_10496_gb300 import build
    build.build()
    import paper_1810_10496_gb300 as m
    return m


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _db(fs, x, metric, seg_off=None):
    off, ids = fsgen.phase_orders(9, x.shape[0])
    db = fs.fs_build_db(_dev(x), _dev(off), _dev(ids), seg_off, "fp32")
    fs.fs_db_set_metric(db, metric)
    return db, off, ids


def _check(idx, dist, i_o, d_o):
    assert np.array_equal(idx, i_o), np.nonzero(np.any(idx != i_o, axis=1))[0][:8]
    v = i_o >= 0
    assert np.all(np.abs(dist[v].astype(np.float64) - d_o[v]) <= RTOL * d_o[v] + ATOL)
    assert np.all(np.isinf(dist[~v]))


def _knn(fs, db, q, k, **kw):
    import torch
    idx, dist = fs.fs_knn(db, _dev(q), k, **kw)
    torch.cuda.synchronize()
    fs.fs_db_check(db)
    return idx.cpu().numpy(), dist.cpu().numpy()


@pytest.mark.parametrize("metric", METRICS)
@pytest.mark.parametrize("n,f,q,k", [(64, 64, 15, 3), (5003, 55, 300, 3), (20_000, 128, 129, 1),
                                     (3000, 32, 40, 16)])
def test_metric_matches_oracle(fs, metric, n, f, q, k):
    x = fsgen.db_rows(21, n, f)
    qy = fsgen.query_rows(21, q, f)
    db, _, _ = _db(fs, x, metric)
    idx, dist = _knn(fs, db, qy, k)
    i_o, d_o = oracle.knn_metric(x, qy, k, metric)
    _check(idx, dist, i_o, d_o)
    db.close()


@pytest.mark.parametrize("metric", METRICS)
def test_metric_constant_columns_exclude_and_duplicates(fs, metric):
    """A constant feature, leave-one-out, and 30 exact copies of a row (ties
    among more rows than a candidate list holds: the binary64 scan answers)."""
    x = fsgen.db_rows(22, 6000, 40)
    x[:, 7] = 5.0
    x[2000:2030] = x[17]
    qy = np.concatenate([x[:50], x[17:18]])
    excl = np.concatenate([np.arange(50), [-1]]).astype(np.int32)
    db, _, _ = _db(fs, x, metric)
    idx, dist = _knn(fs, db, qy, 5, exclude=_dev(excl))
    i_o, d_o = oracle.knn_metric(x, qy, 5, metric, exclude=excl)
    _check(idx, dist, i_o, d_o)
    assert list(idx[-1]) == [17, 2000, 2001, 2002, 2003]
    db.close()


@pytest.mark.parametrize("metric", METRICS)
def test_metric_segments(fs, metric):
    """Each database standardises with its own statistics."""
    rng = np.random.default_rng(23)
    sizes = rng.integers(20, 3000, size=30)
    nq = rng.integers(0, 30, size=30)
    ks = rng.choice(np.array([1, 3]), size=30).astype(np.int32)
    seg = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    qseg = np.concatenate([[0], np.cumsum(nq)]).astype(np.int32)
    x = fsgen.db_rows(23, int(seg[-1]), 48)
    qy = fsgen.query_rows(23, int(qseg[-1]), 48)
    db, _, _ = _db(fs, x, metric, seg_off=seg)
    idx, dist = _knn(fs, db, qy, ks, q_seg_off=qseg)
    for s in range(30):
        a, b = qseg[s], qseg[s + 1]
        if a == b:
            continue
        i_o, d_o = oracle.knn_metric(x[seg[s]:seg[s + 1]], qy[a:b], int(ks[s]), metric)
        _check(idx[a:b, :ks[s]], dist[a:b, :ks[s]], i_o, d_o)
    db.close()


def test_metric_switch_back_and_errors(fs):
    x = fsgen.db_rows(24, 2000, 64)
    qy = fsgen.query_rows(24, 20, 64)
    db, _, _ = _db(fs, x, "manhattan")
    fs.fs_db_set_metric(db, "cosine")
    idx, dist = _knn(fs, db, qy, 3)
    i_o, d_o, _ = oracle.knn(x, qy, 3)
    _check(idx, dist, i_o, d_o)
    db.close()
    off, ids = fsgen.phase_orders(9, 2000)
    db2 = fs.fs_build_db(_dev(x), _dev(off), _dev(ids), None, "bf16")
    with pytest.raises(fs.FsError) as e:
        fs.fs_db_set_metric(db2, "euclidean")
    assert e.value.status == fs.FS_EUNSUPPORTED
    db2.close()
