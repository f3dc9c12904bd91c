"""The autotuner and the tuning parameters on the GPU: every tuning gives
the oracle's answers, the tuner applies and caches its choice, and the
parameters are range-checked."""
import numpy as np
import pytest

import fsgen
import oracle

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


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_every_tuning_matches_oracle(fs, prec):
    """Single segment, several query tiles and row chunks: each candidate of
    the tuner (items per block, list length, L2 share) gives the oracle's
    rows and distances."""
    from paper_1810_10496_gb300 import tune
    import torch
    n, q, f, k = 70_001, 300, 128, 3
    x = fsgen.db_rows(41, n, f)
    qy = fsgen.query_rows(41, q, f)
    off, ids = fsgen.phase_orders(41, n)
    db = fs.fs_build_db(_dev(x), _dev(off), _dev(ids), None, prec)
    i_o, d_o, _ = oracle.knn(x, qy, k)
    qd = _dev(qy)
    for c in tune.candidates(prec, 1, k):
        fs.fs_db_set_tuning(db, c)
        assert fs.fs_db_get_tuning(db) == {**dict.fromkeys(fs.TUNING_FIELDS, 0), **c}
        idx, dist = fs.fs_knn(db, qd, k)
        torch.cuda.synchronize()
        fs.fs_db_check(db)
        ig, dg = idx.cpu().numpy(), dist.cpu().numpy()
        assert np.array_equal(ig, i_o), c
        assert np.all(np.abs(dg - d_o) <= 1e-5 * np.abs(d_o) + 1e-6), c
    db.close()


def test_autotune_segments_and_cache(fs, tmp_path):
    """Many uneven segments: the tuner picks a tuning, applies it, caches it;
    a second call reads the cache; answers equal the oracle's."""
    from paper_1810_10496_gb300 import tune
    import torch
    rng = np.random.default_rng(12)
    sizes = np.floor(np.exp(rng.uniform(np.log(100), np.log(20000), size=64))).astype(np.int64)
    nq = rng.integers(1, 64, size=64)
    ks = rng.choice(np.array([1, 3]), size=64).astype(np.int32)
    seg = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    qseg = np.concatenate([[0], np.cumsum(nq)]).astype(np.int32)
    x = fsgen.db_rows(43, int(seg[-1]), 128)
    qy = fsgen.query_rows(43, int(qseg[-1]), 128)
    off, ids = fsgen.phase_orders(43, int(seg[-1]))
    db = fs.fs_build_db(_dev(x), _dev(off), _dev(ids), seg, "bf16")
    qd = _dev(qy)
    cache = str(tmp_path / "tuning.json")
    res = tune.autotune(db, qd, ks, q_seg_off=qseg, reps=2, cache_path=cache)
    assert not res["cached"] and res["ms"] <= res["default_ms"]
    full = {**dict.fromkeys(fs.TUNING_FIELDS, 0), **res["tuning"]}
    assert fs.fs_db_get_tuning(db) == full
    fs.fs_db_set_tuning(db, None)
    again = tune.autotune(db, qd, ks, q_seg_off=qseg, cache_path=cache)
    assert again["cached"] and again["tuning"] == res["tuning"]
    assert fs.fs_db_get_tuning(db) == full
    idx, dist = fs.fs_knn(db, qd, ks, q_seg_off=qseg)
    torch.cuda.synchronize()
    idx = idx.cpu().numpy()
    for s in range(64):
        a, b = qseg[s], qseg[s + 1]
        i_o, _, _ = oracle.knn(x[seg[s]:seg[s + 1]], qy[a:b], int(ks[s]))
        assert np.array_equal(idx[a:b, :ks[s]], i_o), s
    db.close()


def test_tuning_range_checks(fs):
    x = fsgen.db_rows(44, 1000, 64)
    off, ids = fsgen.phase_orders(44, 1000)
    db = fs.fs_build_db(_dev(x), _dev(off), _dev(ids), None, "bf16")
    for bad in ({"items_per_block": 65}, {"items_per_block": -1}, {"list_len": 12},
                {"l2_share_pct": 101}, {"l2_share_pct": -2}, {"scan_pairs": 2}):
        with pytest.raises(fs.FsError):
            fs.fs_db_set_tuning(db, bad)
    assert fs.fs_db_get_tuning(db) == dict.fromkeys(fs.TUNING_FIELDS, 0)
    with pytest.raises(ValueError):
        fs.fs_db_set_tuning(db, {"tile": 3})
    db.close()


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_scan_pairs_match_oracle(fs, prec):
    """Tensor-core scans on clusters of two SMs (scan_pairs): one segment
    with an odd number of query tiles (the last pair's second tile lies past
    the queries), k = 1, 3 and 16, and many uneven segments."""
    import torch
    n, q, f = 50_001, 300, 128
    x = fsgen.db_rows(45, n, f)
    qy = fsgen.query_rows(45, q, f)
    off, ids = fsgen.phase_orders(45, n)
    db = fs.fs_build_db(_dev(x), _dev(off), _dev(ids), None, prec)
    fs.fs_db_set_tuning(db, {"scan_pairs": 1})
    qd = _dev(qy)
    for k in (1, 3, 16):
        idx, dist = fs.fs_knn(db, qd, k)
        torch.cuda.synchronize()
        fs.fs_db_check(db)
        i_o, d_o, _ = oracle.knn(x, qy, k)
        assert np.array_equal(idx.cpu().numpy(), i_o), k
        dg = dist.cpu().numpy()
        assert np.all(np.abs(dg - d_o) <= 1e-5 * np.abs(d_o) + 1e-6), k
    db.close()

    rng = np.random.default_rng(46)
    sizes = np.floor(np.exp(rng.uniform(np.log(50), np.log(8000), size=40))).astype(np.int64)
    nq = rng.integers(0, 300, size=40)
    ks = rng.choice(np.array([1, 3]), size=40).astype(np.int32)
    seg = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    qseg = np.concatenate([[0], np.cumsum(nq)]).astype(np.int32)
    x = fsgen.db_rows(47, int(seg[-1]), 64)
    qy = fsgen.query_rows(47, int(qseg[-1]), 64)
    off, ids = fsgen.phase_orders(47, int(seg[-1]))
    db = fs.fs_build_db(_dev(x), _dev(off), _dev(ids), seg, prec)
    fs.fs_db_set_tuning(db, {"scan_pairs": 1})
    idx, dist = fs.fs_knn(db, _dev(qy), ks, q_seg_off=qseg)
    torch.cuda.synchronize()
    fs.fs_db_check(db)
    idx = idx.cpu().numpy()
    for s in range(40):
        a, b = qseg[s], qseg[s + 1]
        if a == b:
            continue
        i_o, _, _ = oracle.knn(x[seg[s]:seg[s + 1]], qy[a:b], int(ks[s]))
        assert np.array_equal(idx[a:b, :ks[s]], i_o), s
    db.close()
