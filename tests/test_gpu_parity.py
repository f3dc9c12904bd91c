"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Neighbour indices and gathered phase orders must match the oracle exactly;
distances must satisfy |d_gpu - d_oracle| <= 1e-5 * d_oracle + 1e-6 (the
relative tolerance of the result contract with an absolute floor, because
d = 1 - s is rounded to float). Every case runs for each scan precision:
the precision changes how candidates are found, never the answer.
"""
import numpy as np
import pytest

import fsgen
import oracle

pytestmark = pytest.mark.gpu

PRECS = ["fp32", "bf16", "fp8"]
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


def build_db(fs, x, seq_off, seq_ids, prec, seg_off=None):
    return fs.fs_build_db(_dev(x), _dev(seq_off), _dev(seq_ids), seg_off, prec)


def run(fs, db, queries, k, q_seg_off=None, exclude=None, l_max=128):
    import torch
    ex = None if exclude is None else _dev(np.asarray(exclude, dtype=np.int32))
    idx, dist, seqs, lens, dup = fs.fs_recommend(db, _dev(queries), k, q_seg_off=q_seg_off,
                                                 exclude=ex, l_max=l_max, want_dup=True)
    torch.cuda.synchronize()
    fs.fs_db_check(db)
    return (idx.cpu().numpy(), dist.cpu().numpy(), seqs.cpu().numpy(), lens.cpu().numpy(),
            dup.cpu().numpy())


def assert_same(idx_g, dist_g, idx_o, dist_o, k=None):
    k = idx_o.shape[1] if k is None else k
    ig, dg = idx_g[:, :k], dist_g[:, :k]
    bad = np.nonzero(np.any(ig != idx_o, axis=1))[0]
    assert len(bad) == 0, f"index mismatch in queries {bad[:8]}: gpu {ig[bad[:3]]} oracle {idx_o[bad[:3]]}"
    valid = idx_o >= 0
    err = np.abs(dg[valid].astype(np.float64) - dist_o[valid])
    assert np.all(err <= RTOL * np.abs(dist_o[valid]) + ATOL), float(err.max())
    assert np.all(np.isinf(dg[~valid]))


def dup_reference(idx, seq_off, seq_ids):
    out = np.full(idx.shape, -1, dtype=np.int32)
    for r in range(idx.shape[0]):
        for c in range(idx.shape[1]):
            j = idx[r, c]
            if j < 0:
                continue
            a = seq_ids[seq_off[j]:seq_off[j + 1]]
            for c2 in range(c):
                j2 = idx[r, c2]
                if j2 >= 0 and np.array_equal(seq_ids[seq_off[j2]:seq_off[j2 + 1]], a):
                    out[r, c] = c2
                    break
    return out


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", ["tiny_k1", "tiny_k3"])
def test_tiny(fs, name, prec):
    w = fsgen.make(name)
    k = w.k[0]
    db = build_db(fs, w.x, w.seq_off, w.seq_ids, prec)
    idx, dist, seqs, lens, dup = run(fs, db, w.queries, k)
    i_o, d_o, s_o, l_o = oracle.recommend(w.x, w.queries, k, w.seq_off, w.seq_ids, 128)
    assert_same(idx, dist, i_o, d_o)
    assert np.array_equal(seqs, s_o) and np.array_equal(lens, l_o)
    assert np.array_equal(dup, dup_reference(i_o, w.seq_off, w.seq_ids))
    st = fs.fs_db_stats(db)
    assert st["queries"] == w.q and st["certified"] + st["fallback"] == w.q


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("f,n,q,k", [(128, 20011, 300, 3), (55, 9000, 131, 5), (256, 6151, 77, 1),
                                     (64, 4097, 260, 16)])
def test_medium_ragged(fs, prec, f, n, q, k):
    """Several scan tiles, query tiles and chunks, all with ragged tails."""
    w = fsgen.make("tiny_k3", n=n, q=q, f=f, seed=11)
    db = build_db(fs, w.x, w.seq_off, w.seq_ids, prec)
    idx, dist, seqs, lens, _ = run(fs, db, w.queries, k, l_max=64)
    i_o, d_o, s_o, l_o = oracle.recommend(w.x, w.queries, k, w.seq_off, w.seq_ids, 64)
    assert_same(idx, dist, i_o, d_o)
    assert np.array_equal(seqs, s_o) and np.array_equal(lens, l_o)


@pytest.mark.parametrize("prec", PRECS)
def test_non_integer_features(fs, prec):
    """Averages of counts (Sec. 4.1) are not integers: the binary64 step must
    still reproduce the oracle's sequential sums bit for bit."""
    rng = np.random.default_rng(5)
    x = (rng.gamma(0.5, 3.0, size=(3000, 55)) * (rng.random((3000, 55)) < 0.6)).astype(np.float32)
    qy = (rng.gamma(0.5, 3.0, size=(40, 55))).astype(np.float32)
    off, ids = fsgen.phase_orders(1, 3000)
    db = build_db(fs, x, off, ids, prec)
    idx, dist, *_ = run(fs, db, qy, 4)
    i_o, d_o, _ = oracle.knn(x, qy, 4)
    assert_same(idx, dist, i_o, d_o)


@pytest.mark.parametrize("prec", PRECS)
def test_padding_zero_rows_and_queries(fs, prec):
    w = fsgen.make("tiny_k3", n=5, q=4, f=32)
    x = w.x.copy()
    x[1] = 0.0
    qy = w.queries.copy()
    qy[2] = 0.0
    db = build_db(fs, x, w.seq_off, w.seq_ids, prec)
    idx, dist, seqs, lens, _ = run(fs, db, qy, 8)
    i_o, d_o, s_o, l_o = oracle.recommend(x, qy, 8, w.seq_off, w.seq_ids, 128)
    assert_same(idx, dist, i_o, d_o)
    assert np.all(idx[:, 5:] == -1) and np.all(lens[:, 5:] == 0) and np.all(seqs[:, 5:] == -1)
    assert list(idx[2, :5]) == [0, 1, 2, 3, 4] and np.all(dist[2, :5] == 1.0)


@pytest.mark.parametrize("prec", PRECS)
def test_zero_queries_among_many(fs, prec):
    """Zero queries spread over several query tiles and the ragged tail, some
    with a row excluded: every cosine is 0, so the lowest usable indices win
    at d = 1, and the queries sharing their tiles and warps keep their own
    answers."""
    w = fsgen.make("tiny_k3", n=20000, q=300, f=256, seed=11)
    qy = w.queries.copy()
    zero = [0, 31, 32, 127, 130, 255, 299]
    qy[zero] = 0.0
    excl = np.full(300, -1, np.int32)
    excl[[31, 130, 299]] = [0, 2, 5]
    excl[[1, 200]] = [4, 19999]
    db = build_db(fs, w.x, w.seq_off, w.seq_ids, prec)
    for ex in (None, excl):
        idx, dist, *_ = run(fs, db, qy, 4, exclude=ex)
        i_o, d_o, _ = oracle.knn(w.x, qy, 4, exclude=ex)
        assert_same(idx, dist, i_o, d_o)
        for z in zero:
            e = -1 if ex is None else ex[z]
            assert list(idx[z]) == [r for r in range(6) if r != e][:4]
            assert np.all(dist[z] == 1.0)


@pytest.mark.parametrize("prec", PRECS)
def test_ties_and_duplicates_take_lower_index(fs, prec):
    """Exact duplicates: equal binary64 scores, lower index first. 200 copies
    of the best row overflow every candidate list, so the exact fallback scan
    must answer."""
    w = fsgen.make("tiny_k3", n=3000, q=6, f=64, seed=3)
    x = w.x.copy()
    x[1000:1200] = x[7]
    x[2000:2003] = 2 * x[8]        # parallel rows: s = 1 exactly
    qy = np.stack([x[7], x[8], 3 * x[7], w.queries[0], w.queries[1], x[2500]])
    off, ids = fsgen.phase_orders(2, 3000)
    db = build_db(fs, x, off, ids, prec)
    idx, dist, *_ = run(fs, db, qy, 5)
    i_o, d_o, _ = oracle.knn(x, qy, 5)
    assert_same(idx, dist, i_o, d_o)
    assert list(idx[0]) == [7, 1000, 1001, 1002, 1003]
    st = fs.fs_db_stats(db)
    assert st["fallback"] >= 1 and st["certified"] + st["fallback"] == 6


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_four_entry_lists(fs, prec):
    """The 4-entry candidate lists of the tensor-core scans (a tuning): k = 3
    and k = 4 on random rows, and k = 3 with 20 copies of a query's best row
    (more rows tied than a list holds, so the fallback answers)."""
    w = fsgen.make("tiny_k3", n=20_000, q=200, f=64, seed=17)
    x = w.x.copy()
    x[5000:5020] = x[11]
    qy = w.queries.copy()
    qy[0] = x[11]
    db = build_db(fs, x, w.seq_off, w.seq_ids, prec)
    fs.fs_db_set_tuning(db, {"list_len": 4})
    for k in (3, 4):
        idx, dist, *_ = run(fs, db, qy, k)
        i_o, d_o, _ = oracle.knn(x, qy, k)
        assert_same(idx, dist, i_o, d_o)
    assert list(idx[0, :3]) == [11, 5000, 5001]


@pytest.mark.parametrize("prec", PRECS)
def test_leave_one_out(fs, prec):
    """Sec. 4.2: each kernel queries the database without its own entry."""
    w = fsgen.make("tiny_k3", n=2000, q=1, f=64, seed=9)
    qy = w.x[:300]
    excl = np.arange(300, dtype=np.int32)
    excl[::7] = -1
    db = build_db(fs, w.x, w.seq_off, w.seq_ids, prec)
    idx, dist, *_ = run(fs, db, qy, 3, exclude=excl)
    i_o, d_o, _ = oracle.knn(w.x, qy, 3, exclude=excl)
    assert_same(idx, dist, i_o, d_o)
    assert np.all(idx[excl >= 0, :] != excl[excl >= 0, None])


@pytest.mark.parametrize("prec", PRECS)
def test_segments(fs, prec):
    """Independent databases of uneven size searched in one call, including
    empty databases and segments without queries."""
    rng = np.random.default_rng(4)
    sizes = np.array([1000, 0, 37, 5000, 1, 2600, 300, 0, 12000])
    nq = np.array([5, 3, 0, 130, 2, 17, 0, 4, 260])
    ks = np.array([3, 1, 2, 3, 16, 1, 3, 2, 4])
    seg = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    qseg = np.concatenate([[0], np.cumsum(nq)]).astype(np.int32)
    x = fsgen.db_rows(21, int(seg[-1]), 128)
    qy = fsgen.query_rows(21, int(qseg[-1]), 128)
    off, ids = fsgen.phase_orders(21, int(seg[-1]))
    excl = rng.integers(-1, 3, size=int(qseg[-1])).astype(np.int32)
    db = build_db(fs, x, off, ids, prec, seg_off=seg)
    idx, dist, seqs, lens, _ = run(fs, db, qy, ks, q_seg_off=qseg, exclude=excl)
    kmax = ks.max()
    for s in range(len(sizes)):
        a, b = qseg[s], qseg[s + 1]
        if a == b:
            continue
        xs = x[seg[s]:seg[s + 1]]
        i_o, d_o, _ = oracle.knn(xs, qy[a:b], int(ks[s]), exclude=excl[a:b])
        assert_same(idx[a:b], dist[a:b], i_o, d_o)
        assert np.all(idx[a:b, ks[s]:] == -1) and np.all(np.isinf(dist[a:b, ks[s]:kmax]))
        so, _ = oracle.gather(i_o, off[seg[s]:seg[s + 1] + 1] - off[seg[s]],
                              ids[off[seg[s]]:off[seg[s + 1]]], 128)
        assert np.array_equal(seqs[a:b, :ks[s]], so)


@pytest.mark.parametrize("prec", PRECS)
def test_gather_truncation_and_empty_orders(fs, prec):
    w = fsgen.make("tiny_k3", n=800, q=50, f=64, seed=2)
    off, ids = fsgen.phase_orders(2, 800, min_len=0)
    db = build_db(fs, w.x, off, ids, prec)
    idx, dist, seqs, lens, dup = run(fs, db, w.queries, 6, l_max=40)
    i_o, d_o, s_o, l_o = oracle.recommend(w.x, w.queries, 6, off, ids, 40)
    assert_same(idx, dist, i_o, d_o)
    assert np.array_equal(seqs, s_o) and np.array_equal(lens, l_o)
    assert np.array_equal(dup, dup_reference(i_o, off, ids))


def test_normalize_matches_float64(fs):
    import torch
    rng = np.random.default_rng(0)
    x = np.zeros((1000, 72), np.float32)
    x[:, :55] = rng.gamma(0.4, 5.0, size=(1000, 55))
    x[10] = 0.0
    x[11, 3] = np.nan
    xt = _dev(x)[:, :55]            # strided rows (ld = 72)
    xu, inv = fs.fs_normalize(xt)
    xu, inv = xu.cpu().numpy(), inv.cpu().numpy()
    x64 = x[:, :55].astype(np.float64)
    nrm = np.sqrt((x64 ** 2).sum(1))
    ok = np.isfinite(nrm) & (nrm > 0)
    ref = x64[ok] / nrm[ok, None]
    assert np.max(np.abs(xu[ok] - ref)) < 4e-7
    assert np.all(np.abs(inv[ok] * nrm[ok] - 1) < 4e-7)
    assert np.all(xu[10] == 0) and inv[10] == 0
    assert np.all(np.isnan(xu[11])) and np.isnan(inv[11])


def test_errors_are_reported(fs):
    import torch
    w = fsgen.make("tiny_k3", n=100, q=4, f=32)
    bad = w.x.copy()
    bad[3, 4] = np.inf
    with pytest.raises(fs.FsError) as e:
        build_db(fs, bad, w.seq_off, w.seq_ids, "fp32")
    assert e.value.status == fs.FS_EINVAL
    bad_off = w.seq_off.copy()
    bad_off[5] = bad_off[6] + 1
    with pytest.raises(fs.FsError):
        build_db(fs, w.x, bad_off, w.seq_ids, "fp32")
    db = build_db(fs, w.x, w.seq_off, w.seq_ids, "fp32")
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(fs.FsError) as e:
        fs.fs_knn(db, _dev(w.queries), 3, workspace=ws)
    assert e.value.status == fs.FS_ENOMEM
    qy = w.queries.copy()
    qy[1, 0] = np.nan
    fs.fs_knn(db, _dev(qy), 3)
    with pytest.raises(fs.FsError) as e:
        fs.fs_db_check(db)
    assert e.value.status == fs.FS_EINVAL
    fs.fs_db_check(db)        # the status word was cleared


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_full_scale_sampled(fs, prec):
    """1,048,576 x 128 database, 4,096 queries, k = 3 (the FP32-at-scale
    workload), in the launch configuration the benchmark times; 256 sampled
    queries are checked against the oracle on the whole database."""
    import torch
    w = fsgen.make("fp32_scale", workers=8)
    db = build_db(fs, w.x, w.seq_off, w.seq_ids, prec)
    idx, dist, seqs, lens, _ = run(fs, db, w.queries, 3)
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(w.q, size=256, replace=False))
    i_o, d_o, s_o, l_o = oracle.recommend(w.x, w.queries[pick], 3, w.seq_off, w.seq_ids, 128)
    assert_same(idx[pick], dist[pick], i_o, d_o)
    assert np.array_equal(seqs[pick], s_o) and np.array_equal(lens[pick], l_o)
    st = fs.fs_db_stats(db)
    assert st["certified"] + st["fallback"] == w.q
    # every query: the returned rows are ordered and their distances valid
    assert np.all(np.diff(dist, axis=1) >= -1e-6) and np.all((dist >= 0) & (dist <= 1))


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_many_uneven_segments(fs, prec):
    """300 databases of log-uniform size (10..5000 rows), 0-40 queries each,
    k in {1, 3}: every database's answer equals the oracle's on it alone."""
    rng = np.random.default_rng(8)
    sizes = np.floor(np.exp(rng.uniform(np.log(10), np.log(5000), size=300))).astype(np.int64)
    nq = rng.integers(0, 41, size=300)
    ks = rng.choice(np.array([1, 3]), size=300)
    seg = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    qseg = np.concatenate([[0], np.cumsum(nq)]).astype(np.int32)
    x = fsgen.db_rows(31, int(seg[-1]), 64)
    qy = fsgen.query_rows(31, int(qseg[-1]), 64)
    off, ids = fsgen.phase_orders(31, int(seg[-1]))
    db = build_db(fs, x, off, ids, prec, seg_off=seg)
    idx, dist, *_ = run(fs, db, qy, ks, q_seg_off=qseg)
    for s in range(300):
        a, b = qseg[s], qseg[s + 1]
        if a == b:
            continue
        i_o, d_o, _ = oracle.knn(x[seg[s]:seg[s + 1]], qy[a:b], int(ks[s]))
        assert_same(idx[a:b], dist[a:b], i_o, d_o)


def test_cuda_graph_replay(fs):
    """A captured call replays to the eager answer, also after the query
    buffer is refilled (the plan and tensor maps are baked into the graph)."""
    import torch
    rng = np.random.default_rng(12)
    sizes = np.array([3000, 17, 9000, 1200, 0, 4000])
    nq = np.array([40, 3, 130, 0, 5, 70])
    ks = np.array([3, 1, 3, 1, 2, 3])
    seg = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    qseg = np.concatenate([[0], np.cumsum(nq)]).astype(np.int32)
    x = fsgen.db_rows(41, int(seg[-1]), 128)
    off, ids = fsgen.phase_orders(41, int(seg[-1]))
    db = build_db(fs, x, off, ids, "bf16", seg_off=seg)
    q1 = fsgen.query_rows(41, int(qseg[-1]), 128)
    q2 = fsgen.query_rows(42, int(qseg[-1]), 128)
    qd = _dev(q1)
    ws = torch.empty(fs.fs_workspace_size(db, qd.shape[0], qseg), dtype=torch.uint8, device="cuda")
    out = dict(idx=torch.empty((qd.shape[0], 3), dtype=torch.int32, device="cuda"),
               dist=torch.empty((qd.shape[0], 3), dtype=torch.float32, device="cuda"),
               seq_out=torch.empty((qd.shape[0], 3, 128), dtype=torch.int16, device="cuda"),
               seq_len=torch.empty((qd.shape[0], 3), dtype=torch.int32, device="cuda"))
    fs.fs_recommend(db, qd, ks, q_seg_off=qseg, workspace=ws, **out)   # warm-up, eager
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fs.fs_recommend(db, qd, ks, q_seg_off=qseg, workspace=ws, **out)
    for qh in (q1, q2, q1):
        qd.copy_(torch.from_numpy(qh))
        g.replay()
        torch.cuda.synchronize()
        gi, gd = out["idx"].cpu().numpy(), out["dist"].cpu().numpy()
        ei, ed, *_ = run(fs, db, qh, ks, q_seg_off=qseg)
        assert np.array_equal(gi, ei) and np.array_equal(gd, ed)
    for s in range(len(sizes)):
        a, b = qseg[s], qseg[s + 1]
        if a < b:
            i_o, d_o, _ = oracle.knn(x[seg[s]:seg[s + 1]], q1[a:b], int(ks[s]))
            assert_same(gi[a:b], gd[a:b], i_o, d_o)


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_mid_size_many_query_tiles(fs, prec):
    """150,001 rows and 600 queries (5 query tiles, chunked so the chunks in
    flight fit L2, with a ragged last chunk)."""
    w = fsgen.make("tiny_k3", n=150_001, q=600, f=128, seed=23)
    db = build_db(fs, w.x, w.seq_off, w.seq_ids, prec)
    idx, dist, seqs, lens, _ = run(fs, db, w.queries, 3)
    i_o, d_o, s_o, l_o = oracle.recommend(w.x, w.queries, 3, w.seq_off, w.seq_ids, 128)
    assert_same(idx, dist, i_o, d_o)
    assert np.array_equal(seqs, s_o) and np.array_equal(lens, l_o)


@pytest.mark.parametrize("prec", PRECS)
def test_near_duplicates_relative_distance(fs, prec):
    """Rows that differ from a query in one feature (distances of about 1e-8
    to 2e-4) and a row parallel to it (distance 0): the distances must hold
    1e-5 relative with no absolute floor, and 0 exactly."""
    w = fsgen.make("tiny_k3", n=6000, q=40, f=128, seed=29)
    x = w.x.copy()
    qy = 16.0 * w.queries                     # larger counts: one count is a small change
    for i in range(40):
        base = qy[i]
        j = 150 * i
        top = int(np.argmax(base))
        x[j] = base
        x[j, top] += 1.0                      # one count more on the largest feature
        x[j + 1] = base
        x[j + 1, (top + 1) % 128] += 3.0      # three counts more elsewhere
        x[j + 2] = 2.0 * base                 # parallel: s = 1 exactly
    db = build_db(fs, x, w.seq_off, w.seq_ids, prec)
    idx, dist, *_ = run(fs, db, qy, 3)
    i_o, d_o, _ = oracle.knn(x, qy, 3)
    assert np.array_equal(idx, i_o)
    assert np.all(d_o[:, 0] == 0.0) and np.all(dist[:, 0] == 0.0)
    err = np.abs(dist.astype(np.float64) - d_o)
    assert np.all(err <= 1e-5 * d_o), float(np.max(err / np.maximum(d_o, 1e-300)))
    assert np.all(d_o[:, 1:] < 1e-3)          # the case is what it says


@pytest.mark.parametrize("k", [1, 3])
def test_fp8_certified_path(fs, k):
    """Queries that are scaled copies of database rows, far from every other
    row: FP8's candidate lists certify their answers, so the certified path
    (not the exact fallback) gives them, and they must equal the oracle's."""
    w = fsgen.make("tiny_k3", n=20000, q=1, f=128, seed=19)
    pick = np.arange(3, 20000, 97)[:200]
    qy = 3.0 * w.x[pick]
    db = build_db(fs, w.x, w.seq_off, w.seq_ids, "fp8")
    fs.fs_db_stats(db, reset=True)
    idx, dist, seqs, lens, _ = run(fs, db, qy, k)
    i_o, d_o, s_o, l_o = oracle.recommend(w.x, qy, k, w.seq_off, w.seq_ids, 128)
    assert_same(idx, dist, i_o, d_o)
    assert np.array_equal(seqs, s_o) and np.array_equal(lens, l_o)
    st = fs.fs_db_stats(db)
    assert st["queries"] == len(pick) and st["certified"] + st["fallback"] == len(pick)
    # (a 20,000-row database in one-tile chunks: 158 lists per query start
    # together, the band's worst case; at scale FP8 certifies every query)
    assert st["certified"] >= 0.9 * len(pick), st
