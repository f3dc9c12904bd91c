"""Pins for the CPU oracle: it is checked against things other than itself.

* closed forms worked out by hand (tests/golden/closed_forms.json);
* a second, independent brute force in plain C (oracle/naive_knn.c);
* exact rational arithmetic on integer features;
* invariants of cosine k-NN (self match, permutation, prefix, scaling);
* a library special case (torch.topk of a float64 product of unit vectors);
* the Table 1 phase orders gathered back exactly.

A final test plants typical mistakes into a copy of the oracle's arithmetic
and checks that these pins catch each one.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import fsgen
import oracle
from oracle import build as cbuild


def _case_s(c):
    if "s_inv_sqrt" in c:
        return 1.0 / math.sqrt(c["s_inv_sqrt"])
    return c["s_num"] / c["s_den"]


def test_closed_forms(golden_dir):
    cases = json.load(open(os.path.join(golden_dir, "closed_forms.json")))["cases"]
    for c in cases:
        q = np.array([c["q"]], dtype=np.float32)
        x = np.array([c["x"]], dtype=np.float32)
        s = oracle.cosine_scores(q, x)[0, 0]
        # D, A, B themselves
        assert oracle.dot_seq(q, x)[0, 0] == c["D"], c["name"]
        assert oracle.norm2(q)[0] == c["A"] and oracle.norm2(x)[0] == c["B"], c["name"]
        want = _case_s(c)
        assert abs(s - want) <= 2 * np.spacing(abs(want) + 1e-300), (c["name"], s, want)
        idx, dist, _ = oracle.knn(x, q, 1)
        assert idx[0, 0] == 0
        assert abs(dist[0, 0] - (1.0 - want)) <= 4e-16, c["name"]


def test_exact_rationals_hit_exactly():
    # s = 8/9, 24/25, 2/7 and 1 are the correctly rounded quotients
    q = np.array([[1, 2, 2], [3, 4, 0], [2, 3, 6]], dtype=np.float32)
    x = np.array([[2, 1, 2], [4, 3, 0], [1, 0, 0]], dtype=np.float32)
    s = oracle.cosine_scores(q, x)
    assert s[0, 0] == 8 / 9 and s[1, 1] == 24 / 25 and s[2, 2] == 2 / 7


@pytest.mark.parametrize("name", ["tiny_k1", "tiny_k3"])
def test_c_brute_force_matches_integer(name):
    w = fsgen.make(name)
    k = w.k[0]
    i1, d1, s1 = cbuild.naive_knn(w.x, w.queries, k)
    i2, d2, s2 = oracle.knn(w.x, w.queries, k)
    assert np.array_equal(i1, i2)
    assert np.array_equal(d1, d2) and np.array_equal(s1, s2)


def test_c_brute_force_matches_non_integer():
    rng = np.random.default_rng(7)
    x = rng.standard_normal((90, 55)).astype(np.float32)
    q = rng.standard_normal((9, 55)).astype(np.float32)
    x[5] = 0.0
    i1, d1, s1 = cbuild.naive_knn(x, q, 5)
    i2, d2, s2 = oracle.knn(x, q, 5, chunk=37)
    assert np.array_equal(i1, i2)
    assert np.array_equal(s1, s2)


def test_blas_product_equals_sequential_loop_on_integers():
    w = fsgen.make("tiny_k3", n=300, q=20, f=128)
    assert oracle.exact_integer_inputs(w.queries, w.x)
    a = oracle.cosine_scores(w.queries, w.x, use_blas=True)
    b = oracle.cosine_scores(w.queries, w.x, use_blas=False)
    assert np.array_equal(a, b)


def test_exact_rational_order():
    """Integer features: sign(D)*D^2/(A*B) in exact rationals orders rows as
    the binary64 score does, except where binary64 rounds two distinct
    rationals to one value (then the lower index must come first)."""
    w = fsgen.make("tiny_k3", n=200, q=6, f=64)
    xi = w.x.astype(np.int64)
    qi = w.queries.astype(np.int64)
    s = oracle.cosine_scores(w.queries, w.x)
    merged = 0
    for r in range(qi.shape[0]):
        A = int((qi[r] * qi[r]).sum())
        keys = []
        for j in range(xi.shape[0]):
            D = int((qi[r] * xi[j]).sum())
            B = int((xi[j] * xi[j]).sum())
            keys.append(Fraction(0) if A == 0 or B == 0 else
                        Fraction(D * abs(D), A * B))
        exact = sorted(range(len(keys)), key=lambda j: (-keys[j], j))
        fp = np.lexsort((np.arange(len(keys)), -s[r]))
        for a, b in zip(exact[:-1], exact[1:]):
            if keys[a] != keys[b] and s[r, a] == s[r, b]:
                merged += 1
        # every strict rational inequality is kept or merged, never inverted
        for a, b in zip(fp[:-1], fp[1:]):
            assert keys[a] >= keys[b] or s[r, a] == s[r, b]
            if s[r, a] == s[r, b]:
                assert a < b
    assert merged <= 2


def test_self_match_and_duplicates():
    w = fsgen.make("tiny_k3", n=100, q=8, f=64)
    for r in range(8):
        pos = 17 + 9 * r
        x = np.insert(w.x, pos, w.queries[r], axis=0)
        idx, dist, sc = oracle.knn(x, w.queries[r:r + 1], 1)
        s_all = oracle.cosine_scores(w.queries[r:r + 1], x)[0]
        first_one = int(np.nonzero(s_all == s_all.max())[0][0])
        assert sc[0, 0] == 1.0 and dist[0, 0] == 0.0
        assert idx[0, 0] == first_one and first_one <= pos
    # exact duplicates rank by index
    x = np.repeat(w.x[:5], 3, axis=0)
    idx, _, sc = oracle.knn(x, w.x[2:3], 3)
    assert list(idx[0]) == [6, 7, 8]


def test_permutation_permutes_result():
    w = fsgen.make("tiny_k3", n=500, q=10, f=64)
    rng = np.random.default_rng(3)
    perm = rng.permutation(w.n)
    i1, d1, s1 = oracle.knn(w.x, w.queries, 3)
    i2, d2, s2 = oracle.knn(w.x[perm], w.queries, 3)
    s = oracle.cosine_scores(w.queries, w.x)
    for r in range(w.q):
        # same scores; the same rows unless two rows tie exactly
        assert np.array_equal(s1[r], s2[r])
        if len(set(s[r][i1[r]])) == 3 and np.sum(s[r] >= s1[r, -1]) == 3:
            assert list(perm[i2[r]]) == list(i1[r])


def test_k3_prefix_is_k1():
    w = fsgen.make("tiny_k3")
    i1, d1, _ = oracle.knn(w.x, w.queries, 1)
    i3, d3, _ = oracle.knn(w.x, w.queries, 3)
    assert np.array_equal(i3[:, :1], i1) and np.array_equal(d3[:, :1], d1)


def test_scaling_rows():
    w = fsgen.make("tiny_k3", n=300, q=10, f=64)
    s = oracle.cosine_scores(w.queries, w.x)
    s2 = oracle.cosine_scores(w.queries, w.x * 4)   # power of two: same bits
    assert np.array_equal(s, s2)
    s3 = oracle.cosine_scores(w.queries, w.x * 3)   # other factor: same up to rounding
    assert np.max(np.abs(s - s3)) < 1e-15
    i1, _, _ = oracle.knn(w.x, w.queries, 3)
    i3, _, _ = oracle.knn(w.x * 3, w.queries, 3)
    assert np.array_equal(i1, i3)


def test_library_topk_agrees():
    torch = pytest.importorskip("torch")
    w = fsgen.make("tiny_k3", n=2000, q=16, f=128)
    x = torch.from_numpy(w.x.astype(np.float64))
    q = torch.from_numpy(w.queries.astype(np.float64))
    xn = x / x.norm(dim=1, keepdim=True).clamp_min(1e-300)
    qn = q / q.norm(dim=1, keepdim=True).clamp_min(1e-300)
    sc = qn @ xn.T
    top = torch.topk(sc, 3, dim=1)
    idx, _, s = oracle.knn(w.x, w.queries, 3)
    for r in range(w.q):
        if np.all(np.diff(s[r]) < -1e-12):
            assert list(top.indices[r].numpy()) == list(idx[r])
        assert np.allclose(top.values[r].numpy(), s[r], rtol=0, atol=1e-14)


def test_zero_vectors_and_padding():
    x = np.array([[0, 0, 0], [1, 0, 0], [0, 0, 0], [0, 2, 0]], dtype=np.float32)
    idx, dist, sc = oracle.knn(x, np.zeros((1, 3), np.float32), 6)
    assert list(idx[0]) == [0, 1, 2, 3, -1, -1]
    assert list(dist[0, :4]) == [1.0] * 4 and np.all(np.isinf(dist[0, 4:]))
    idx, dist, _ = oracle.knn(x, np.array([[0, 1, 0]], np.float32), 3)
    assert list(idx[0]) == [3, 0, 1] and dist[0, 0] == 0.0 and dist[0, 1] == 1.0
    idx, dist, _ = oracle.knn(np.zeros((0, 3), np.float32), np.ones((2, 3), np.float32), 2)
    assert np.all(idx == -1) and np.all(np.isinf(dist))


def test_zero_padding_features():
    """55 features (the paper's MILEPOST count, Sec. 4.1) padded with zeros
    to 64 give the same neighbours and distances."""
    w = fsgen.make("tiny_k3", n=400, q=12, f=55)
    pad = lambda a: np.concatenate([a, np.zeros((a.shape[0], 9), np.float32)], axis=1)
    i1, d1, _ = oracle.knn(w.x, w.queries, 3)
    i2, d2, _ = oracle.knn(pad(w.x), pad(w.queries), 3)
    assert np.array_equal(i1, i2) and np.array_equal(d1, d2)


def _table1(golden_dir):
    names, orders = [], []
    for line in open(os.path.join(golden_dir, "table1_phase_orders.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        names.append(parts[0])
        orders.append(parts[1:])
    return names, orders


def test_table1_gather(golden_dir):
    names, orders = _table1(golden_dir)
    assert len(names) == 15 and sum(1 for o in orders if not o) == 3
    vocab = {}
    for o in orders:
        for p in o:
            vocab.setdefault(p, len(vocab))
    lens = [len(o) for o in orders]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    ids = np.array([vocab[p] for o in orders for p in o], dtype=np.int16)
    n = len(names)
    # benchmark b: a strong feature b and a weak feature b+1 (mod n)
    x = np.zeros((n, 16), np.float32)
    for b in range(n):
        x[b, b] = 10
        x[b, (b + 1) % n] = 3
    q = np.zeros((n, 16), np.float32)
    for b in range(n):
        q[b, b] = 10
        q[b, (b + 1) % n] = 4
    idx, dist, seqs, slen = oracle.recommend(x, q, 2, off, ids, l_max=16)
    for b in range(n):
        assert idx[b, 0] == b
        assert idx[b, 1] in ((b - 1) % n, (b + 1) % n)
        for c in range(2):
            j = idx[b, c]
            want = [vocab[p] for p in orders[j]]
            assert slen[b, c] == len(want)
            assert list(seqs[b, c, :len(want)]) == want
            assert np.all(seqs[b, c, len(want):] == -1)
    # COVAR repeats -loop-unswitch three times; order and repeats survive
    cv = names.index("COVAR")
    got = seqs[cv, 0, :slen[cv, 0]]
    assert list(got).count(vocab["-loop-unswitch"]) == 3


def test_segments_are_independent():
    w = fsgen.make("tiny_k3", n=700, q=30, f=64)
    seg = np.array([0, 100, 100, 450, 700])
    qseg = np.array([0, 5, 9, 9, 30])
    ks = [3, 1, 2, 3]
    res = oracle.knn_segments(w.x, w.queries, seg, qseg, ks)
    for s in range(4):
        i, d, _ = oracle.knn(w.x[seg[s]:seg[s + 1]], w.queries[qseg[s]:qseg[s + 1]], ks[s])
        assert np.array_equal(res[s][0], i)
    assert np.all(res[1][0] == -1)


def test_leave_one_out_equals_deleting_the_row():
    """Sec. 4.2: with a kernel as the query, only the other kernels are
    candidates. Excluding row j must equal searching the database without
    row j (indices above j shift by one)."""
    w = fsgen.make("tiny_k3", n=150, q=12, f=32)
    excl = np.array([3, -1, 0, 149, 77, 77, 5, 6, 7, 8, 9, 10])
    i1, d1, _ = oracle.knn(w.x, w.queries, 3, exclude=excl, chunk=40)
    for r in range(12):
        j = excl[r]
        if j < 0:
            i2, d2, _ = oracle.knn(w.x, w.queries[r:r + 1], 3)
        else:
            i2, d2, _ = oracle.knn(np.delete(w.x, j, axis=0), w.queries[r:r + 1], 3)
            i2 = np.where(i2 >= j, i2 + 1, i2)
        assert np.array_equal(i1[r], i2[0]) and np.array_equal(d1[r], d2[0])
    # a database row as its own query, left out: never returned, d > 0
    i3, d3, _ = oracle.knn(w.x[:20], w.x[:20], 1, exclude=np.arange(20))
    assert np.all(i3[:, 0] != np.arange(20))


def test_gather_truncates_and_pads():
    off = np.array([0, 0, 5, 9], dtype=np.int64)
    ids = np.arange(9, dtype=np.int16)
    seqs, lens = oracle.gather(np.array([[2, 0, 1, -1]]), off, ids, 3)
    assert list(lens[0]) == [4, 0, 5, 0]
    assert list(seqs[0, 0]) == [5, 6, 7] and list(seqs[0, 1]) == [-1, -1, -1]
    assert list(seqs[0, 2]) == [0, 1, 2] and list(seqs[0, 3]) == [-1, -1, -1]


# ---------------------------------------------------------------------------
# planted mistakes: each mutant must fail at least one pin


def _pins_pass(score_fn, knn_fn, golden_dir):
    """Re-run the numeric pins with a substitute score and k-NN function."""
    cases = json.load(open(os.path.join(golden_dir, "closed_forms.json")))["cases"]
    for c in cases:
        q = np.array([c["q"]], dtype=np.float64)
        x = np.array([c["x"]], dtype=np.float64)
        if abs(score_fn(q, x)[0, 0] - _case_s(c)) > 1e-12:
            return False
    x = np.array([[0, 0, 0], [1, 0, 0], [0, 0, 0], [0, 2, 0]], dtype=np.float64)
    if list(knn_fn(x, np.array([[0, 1, 0]], float), 3)[0][0]) != [3, 0, 1]:
        return False
    w = fsgen.make("tiny_k3", n=120, q=6, f=32)
    xd = np.repeat(w.x[:5], 3, axis=0).astype(np.float64)
    if list(knn_fn(xd, w.x[2:3].astype(np.float64), 3)[0][0]) != [6, 7, 8]:
        return False
    i_ref, _, _ = cbuild.naive_knn(w.x, w.queries, 3)
    if not np.array_equal(knn_fn(w.x.astype(np.float64), w.queries.astype(np.float64), 3)[0], i_ref):
        return False
    return True


def _mk_knn(score_fn, order="desc", tie="low"):
    def knn_fn(x, q, k):
        s = score_fn(q, x)
        idx = np.zeros((q.shape[0], k), dtype=np.int64)
        for r in range(q.shape[0]):
            j = np.arange(x.shape[0])
            key = -s[r] if order == "desc" else s[r]
            o = np.lexsort(((j if tie == "low" else -j), key))[:k]
            idx[r] = j[o]
        return idx, None, None
    return knn_fn


def test_planted_mistakes_are_caught(golden_dir):
    def good(q, x):
        return oracle.cosine_scores(q, x)

    def no_sqrt(q, x):
        s = oracle.dot_seq(q, x) / (oracle.norm2(q)[:, None] * oracle.norm2(x)[None, :])
        return np.nan_to_num(s)

    def wrong_norm(q, x):      # uses A twice instead of A and B
        a = oracle.norm2(q)
        return np.nan_to_num(oracle.dot_seq(q, x) / np.sqrt(a[:, None] * a[:, None]))

    def transposed(q, x):      # feature index taken from the wrong operand end
        return oracle.cosine_scores(q, x[:, ::-1])

    def dropped_term(q, x):    # last feature left out of D
        return np.nan_to_num(oracle.dot_seq(q[:, :-1], x[:, :-1])
                             / np.sqrt(oracle.norm2(q)[:, None] * oracle.norm2(x)[None, :]))

    def distance_as_score(q, x):
        return 1.0 - oracle.cosine_scores(q, x)

    assert _pins_pass(good, _mk_knn(good), golden_dir)
    for bad in (no_sqrt, wrong_norm, transposed, dropped_term, distance_as_score):
        assert not _pins_pass(bad, _mk_knn(bad), golden_dir), bad.__name__
    assert not _pins_pass(good, _mk_knn(good, order="asc"), golden_dir)
    assert not _pins_pass(good, _mk_knn(good, tie="high"), golden_dir)


# ---------------------------------------------------------------------------
# other metrics (standardised Euclidean and Manhattan)

def test_metric_closed_form_grid():
    """Rows at the corners of a 2 x 2 grid: mu = (1, 1), sigma = (1, 1), so
    z is the row minus (1, 1); the query (2, 0) sits on row 1."""
    x = np.array([[0, 0], [2, 0], [0, 2], [2, 2]], dtype=np.float32)
    mu, sigma = oracle.standardize_stats(x)
    assert np.array_equal(mu, [1.0, 1.0]) and np.array_equal(sigma, [1.0, 1.0])
    q = np.array([[2, 0]], dtype=np.float32)
    de = oracle.metric_distances(q, x, "euclidean", mu, sigma)[0]
    dm = oracle.metric_distances(q, x, "manhattan", mu, sigma)[0]
    assert np.array_equal(de, [2.0, 0.0, np.sqrt(8.0), 2.0])
    assert np.array_equal(dm, [2.0, 0.0, 4.0, 2.0])
    for m in ("euclidean", "manhattan"):
        idx, d = oracle.knn_metric(x, q, 4, m)
        # row 0 and row 3 tie at 2: the lower index first
        assert list(idx[0]) == [1, 0, 3, 2]
        assert d[0, 0] == 0.0


def test_metric_against_scipy():
    """scipy's z-score (population deviation) and cdist, an independent
    implementation, agree with the oracle to rounding."""
    scipy_stats = pytest.importorskip("scipy.stats")
    from scipy.spatial.distance import cdist
    x = fsgen.db_rows(5, 300, 24).astype(np.float64)
    q = fsgen.query_rows(5, 20, 24).astype(np.float64)
    mu, sigma = oracle.standardize_stats(x)
    zs = scipy_stats.zscore(x, axis=0, ddof=0)
    assert np.allclose(oracle.standardize(x, mu, sigma), np.nan_to_num(zs), rtol=1e-12, atol=1e-12)
    zq = oracle.standardize(q, mu, sigma)
    zx = oracle.standardize(x, mu, sigma)
    for m, sm in (("euclidean", "euclidean"), ("manhattan", "cityblock")):
        d = oracle.metric_distances(q, x, m, mu, sigma)
        assert np.allclose(d, cdist(zq, zx, sm), rtol=1e-12, atol=1e-12)


def test_metric_brute_force_loop_bit_exact():
    """The vectorised distances equal a plain loop in the stated order."""
    import math
    x = fsgen.db_rows(6, 12, 7).astype(np.float64)
    q = fsgen.query_rows(6, 3, 7).astype(np.float64)
    n, f = x.shape
    mu = [0.0] * f
    sg = [0.0] * f
    for j in range(f):
        acc = 0.0
        for i in range(n):
            acc = acc + x[i, j]
        mu[j] = acc / n
        acc = 0.0
        for i in range(n):
            d = x[i, j] - mu[j]
            acc = acc + d * d
        sg[j] = math.sqrt(acc / n)
    m2, s2 = oracle.standardize_stats(x)
    assert list(m2) == mu and list(s2) == sg
    z = lambda v, j: (v - mu[j]) / sg[j] if sg[j] > 0 else 0.0  # noqa: E731
    for metric in ("euclidean", "manhattan"):
        d = oracle.metric_distances(q, x, metric, m2, s2)
        for a in range(q.shape[0]):
            for b in range(n):
                acc = 0.0
                for j in range(f):
                    t = z(q[a, j], j) - z(x[b, j], j)
                    acc = acc + (t * t if metric == "euclidean" else abs(t))
                ref = math.sqrt(acc) if metric == "euclidean" else acc
                assert d[a, b] == ref


def test_metric_invariants():
    """Standardisation makes the ranking independent of each column's scale
    and offset; a constant column contributes nothing; permuting the rows
    permutes the result; the k = 1 answer opens the k = 3 answer."""
    rng = np.random.default_rng(11)
    x = rng.normal(size=(400, 9))
    q = rng.normal(size=(15, 9))
    for m in ("euclidean", "manhattan"):
        i0, d0 = oracle.knn_metric(x, q, 3, m)
        scale = rng.uniform(0.5, 4.0, size=9)
        shift = rng.normal(size=9)
        i1, d1 = oracle.knn_metric(x * scale + shift, q * scale + shift, 3, m)
        assert np.array_equal(i0, i1) and np.allclose(d0, d1, rtol=1e-9)
        xc = np.concatenate([x, np.full((400, 1), 7.0)], axis=1)
        qc = np.concatenate([q, np.full((15, 1), -3.0)], axis=1)
        i2, d2 = oracle.knn_metric(xc, qc, 3, m)
        assert np.array_equal(i0, i2) and np.array_equal(d0, d2)
        perm = rng.permutation(400)
        i3, _ = oracle.knn_metric(x[perm], q, 3, m)
        assert np.array_equal(perm[i3], i0)
        i4, _ = oracle.knn_metric(x, q, 1, m)
        assert np.array_equal(i4[:, 0], i0[:, 0])
        # leave-one-out: a database row as its own query, excluded
        i5, _ = oracle.knn_metric(x, x[:10], 1, m, exclude=np.arange(10))
        assert np.all(i5[:, 0] != np.arange(10))


def test_metric_planted_mistake_is_caught():
    """A plausible slip, the sample deviation (n - 1) instead of the
    population one, changes the distances the grid pins."""
    x = np.array([[0, 0], [2, 0], [0, 2], [2, 2]], dtype=np.float64)
    mu, sigma = oracle.standardize_stats(x)
    wrong = sigma * np.sqrt(4 / 3)
    q = np.array([[2.0, 0.0]])
    assert not np.array_equal(oracle.metric_distances(q, x, "euclidean", mu, wrong)[0],
                              [2.0, 0.0, np.sqrt(8.0), 2.0])
