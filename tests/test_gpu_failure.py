"""Failure reporting of the bounded device-side waits, without a GPU fault.

Every wait of the tensor-core scans gives up after a limit; the scan then
stops, releases what it holds, records FS_ETIMEOUT in the database's status
word and the call's queries get padding instead of a partial answer. The
test makes the waits run out on purpose with the library's test aid
(fs_db_set_wait_test: every scan block skips the copy of its first database
tile, so nothing is ever in flight that could fault), checks that the status
arrives within a host deadline, and that the next normal call on the same
database and context answers as the oracle does.
"""
import time

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


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_wait_runs_out_and_is_reported(fs, prec):
    import torch
    w = fsgen.make("tiny_k3", n=30000, q=300, f=128, seed=5)
    db = fs.fs_build_db(_dev(w.x), _dev(w.seq_off), _dev(w.seq_ids), prec=prec)
    q = _dev(w.queries)
    fs.fs_db_check(db)
    fs.fs_db_set_wait_test(db, True, 100)       # 100 us per wait
    t0 = time.perf_counter()
    idx, dist = fs.fs_knn(db, q, 3)
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    with pytest.raises(fs.FsError) as e:
        fs.fs_db_check(db)
    assert e.value.status == fs.FS_ETIMEOUT
    assert elapsed < 2.0, elapsed               # the waits ran out, far below the default 2 s each
    # no partial answer: every slot is padding
    assert np.all(idx.cpu().numpy() == -1) and np.all(np.isinf(dist.cpu().numpy()))
    fs.fs_db_check(db)                          # the status word was cleared

    # the same database and context work normally afterwards
    fs.fs_db_set_wait_test(db, False, 0)
    idx, dist = fs.fs_knn(db, q, 3)
    torch.cuda.synchronize()
    fs.fs_db_check(db)
    i_o, d_o, _ = oracle.knn(w.x, w.queries, 3)
    assert np.array_equal(idx.cpu().numpy(), i_o)
    err = np.abs(dist.cpu().numpy().astype(np.float64) - d_o)
    assert np.all(err <= 1e-5 * d_o + 1e-6)
    db.close()


def test_wait_limit_argument_checked(fs):
    w = fsgen.make("tiny_k3", n=100, q=2, f=64, seed=1)
    db = fs.fs_build_db(_dev(w.x), _dev(w.seq_off), _dev(w.seq_ids), prec="bf16")
    with pytest.raises(fs.FsError) as e:
        fs.fs_db_set_wait_test(db, True, 3_000_000)
    assert e.value.status == fs.FS_EINVAL
    db.close()
