"""fs_knn_noalloc: the search for callers that cannot allocate device memory.

Its scratch is one fixed array inside the library (FS_NOALLOC_SCRATCH_BYTES
per GPU) instead of a caller-provided workspace. Callers that need it are
those that may not call cudaMalloc at all, for example a plug-in inside a
framework that owns all device memory, or a serving loop whose memory was
fixed at start-up. The test checks, through the C-ABI, that two calls in a
row give the same neighbours and distances as fs_knn with a workspace, and
that a call too large for the array is refused. This file is named so that
pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import fsgen

pytestmark = pytest.mark.gpu

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


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_no_alloc_matches_workspace_path(fs, prec):
    import torch
    w = fsgen.make("tiny_k3", n=30011, q=200, f=128, seed=13)
    db = fs.fs_build_db(_dev(w.x), _dev(w.seq_off), _dev(w.seq_ids), prec=prec)
    q = _dev(w.queries)
    i_ref, d_ref = fs.fs_knn(db, q, 5)
    torch.cuda.synchronize()
    i_ref, d_ref = i_ref.cpu().numpy(), d_ref.cpu().numpy()
    L = fs.lib()
    ks = np.full(1, 5, dtype=np.int32)
    for _ in range(2):      # two calls in a row share the static scratch
        idx = torch.full((w.q, 5), -7, dtype=torch.int32, device="cuda")
        dist = torch.full((w.q, 5), -7.0, dtype=torch.float32, device="cuda")
        st = L.fs_knn_noalloc(db.handle, q.data_ptr(), w.q, None, ks.ctypes.data, None,
                              idx.data_ptr(), dist.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
        assert st == fs.FS_OK, fs.fs_last_error()
        torch.cuda.synchronize()
        fs.fs_db_check(db)
        ig, dg = idx.cpu().numpy(), dist.cpu().numpy()
        assert np.array_equal(ig, i_ref)
        assert np.all(np.abs(dg.astype(np.float64) - d_ref) <= RTOL * np.abs(d_ref) + ATOL)
    db.close()


def test_no_alloc_refuses_oversized_calls(fs):
    import torch
    w = fsgen.make("tiny_k3", n=4096, q=1, f=64, seed=1)
    db = fs.fs_build_db(_dev(w.x), _dev(w.seq_off), _dev(w.seq_ids), prec="fp32")
    nq = 60000
    need = fs.fs_workspace_size(db, nq)
    assert need > fs.FS_NOALLOC_SCRATCH_BYTES
    q = torch.ones((nq, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(fs.FsError) as e:
        fs.fs_knn_noalloc(db, q, 3)
    assert e.value.status == fs.FS_ENOMEM and "static" in str(e.value)
    db.close()
