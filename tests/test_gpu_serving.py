"""Serving on the GPU: each request's answer is the same alone and in the
mix of continuously batched requests, and equals the oracle's."""
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


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_alone_equals_in_the_mix(fs, prec):
    import torch
    from paper_1810_10496_gb300 import serve
    w = fsgen.make("tiny_k3", n=50_000, q=1, f=128, seed=17)
    dev = torch.device("cuda")
    db = fs.fs_build_db(torch.from_numpy(w.x).to(dev), torch.from_numpy(w.seq_off).to(dev),
                        torch.from_numpy(w.seq_ids).to(dev), prec=prec)
    pool = fsgen.query_rows(18, 2000, 128)
    k, slots, max_batch = 3, 3, 256
    arena = 3 * (max_batch * 128 * 4 + max_batch * k * (12 + 256) + fs.fs_workspace_size(db, max_batch)) + (1 << 20)
    eng = serve.GpuEngine(fs, db, 128, k, slots, max_batch, arena)
    srv = serve.Server(eng, arena_bytes=arena, slots=slots, max_batch=max_batch)
    reqs = serve.poisson_requests(pool, rate_qps=2_000_000, duration_s=0.02, bmin=1, bmax=64, seed=5)
    assert len(reqs) > 100
    serve.run_open_loop(srv, reqs)
    assert srv.stats.batches < len(reqs)        # requests were batched together
    # each request alone
    for r in reqs[::7]:
        i, d, s, l, _ = fs.fs_recommend(db, torch.from_numpy(r.queries).to(dev), k)
        torch.cuda.synchronize()
        assert np.array_equal(i.cpu().numpy(), r.idx)
        assert np.array_equal(d.cpu().numpy(), r.dist)
        assert np.array_equal(s.cpu().numpy(), r.seqs) and np.array_equal(l.cpu().numpy(), r.lens)
    # and against the oracle on a sample
    for r in reqs[::37]:
        i_o, d_o, s_o, l_o = oracle.recommend(w.x, r.queries, k, w.seq_off, w.seq_ids, 128)
        assert np.array_equal(r.idx, i_o) and np.array_equal(r.seqs, s_o)
        assert np.all(np.abs(r.dist - d_o) <= 1e-5 * d_o + 1e-6)
