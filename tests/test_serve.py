"""Host logic of the continuous-batching server, driven by a fake engine on
the CPU: admission within the memory budget and the slot limit, requests
joining batches while others are in flight, and every result routed back to
the request that asked for it."""
import numpy as np
import pytest

from paper_1810_10496_gb300 import serve


class FakeEngine:
    """Completes a batch a fixed time after launch; its 'answer' for a query
    row is derived from that row, so misrouted results are detected."""

    def __init__(self, clock, latency=0.002, bytes_per_query=1000):
        self.clock, self.latency, self.bpq = clock, latency, bytes_per_query
        self.launched = []

    def batch_bytes(self, nq):
        return 4096 + nq * self.bpq

    def launch(self, q, offset, slot):
        self.launched.append((self.clock(), q.shape[0], offset, slot))
        return (self.clock() + self.latency, q.copy())

    def done(self, h):
        return self.clock() >= h[0]

    def results(self, h):
        q = h[1]
        idx = (q[:, :3] * 10).astype(np.int32)
        dist = q[:, :3].astype(np.float32)
        seqs = np.repeat(idx[:, :, None], 4, axis=2).astype(np.int16)
        lens = np.full(idx.shape, 4, np.int32)
        return idx, dist, seqs, lens


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-4          # every look at the clock advances it
        return self.t


def _requests(n, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        b = int(rng.integers(1, 40))
        q = rng.integers(0, 1000, size=(b, 8)).astype(np.float32)
        out.append(serve.Request(i, 0.0005 * i, q))
    return out


def test_all_requests_answered_and_routed():
    clock = FakeClock()
    eng = FakeEngine(clock)
    srv = serve.Server(eng, arena_bytes=200_000, slots=3, max_batch=64)
    reqs = _requests(300)
    serve.run_open_loop(srv, reqs, clock=clock, max_wall_s=1e6)
    for r in reqs:
        assert r.done is not None and r.latency >= 0
        assert np.array_equal(r.idx, (r.queries[:, :3] * 10).astype(np.int32))
        assert np.array_equal(r.lens, np.full((r.queries.shape[0], 3), 4))
    st = srv.stats
    assert st.queries == sum(r.queries.shape[0] for r in reqs)
    assert st.max_inflight <= 3
    assert st.max_arena_used <= 200_000
    assert max(st.batch_sizes) <= 64
    # requests were merged into batches while others were in flight
    assert st.batches < len(reqs) and st.max_inflight >= 2
    # no two in-flight batches shared arena bytes
    assert srv.arena.used == 0 and srv.arena.free == [(0, 200_000)]


def test_memory_admission_blocks_and_resumes():
    clock = FakeClock()
    eng = FakeEngine(clock, latency=0.01, bytes_per_query=5000)
    # every request fits, but rarely two batches at once
    srv = serve.Server(eng, arena_bytes=250_000, slots=4, max_batch=64)
    reqs = _requests(60, seed=1)
    serve.run_open_loop(srv, reqs, clock=clock, max_wall_s=1e6)
    assert all(r.done is not None for r in reqs)
    assert srv.stats.admissions_blocked_by_memory > 0
    assert srv.stats.max_arena_used <= 250_000


def test_oversized_requests_are_refused():
    clock = FakeClock()
    srv = serve.Server(FakeEngine(clock), arena_bytes=10_000, slots=2, max_batch=16)
    with pytest.raises(ValueError):
        srv.submit(serve.Request(0, 0.0, np.zeros((17, 8), np.float32)))
    with pytest.raises(ValueError):
        srv.submit(serve.Request(1, 0.0, np.zeros((16, 8), np.float32)))


def test_arena_first_fit_and_coalescing():
    a = serve.Arena(4096)
    x = a.alloc(1000)
    y = a.alloc(1000)
    z = a.alloc(1000)
    assert x[0] == 0 and y[0] == 1024 and z[0] == 2048
    assert a.alloc(2000) is None
    a.release(*y)
    assert a.alloc(2000) is None and a.largest() == 1024
    a.release(*x)
    assert a.largest() == 2048
    w = a.alloc(2000)
    assert w[0] == 0
    a.release(*w)
    a.release(*z)
    assert a.free == [(0, 4096)] and a.used == 0


def test_poisson_arrivals_rate():
    pool = np.zeros((100, 4), np.float32)
    reqs = serve.poisson_requests(pool, rate_qps=100_000, duration_s=2.0, bmin=1, bmax=99, seed=3)
    nq = sum(r.queries.shape[0] for r in reqs)
    assert abs(nq / 2.0 - 100_000) / 100_000 < 0.05
    assert all(np.diff([r.arrival for r in reqs]) >= 0)


def test_min_fill_holds_small_batches_only_while_busy():
    """With a batch in flight, a small new batch waits for min_batch queries
    or max_wait_s; with nothing in flight it starts at once; every request
    is still answered."""
    clock = FakeClock()
    eng = FakeEngine(clock, latency=0.005)
    srv = serve.Server(eng, arena_bytes=400_000, slots=4, max_batch=128, min_batch=64,
                       max_wait_s=0.003)
    rng = np.random.default_rng(5)
    reqs = [serve.Request(i, 0.0004 * i, rng.integers(0, 9, size=(4, 8)).astype(np.float32))
            for i in range(200)]
    serve.run_open_loop(srv, reqs, clock=clock, max_wall_s=1e6)
    assert all(r.done is not None for r in reqs)
    st = srv.stats
    assert st.held_for_fill > 0
    # the first batch went alone at once: nothing was in flight
    assert eng.launched[0][1] == 4
    # later batches either filled up or waited out max_wait_s: far fewer
    # launches than with the greedy policy
    greedy_clock = FakeClock()
    greedy_eng = FakeEngine(greedy_clock, latency=0.005)
    greedy = serve.Server(greedy_eng, arena_bytes=400_000, slots=4, max_batch=128)
    reqs2 = [serve.Request(r.rid, r.arrival, r.queries) for r in reqs]
    serve.run_open_loop(greedy, reqs2, clock=greedy_clock, max_wall_s=1e6)
    assert st.batches < greedy.stats.batches
    # no request waited in the queue much beyond max_wait_s plus one batch
    assert max(r.latency for r in reqs) < 0.003 + 3 * 0.005 + 0.01
    for r in reqs:
        assert np.array_equal(r.idx, (r.queries[:, :3] * 10).astype(np.int32))


def test_overload_sheds_at_admission_and_bounds_latency():
    """Offered load far above capacity: with a queue bound, requests beyond
    it are refused at arrival (never answered), every accepted request is
    answered and routed, and the accepted requests' latency stays bounded by
    the queue's work; without a bound nothing is refused and the latency
    grows with the backlog."""
    def run(max_queued):
        clock = FakeClock()
        eng = FakeEngine(clock, latency=0.01)
        srv = serve.Server(eng, arena_bytes=400_000, slots=2, max_batch=64,
                           max_queued=max_queued)
        rng = np.random.default_rng(9)
        reqs = [serve.Request(i, 0.0002 * i, rng.integers(0, 9, size=(8, 8)).astype(np.float32))
                for i in range(600)]
        serve.run_open_loop(srv, reqs, clock=clock, max_wall_s=1e6)
        return srv, reqs

    srv, reqs = run(128)
    shed = [r for r in reqs if r.shed]
    kept = [r for r in reqs if not r.shed]
    assert srv.stats.shed_requests == len(shed) > 0
    assert srv.stats.shed_queries == sum(r.queries.shape[0] for r in shed)
    assert all(r.done is None and r.idx is None for r in shed)
    assert all(r.done is not None for r in kept)
    for r in kept:
        assert np.array_equal(r.idx, (r.queries[:, :3] * 10).astype(np.int32))
    assert srv.stats.queries == sum(r.queries.shape[0] for r in kept)
    bounded = max(r.latency for r in kept)
    summary = serve.latency_summary(reqs)
    assert summary["n"] == len(kept)

    srv2, reqs2 = run(None)
    assert srv2.stats.shed_requests == 0 and all(r.done is not None for r in reqs2)
    assert max(r.latency for r in reqs2) > 2 * bounded
    assert srv.stats.launch_s >= 0.0 and srv.stats.retire_s >= 0.0
