"""Continuous-batching server for phase-order suggestion requests.

A request is a small batch of query feature vectors (new kernels, Sec. 4)
searched against one device-resident reference database. Requests that
arrive while others are on the GPU join the next batch as soon as an
in-flight slot and device memory are free, so work from different requests
overlaps on the device (one CUDA stream per slot). Every transient byte of a
batch (queries, workspace, outputs) is carved from one device arena; a batch
is admitted only when it fits, which is the memory-based admission.

Admission also sheds load: with `max_queued` set, a request that arrives
while the queue already holds that many queries is refused at once (marked
`shed`, never answered), so an overloaded server keeps bounded latency for
the requests it accepts instead of a queue that grows without end.

Each request's answer does not depend on which other requests share its
batch: the selection is exact (a pure function of the score and index of
each row), so a request alone and in the mix gets the same rows, distances
and phase orders.

The scheduler is host logic only; the device work is whatever `engine`
launches (``GpuEngine`` wraps the C library). Tests drive the scheduler with
a fake engine on the CPU.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

ALIGN = 256


def _round_up(n: int, a: int = ALIGN) -> int:
    return (n + a - 1) // a * a


class Arena:
    """First-fit allocator of byte ranges inside one buffer (offsets only)."""

    def __init__(self, nbytes: int):
        self.size = int(nbytes)
        self.free = [(0, self.size)]          # sorted, coalesced (offset, size)
        self.used = 0

    def alloc(self, nbytes: int):
        n = _round_up(max(int(nbytes), 1))
        for i, (off, sz) in enumerate(self.free):
            if sz >= n:
                if sz == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + n, sz - n)
                self.used += n
                return off, n
        return None

    def release(self, off: int, n: int):
        self.used -= n
        self.free.append((off, n))
        self.free.sort()
        merged = []
        for o, s in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + s)
            else:
                merged.append((o, s))
        self.free = merged

    def largest(self) -> int:
        return max((s for _, s in self.free), default=0)


@dataclass
class Request:
    rid: int
    arrival: float                     # seconds (server clock)
    queries: np.ndarray                # [b, F] float32
    done: float | None = None
    shed: bool = False                 # refused at admission (queue full)
    idx: np.ndarray | None = None
    dist: np.ndarray | None = None
    seqs: np.ndarray | None = None
    lens: np.ndarray | None = None

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival


@dataclass
class _Batch:
    requests: list
    nq: int
    mem: tuple
    handle: object
    slot: int


@dataclass
class ServerStats:
    batches: int = 0
    queries: int = 0
    max_inflight: int = 0
    max_arena_used: int = 0
    admissions_blocked_by_memory: int = 0
    held_for_fill: int = 0
    shed_requests: int = 0             # refused at arrival: the queue was full
    shed_queries: int = 0
    launch_s: float = 0.0              # host seconds spent launching batches
    retire_s: float = 0.0              # host seconds spent handing results back
    batch_sizes: list = field(default_factory=list)


class Server:
    """Continuous batching over `engine` with at most `slots` batches in
    flight, at most `max_batch` queries per batch and `arena_bytes` of
    transient device memory.

    While another batch is in flight, a new one waits until it holds
    `min_batch` queries or its oldest request has waited `max_wait_s`: the
    scan's cost is flat up to one query tile (128 queries), so a batch of a
    few queries launched next to a running one costs nearly as much as a
    full tile. With nothing in flight a batch starts at once."""

    def __init__(self, engine, arena_bytes: int, slots: int = 4, max_batch: int = 1024,
                 min_batch: int = 1, max_wait_s: float = 0.0, max_queued: int | None = None):
        self.engine = engine
        self.max_queued = max_queued
        self.arena = Arena(arena_bytes)
        self.slots = slots
        self.max_batch = max_batch
        self.min_batch = min_batch
        self.max_wait_s = max_wait_s
        self.queued = 0                        # queries waiting
        self.queue = collections.deque()
        self.inflight: list[_Batch] = []
        self.free_slots = list(range(slots))
        self.stats = ServerStats()

    def submit(self, req: Request) -> bool:
        """Queues `req`; False (and `req.shed` set) when the queue is full."""
        n = req.queries.shape[0]
        if n > self.max_batch:
            raise ValueError("a request may not exceed max_batch queries")
        if self.engine.batch_bytes(n) > self.arena.size:
            raise ValueError("a request needs more device memory than the whole arena")
        if self.max_queued is not None and self.queued + n > self.max_queued:
            req.shed = True
            self.stats.shed_requests += 1
            self.stats.shed_queries += n
            return False
        self.queue.append(req)
        self.queued += n
        return True

    def _complete(self, now_fn):
        still = []
        for b in self.inflight:
            if self.engine.done(b.handle):
                t0 = time.perf_counter()
                res = self.engine.results(b.handle)
                t = now_fn()
                row = 0
                for r in b.requests:
                    n = r.queries.shape[0]
                    r.idx, r.dist, r.seqs, r.lens = (a[row:row + n].copy() for a in res)
                    r.done = t
                    row += n
                self.arena.release(*b.mem)
                self.free_slots.append(b.slot)
                self.stats.retire_s += time.perf_counter() - t0
            else:
                still.append(b)
        self.inflight = still

    def _admit(self, now: float):
        while self.queue and self.free_slots:
            if (self.inflight and self.queued < self.min_batch
                    and now - self.queue[0].arrival < self.max_wait_s):
                self.stats.held_for_fill += 1
                return
            # the longest prefix of the queue that fits one batch and the arena
            take, nq = [], 0
            for r in self.queue:
                n = r.queries.shape[0]
                if nq + n > self.max_batch:
                    break
                if self.engine.batch_bytes(nq + n) > self.arena.largest():
                    break
                take.append(r)
                nq += n
            if not take:
                self.stats.admissions_blocked_by_memory += 1
                return
            mem = self.arena.alloc(self.engine.batch_bytes(nq))
            for _ in take:
                self.queue.popleft()
            self.queued -= nq
            slot = self.free_slots.pop()
            t0 = time.perf_counter()
            q = np.concatenate([r.queries for r in take]) if len(take) > 1 else take[0].queries
            handle = self.engine.launch(q, mem[0], slot)
            self.stats.launch_s += time.perf_counter() - t0
            self.inflight.append(_Batch(take, nq, mem, handle, slot))
            st = self.stats
            st.batches += 1
            st.queries += nq
            st.batch_sizes.append(nq)
            st.max_inflight = max(st.max_inflight, len(self.inflight))
            st.max_arena_used = max(st.max_arena_used, self.arena.used)

    def poll(self, now_fn=time.perf_counter):
        """Retire finished batches, then admit queued requests."""
        self._complete(now_fn)
        self._admit(now_fn())

    def idle(self) -> bool:
        return not self.queue and not self.inflight


def poisson_requests(pool: np.ndarray, rate_qps: float, duration_s: float, bmin: int, bmax: int,
                     seed: int = 0):
    """Requests of uniform size in [bmin, bmax] whose arrivals form a Poisson
    process carrying `rate_qps` queries per second on average; queries are
    drawn from `pool`."""
    rng = np.random.default_rng(seed)
    mean_b = (bmin + bmax) / 2.0
    t, rid, out = 0.0, 0, []
    while True:
        t += rng.exponential(mean_b / rate_qps)
        if t > duration_s:
            break
        b = int(rng.integers(bmin, bmax + 1))
        sel = rng.integers(0, pool.shape[0], size=b)
        out.append(Request(rid, t, pool[sel]))
        rid += 1
    return out


def run_open_loop(server: Server, requests, clock=time.perf_counter, max_wall_s: float = 600.0):
    """Replays `requests` at their arrival times (open loop: arrivals never
    wait for completions) and serves them; returns the wall seconds."""
    t0 = clock()
    now = lambda: clock() - t0  # noqa: E731
    i = 0
    reqs = sorted(requests, key=lambda r: r.arrival)
    while i < len(reqs) or not server.idle():
        t = now()
        while i < len(reqs) and reqs[i].arrival <= t:
            server.submit(reqs[i])
            i += 1
        server.poll(now)
        if t > max_wall_s:
            raise TimeoutError("serving did not finish in time")
    return now()


def latency_summary(requests):
    """Latency percentiles of the answered requests (shed ones have none)."""
    lat = np.array([r.latency for r in requests if r.latency is not None]) * 1e3
    if lat.size == 0:
        return {"p50_ms": None, "p99_ms": None, "mean_ms": None, "max_ms": None, "n": 0}
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()), "n": int(len(lat))}


class GpuEngine:
    """Launches one batch through fs_recommend on a slot's stream, with every
    transient buffer inside the server's device arena; results come back to
    pinned host memory."""

    def __init__(self, fs, db, f: int, k: int, slots: int, max_batch: int, arena_bytes: int,
                 l_max: int = 128, device=None):
        import torch
        self.torch, self.fs, self.db = torch, fs, db
        self.f, self.k, self.l_max = f, k, l_max
        self.device = device or torch.device("cuda")
        self.arena_buf = torch.empty(arena_bytes, dtype=torch.uint8, device=self.device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        pin = lambda shape, dt: torch.empty(shape, dtype=dt).pin_memory()  # noqa: E731
        self.h_q = [pin((max_batch, f), torch.float32) for _ in range(slots)]
        self.h_idx = [pin((max_batch, k), torch.int32) for _ in range(slots)]
        self.h_dist = [pin((max_batch, k), torch.float32) for _ in range(slots)]
        self.h_seq = [pin((max_batch, k, l_max), torch.int16) for _ in range(slots)]
        self.h_len = [pin((max_batch, k), torch.int32) for _ in range(slots)]

    def _parts(self, nq):
        k, f, l_max = self.k, self.f, self.l_max
        return [("q", nq * f * 4), ("idx", nq * k * 4), ("dist", nq * k * 4),
                ("seq", nq * k * l_max * 2), ("len", nq * k * 4),
                ("ws", self.fs.fs_workspace_size(self.db, nq))]

    def batch_bytes(self, nq: int) -> int:
        return sum(_round_up(b) for _, b in self._parts(nq))

    def launch(self, queries: np.ndarray, offset: int, slot: int):
        torch, fs = self.torch, self.fs
        nq = queries.shape[0]
        views, off = {}, offset
        for name, nbytes in self._parts(nq):
            views[name] = self.arena_buf[off:off + nbytes]
            off += _round_up(nbytes)
        qd = views["q"].view(torch.float32).view(nq, self.f)
        idx = views["idx"].view(torch.int32).view(nq, self.k)
        dist = views["dist"].view(torch.float32).view(nq, self.k)
        seq = views["seq"].view(torch.int16).view(nq, self.k, self.l_max)
        ln = views["len"].view(torch.int32).view(nq, self.k)
        s = self.streams[slot]
        hq = self.h_q[slot][:nq]
        hq.copy_(torch.from_numpy(queries))
        with torch.cuda.stream(s):
            qd.copy_(hq, non_blocking=True)
            fs.fs_recommend(self.db, qd, self.k, workspace=views["ws"], idx=idx, dist=dist,
                            seq_out=seq, seq_len=ln, l_max=self.l_max, stream=s)
            self.h_idx[slot][:nq].copy_(idx, non_blocking=True)
            self.h_dist[slot][:nq].copy_(dist, non_blocking=True)
            self.h_seq[slot][:nq].copy_(seq, non_blocking=True)
            self.h_len[slot][:nq].copy_(ln, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        return (ev, slot, nq)

    def done(self, handle) -> bool:
        return handle[0].query()

    def results(self, handle):
        _, slot, nq = handle
        return (self.h_idx[slot][:nq].numpy(), self.h_dist[slot][:nq].numpy(),
                self.h_seq[slot][:nq].numpy(), self.h_len[slot][:nq].numpy())
