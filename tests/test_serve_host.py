"""Host logic of the serving loop on the CPU: admission under the byte budget and
by available device memory, eviction of unreferenced graphs least recently used
first, cache hits, preparation off the batch path, and per-request failure
isolation. The library calls and CUDA streams are replaced by fakes, so no GPU
is needed."""
import contextlib
import time

import numpy as np
import pytest

import paper_2009_12457_gb300 as bb
from paper_2009_12457_gb300 import serve


class FakeLib:
    """Stands in for the C ABI: a handle is an int; a graph's count is its n."""

    def __init__(self, sizes):
        self.sizes = sizes          # key -> device bytes reported for the handle
        self.next = 1
        self.by_handle = {}
        self.destroyed = []
        self.created = []
        self.live = {}

    def create(self, n, rowptr, colidx, flags, stream):
        if int(colidx.max(initial=-1)) >= n:
            raise bb.BbtcError(1, "colidx entry outside [0, n)")
        h = self.next
        self.next += 1
        self.by_handle[h] = n
        self.live[h] = self.sizes[n]
        self.created.append(n)
        return h

    def plan(self, handle, opts):
        pass

    def info(self, handle):
        return {"device_bytes": self.sizes[self.by_handle[handle]]}

    def count_batch(self, handles, opts):
        counts = np.array([self.by_handle[h] if h else 0 for h in handles], dtype=np.uint64)
        stats = np.array([0 if h else 1 for h in handles], dtype=np.int32)
        return counts, stats

    def destroy(self, handle):
        self.destroyed.append(self.by_handle[handle])
        self.live.pop(handle, None)

    capacity = 1 << 40  # device bytes; the live handles hold their sizes of it

    def memory(self, device=0):
        return {"available": self.capacity - sum(self.live.values()), "total": self.capacity,
                "pool_reserved": 0, "pool_used": 0}


@pytest.fixture
def fake(monkeypatch):
    import torch
    monkeypatch.setattr(torch.cuda, "Stream", lambda: object())
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    # each handle reports the server's own admission estimate for an edgeless
    # graph of n vertices: 44 n + 48 bytes
    lib = FakeLib({n: 44 * n + 48 for n in range(1, 64)})
    monkeypatch.setattr(serve, "bbtc_device_memory", lib.memory)
    monkeypatch.setattr(serve, "bbtc_graph_create_async", lib.create)
    monkeypatch.setattr(serve, "bbtc_graph_plan", lib.plan)
    monkeypatch.setattr(serve, "bbtc_graph_get_info", lib.info)
    monkeypatch.setattr(serve, "bbtc_count_batch", lib.count_batch)
    monkeypatch.setattr(serve, "bbtc_graph_destroy", lib.destroy)
    monkeypatch.setattr(serve, "make_opts", lambda **kw: None)
    return lib


SLOW_S = 0.5


def source(key):
    """Graph `key` (an int n, "bad", or ("slow", n)): n vertices and no edges;
    "bad" has an out-of-range column; ("slow", n) takes SLOW_S to load."""
    if key == "bad":
        return 2, np.array([0, 1, 1], dtype=np.int64), np.array([5], dtype=np.int32)
    if isinstance(key, tuple):
        time.sleep(SLOW_S)
        key = key[1]
    return key, np.zeros(key + 1, dtype=np.int64), np.zeros(0, dtype=np.int32)


def serve_in_order(srv, keys, start=0):
    """Submit the keys one request at a time, each after the previous finished."""
    out = []
    for i, k in enumerate(keys):
        r = serve.Request(start + i, k, time.perf_counter())
        srv.submit(r)
        srv.drain(start + i + 1, timeout_s=10)
        out.append(r)
    return out


def test_cache_hits_and_lru_eviction(fake):
    # graphs 3, 4, 5 take 180, 224 and 268 bytes; a 500-byte budget holds two
    srv = serve.Server(source, device_budget_bytes=500, workers=1)
    try:
        reqs = serve_in_order(srv, [3, 4, 3, 5, 3])
        evicted = list(fake.destroyed)
        cached = sorted(srv.cache)
    finally:
        srv.close()
    assert [r.count for r in reqs] == [3, 4, 3, 5, 3]
    assert all(r.status == 0 for r in reqs)
    # 3 was used again after 4, so admitting 5 evicts 4, and 3 is still cached
    assert evicted == [4] and srv.evictions == 1 and cached == [3, 5]
    assert srv.hits == 2 and srv.misses == 3
    assert fake.created == [3, 4, 5]
    assert sorted(fake.destroyed[1:]) == [3, 5]  # closing frees what is cached


def test_a_failed_graph_fails_only_its_requests(fake):
    srv = serve.Server(source, device_budget_bytes=1 << 20, max_batch=64, workers=1)
    keys = [3, "bad", 4, 5, "bad", 3]
    try:
        reqs = [serve.Request(i, k, time.perf_counter()) for i, k in enumerate(keys)]
        with srv.cv:  # one burst: the worker takes it as one batch
            for r in reqs:
                srv.submit(r)
        srv.drain(len(reqs), timeout_s=10)
        later = serve_in_order(srv, [4], start=len(reqs))
    finally:
        srv.close()
    assert [r.status for r in reqs] == [0, 1, 0, 0, 1, 0]
    assert [r.count for r in reqs if r.key != "bad"] == [3, 4, 5, 3]
    # "bad" was prepared once for both of its requests, and failed once
    assert len(srv.errors) == 1 and "outside" in srv.errors[0]
    assert later[0].status == 0 and later[0].count == 4
    assert "bad" not in srv.cache  # a failed entry does not stay cached


def test_a_miss_does_not_delay_cached_graphs(fake):
    """A graph that takes long to load is prepared off the batch path: requests on
    cached graphs that arrive after it finish before it does."""
    srv = serve.Server(source, device_budget_bytes=1 << 20, max_batch=64, workers=1)
    try:
        serve_in_order(srv, [3, 4])                       # 3 and 4 are now cached
        t0 = time.perf_counter()
        slow = serve.Request(2, ("slow", 5), t0)
        srv.submit(slow)
        fast = [serve.Request(3 + i, k, time.perf_counter()) for i, k in enumerate([3, 4, 3])]
        for r in fast:
            srv.submit(r)
        srv.drain(6, timeout_s=10)
    finally:
        srv.close()
    assert slow.status == 0 and slow.count == 5
    assert [r.count for r in fast] == [3, 4, 3]
    assert max(r.finish for r in fast) < slow.finish
    assert max(r.finish for r in fast) - t0 < SLOW_S / 2


def test_admission_by_available_device_memory(fake):
    """A graph larger than the available device memory (after the reserve) fails its
    own requests once nothing can be evicted; the others are served, and an
    unreferenced cached graph is evicted to make room for one that fits."""
    fake.capacity = 600
    srv = serve.Server(source, device_budget_bytes=None, reserve_bytes=100, workers=1,
                       admit_timeout_s=0.2)
    try:
        first = serve_in_order(srv, [3])                  # 180 bytes cached
        big = serve_in_order(srv, [20], start=1)          # 928 bytes: never fits
        cached_after_big = sorted(srv.cache)
        fake.capacity = 450                               # 170 bytes left after the reserve
        mid = serve_in_order(srv, [4], start=2)           # 224 bytes: evicts 3
    finally:
        srv.close()
    assert first[0].status == 0 and first[0].count == 3
    assert big[0].status != 0 and any("does not fit" in e for e in srv.errors)
    assert cached_after_big == [3]                        # nothing evicted in vain
    assert mid[0].status == 0 and mid[0].count == 4
    assert fake.destroyed[0] == 3 and srv.evictions == 1
