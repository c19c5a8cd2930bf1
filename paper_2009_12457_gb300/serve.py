"""Continuous-batching triangle-count server over the C ABI.

Requests name a graph (any hashable key); a `source(key)` callable returns its
host CSR. The server keeps prepared graphs resident: a cache entry is the
handle that bbtc_graph_create built (the oriented CSR) together with the plan
that bbtc_graph_plan built on it (blocks, tasks, work items).

Three kinds of threads share the device, each on its own CUDA stream:

* the submitting thread only queues: a request whose graph is cached goes
  straight to the ready queue, one whose graph is missing (or still being
  prepared) waits beside its cache entry;
* a preparation worker takes missing graphs in arrival order, admits each by
  free device memory (`bbtc_device_memory`: the driver's free bytes plus the
  library pool's unused bytes, minus a reserve; and, when a byte budget is
  set, by the cache's size), evicting unreferenced cache entries least
  recently used first, then creates and plans it. A graph that does not fit
  waits until references drop or the admission timeout passes, and then fails
  its own requests only. Its requests move to the ready queue once it is ready
  (or has failed);
* `workers` batch workers: a worker that frees up takes every ready request
  (up to `max_batch`) and counts the whole batch with one bbtc_count_batch
  call -- one persistent launch over the work items of all the batch's
  graphs, each read from its own cached plan. A request whose graph failed
  rides as a NULL handle, which the library reports per graph.

So a cache miss never stalls a batch of cached graphs, requests that arrive
while batches are on the GPU are admitted as slots and memory free up, and
batches of different workers overlap on the device.

Counts are exact integers: a request's result does not depend on which batch
it rode in.
"""
from __future__ import annotations

import collections
import threading
import time

import numpy as np

from . import (Graph, bbtc_count_batch, bbtc_device_memory, bbtc_graph_create_async,
               bbtc_graph_destroy, bbtc_graph_get_info, bbtc_graph_plan, make_opts)


class Request:
    __slots__ = ("rid", "key", "arrival", "start", "finish", "count", "status", "batch_size")

    def __init__(self, rid, key, arrival):
        self.rid, self.key, self.arrival = rid, key, arrival
        self.start = self.finish = None
        self.count = None
        self.status = None
        self.batch_size = 0


class _Entry:
    __slots__ = ("handle", "bytes", "refs", "state", "waiting")
    PREPARING, READY, FAILED = 0, 1, 2

    def __init__(self):
        self.handle = 0
        self.bytes = 0
        self.refs = 0              # requests queued or in a batch that read the handle
        self.state = _Entry.PREPARING
        self.waiting: list[Request] = []  # requests that arrived while preparing


class Server:
    def __init__(self, source, device_budget_bytes: int | None = None, max_batch: int = 256,
                 workers: int = 2, p: int = 0, kernel: str = "auto", symmetric: bool = False,
                 reserve_bytes: int = 4 << 30, admit_timeout_s: float = 30.0,
                 device: int | None = None):
        import torch
        self.torch = torch
        self.device = torch.cuda.current_device() if device is None else device
        self.source = source
        self.budget = None if device_budget_bytes is None else int(device_budget_bytes)
        self.reserve = int(reserve_bytes)
        self.admit_timeout = admit_timeout_s
        self.max_batch = max_batch
        self.p, self.kernel, self.symmetric = p, kernel, symmetric
        self.ready: collections.deque = collections.deque()   # (request, entry)
        self.prep: collections.deque = collections.deque()    # keys to prepare
        self.cv = threading.Condition()
        self.cache: collections.OrderedDict = collections.OrderedDict()
        self.cache_bytes = 0
        self.stop = False
        self.done: list[Request] = []
        self.hits = self.misses = self.evictions = self.admission_waits = 0
        self.errors: list[str] = []
        self.streams = [torch.cuda.Stream() for _ in range(workers)]
        self.prep_stream = torch.cuda.Stream()
        self.threads = [threading.Thread(target=self._worker, args=(i,), daemon=True)
                        for i in range(workers)]
        self.threads.append(threading.Thread(target=self._preparer, daemon=True))
        for t in self.threads:
            t.start()

    # ------------------------------------------------------------ cache
    @staticmethod
    def _estimate_bytes(n, nnz):
        # oriented CSR (rowptr, colidx, esrc, perm, degree), the plan (16-byte
        # in-edge records, split table, tasks) and the preparation's temporaries,
        # from the input size
        m = nnz // 2 + 1
        return 44 * n + 48 * m

    def _available(self):
        return bbtc_device_memory(self.device)["available"] - self.reserve

    def _fits(self, need):
        if self.budget is not None and self.cache_bytes + need > self.budget:
            return False
        return need <= self._available()

    def _evict_one(self):
        """Destroys the least recently used unreferenced ready entry (cv held)."""
        victim = next((k for k, e in self.cache.items()
                       if e.refs == 0 and e.state == _Entry.READY), None)
        if victim is None:
            return False
        e = self.cache.pop(victim)
        self.cache_bytes -= e.bytes
        self.evictions += 1
        bbtc_graph_destroy(e.handle)
        return True

    def _note_error(self, exc):
        with self.cv:
            if len(self.errors) < 16:
                self.errors.append(f"{type(exc).__name__}: {exc}")

    # ------------------------------------------------------- preparation
    def _preparer(self):
        torch = self.torch
        torch.cuda.set_device(self.device)
        while True:
            with self.cv:
                while not self.prep and not self.stop:
                    self.cv.wait()
                if self.stop:
                    return
                key = self.prep.popleft()
                ent = self.cache[key]
            try:
                n, rowptr, colidx = self.source(key)
                need = self._estimate_bytes(n, int(rowptr[n]))
                deadline = time.perf_counter() + self.admit_timeout
                with self.cv:
                    # admission: evict unreferenced entries least recently used
                    # first until the graph fits; while referenced entries hold
                    # the memory it needs, wait for their references to drop
                    waited = False
                    while not self._fits(need):
                        evictable = sum(e.bytes for e in self.cache.values()
                                        if e.refs == 0 and e.state == _Entry.READY)
                        held = any(e.refs > 0 for e in self.cache.values())
                        room = self._available() + evictable
                        if self.budget is not None:
                            room = min(room, self.budget - (self.cache_bytes - evictable))
                        if need <= room and self._evict_one():
                            continue
                        remaining = deadline - time.perf_counter()
                        if not held or remaining <= 0 or self.stop:
                            raise MemoryError(f"graph {key!r} ({need} bytes) does not fit in "
                                              "free device memory")
                        waited = True
                        self.cv.wait(timeout=min(remaining, 0.05))
                    if waited:
                        self.admission_waits += 1
                    self.cache_bytes += need
                    ent.bytes = need
                flags = 0x2 if self.symmetric else 0
                handle = bbtc_graph_create_async(n, rowptr, colidx, flags, self.prep_stream)
                try:
                    bbtc_graph_plan(handle, make_opts(p=self.p, kernel=self.kernel,
                                                      stream=self.prep_stream))
                    actual = int(bbtc_graph_get_info(handle)["device_bytes"])
                except BaseException:
                    bbtc_graph_destroy(handle)
                    raise
                with self.cv:
                    self.cache_bytes += actual - ent.bytes
                    ent.bytes, ent.handle, ent.state = actual, handle, _Entry.READY
                    self._release_waiting(ent)
            except Exception as exc:  # the graph fails its own requests only
                self._note_error(exc)
                with self.cv:
                    self.cache.pop(key, None)
                    self.cache_bytes -= ent.bytes
                    ent.bytes, ent.state = 0, _Entry.FAILED
                    self._release_waiting(ent)

    def _release_waiting(self, ent):
        """Moves the requests that waited for ent to the ready queue (cv held)."""
        for r in ent.waiting:
            ent.refs += 1
            self.ready.append((r, ent))
        ent.waiting = []
        self.cv.notify_all()

    # ---------------------------------------------------------- workers
    def _worker(self, wi):
        stream = self.streams[wi]
        torch = self.torch
        torch.cuda.set_device(self.device)
        while True:
            with self.cv:
                while not self.ready and not self.stop:
                    self.cv.wait()
                if not self.ready and self.stop:
                    return
                batch = [self.ready.popleft()
                         for _ in range(min(self.max_batch, len(self.ready)))]
            t0 = time.perf_counter()
            for r, _ in batch:
                r.start = t0
            handles = [e.handle if e.state == _Entry.READY else None for _, e in batch]
            try:
                with torch.cuda.stream(stream):
                    opts = make_opts(p=self.p, kernel=self.kernel, stream=stream)
                    counts, stats = bbtc_count_batch(handles, opts)
            except Exception as exc:  # the count failed: the batch fails, the server keeps running
                self._note_error(exc)
                counts = np.zeros(len(batch), dtype=np.uint64)
                stats = np.full(len(batch), 6, dtype=np.int32)
            t1 = time.perf_counter()
            for (r, _), c, s in zip(batch, counts, stats):
                r.count, r.status, r.finish, r.batch_size = int(c), int(s), t1, len(batch)
            with self.cv:
                for _, e in batch:
                    if e.state == _Entry.READY:
                        e.refs -= 1
                self.done.extend(r for r, _ in batch)
                self.cv.notify_all()

    # ------------------------------------------------------------- API
    def submit(self, req: Request):
        with self.cv:
            ent = self.cache.get(req.key)
            if ent is not None:
                self.hits += 1
                self.cache.move_to_end(req.key)
                if ent.state == _Entry.READY:
                    ent.refs += 1
                    self.ready.append((req, ent))
                else:
                    ent.waiting.append(req)
            else:
                self.misses += 1
                ent = _Entry()
                ent.waiting.append(req)
                self.cache[req.key] = ent
                self.prep.append(req.key)
            self.cv.notify_all()

    def drain(self, total: int, timeout_s: float = 600.0):
        deadline = time.perf_counter() + timeout_s
        with self.cv:
            while len(self.done) < total and time.perf_counter() < deadline:
                self.cv.wait(timeout=0.5)
        return list(self.done)

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        for t in self.threads:
            t.join()
        for ent in self.cache.values():
            if ent.handle:
                bbtc_graph_destroy(ent.handle)
        self.cache.clear()


def poisson_trace(rate_hz: float, duration_s: float, seed: int):
    """Arrival times (s) of a Poisson process, from a seeded generator."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            return np.array(out)
        out.append(t)


def run_open_loop(server: Server, keys, arrivals):
    """Submit request i with key keys[i] at arrivals[i] seconds; wait for all."""
    t0 = time.perf_counter()
    reqs = []
    for i, (k, a) in enumerate(zip(keys, arrivals)):
        now = time.perf_counter() - t0
        if a > now:
            time.sleep(a - now)
        r = Request(i, k, t0 + a)
        reqs.append(r)
        server.submit(r)
    server.drain(len(reqs))
    return reqs


def latency_summary(reqs):
    lat = np.array([r.finish - r.arrival for r in reqs if r.finish is not None])
    span = max(r.finish for r in reqs) - min(r.arrival for r in reqs)
    return {"requests": len(reqs), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "graphs_per_s": len(reqs) / span,
            "mean_batch": float(np.mean([r.batch_size for r in reqs]))}


def serial_baseline(source, keys, symmetric: bool = False, p: int = 0):
    """One plain create + count + destroy per request, back to back (no cache, no batch)."""
    counts = []
    t0 = time.perf_counter()
    for k in keys:
        n, rp, ci = source(k)
        g = Graph(n, rp, ci, symmetric=symmetric)
        counts.append(g.count(p=p))
        g.close()
    dt = time.perf_counter() - t0
    return counts, len(keys) / dt


def serial_cached_baseline(source, keys, symmetric: bool = False, p: int = 0):
    """One bbtc_count per request, back to back, on handles prepared and planned
    beforehand (the cache without the batching): isolates what batching adds."""
    handles = {}
    try:
        for k in dict.fromkeys(keys):
            n, rp, ci = source(k)
            g = Graph(n, rp, ci, symmetric=symmetric)
            g.count(p=p)  # builds and caches the plan
            handles[k] = g
        counts = []
        t0 = time.perf_counter()
        for k in keys:
            counts.append(handles[k].count(p=p))
        dt = time.perf_counter() - t0
    finally:
        for g in handles.values():
            g.close()
    return counts, len(keys) / dt
