"""Continuous-batching triangle-count server over the C ABI.

Requests name a graph (any hashable key); a `source(key)` callable returns its
host CSR. The server keeps prepared graphs resident -- the cache entry is the
handle that bbtc_graph_create built (the oriented CSR) together with the plan
that bbtc_graph_plan built on it (blocks, tasks, work items) -- and admits a
graph into device memory only while the cache stays under a byte budget
(evicting unreferenced entries, least recently used first). `workers` worker
threads run, each on its own CUDA stream. A worker that frees up takes every
request that has arrived (up to `max_batch`), prepares the graphs that are not
cached, and counts the whole batch with one bbtc_count_batch call: one
persistent launch over the work items of all the batch's graphs, each read
from its own cached plan. Requests that arrive while batches are on the GPU
wait for the next free worker, so batches overlap on the device and new work
is admitted as slots and memory free up.

Counts are exact integers: a request's result does not depend on which batch
it rode in.
"""
from __future__ import annotations

import collections
import math
import threading
import time

import numpy as np

from . import (Graph, bbtc_count_batch, bbtc_graph_create_async, bbtc_graph_destroy,
               bbtc_graph_get_info, bbtc_graph_plan, make_opts)


class Request:
    __slots__ = ("rid", "key", "arrival", "start", "finish", "count", "status", "batch_size")

    def __init__(self, rid, key, arrival):
        self.rid, self.key, self.arrival = rid, key, arrival
        self.start = self.finish = None
        self.count = None
        self.status = None
        self.batch_size = 0


class _Entry:
    __slots__ = ("handle", "bytes", "refs", "ready")

    def __init__(self):
        self.handle = 0
        self.bytes = 0
        self.refs = 0
        # set once the handle and its plan exist; from then on batch counts
        # only read them, so workers on different streams may share the entry
        self.ready = threading.Event()


class Server:
    def __init__(self, source, device_budget_bytes: int, max_batch: int = 256,
                 workers: int = 2, p: int = 0, kernel: str = "auto", symmetric: bool = False):
        import torch
        self.torch = torch
        self.source = source
        self.budget = int(device_budget_bytes)
        self.max_batch = max_batch
        self.n_workers = workers
        self.p, self.kernel, self.symmetric = p, kernel, symmetric
        self.queue: collections.deque[Request] = collections.deque()
        self.cv = threading.Condition()
        self.cache: collections.OrderedDict = collections.OrderedDict()
        self.cache_bytes = 0
        self.stop = False
        self.done: list[Request] = []
        self.hits = self.misses = self.evictions = 0
        self.errors: list[str] = []
        self.streams = [torch.cuda.Stream() for _ in range(workers)]
        self.threads = [threading.Thread(target=self._worker, args=(i,), daemon=True)
                        for i in range(workers)]
        for t in self.threads:
            t.start()

    # ------------------------------------------------------------ cache
    @staticmethod
    def _estimate_bytes(n, nnz):
        # oriented CSR (rowptr, colidx, esrc, perm, degree) and the plan
        # (block columns, in-edges, row pointers), from the input size
        m = nnz // 2 + 1
        return 28 * n + 24 * m

    def _acquire(self, key, stream):
        """Cache entry for key (creating the graph if missing); holds a reference."""
        with self.cv:
            ent = self.cache.get(key)
            if ent is not None:
                ent.refs += 1
                self.cache.move_to_end(key)
                self.hits += 1
                creator = False
            else:
                ent = _Entry()
                ent.refs = 1
                self.cache[key] = ent
                self.misses += 1
                creator = True
        if not creator:
            ent.ready.wait()
            if not ent.handle:
                raise RuntimeError(f"graph {key!r} could not be prepared")
            return ent
        try:
            return self._create(key, ent, stream)
        except BaseException:
            with self.cv:
                self.cache.pop(key, None)
                self.cache_bytes -= ent.bytes
            ent.ready.set()  # waiters see handle == 0 and fail
            raise

    def _create(self, key, ent, stream):
        n, rowptr, colidx = self.source(key)
        need = self._estimate_bytes(n, int(rowptr[n]))
        with self.cv:
            # admission: evict unreferenced entries until the new graph fits
            while self.cache_bytes + need > self.budget:
                victim = next((k for k, e in self.cache.items()
                               if e.refs == 0 and e.ready.is_set()), None)
                if victim is None:
                    break
                e = self.cache.pop(victim)
                self.cache_bytes -= e.bytes
                self.evictions += 1
                bbtc_graph_destroy(e.handle)
            self.cache_bytes += need
        ent.bytes = need
        flags = 0x2 if self.symmetric else 0
        ent.handle = bbtc_graph_create_async(n, rowptr, colidx, flags, stream)
        bbtc_graph_plan(ent.handle, make_opts(p=self.p, kernel=self.kernel, stream=stream))
        actual = int(bbtc_graph_get_info(ent.handle)["device_bytes"])
        with self.cv:
            self.cache_bytes += actual - need
            ent.bytes = actual
        ent.ready.set()
        return ent

    def _note_error(self, exc):
        with self.cv:
            if len(self.errors) < 16:
                self.errors.append(f"{type(exc).__name__}: {exc}")

    def _release(self, key):
        with self.cv:
            ent = self.cache.get(key)
            if ent is not None:
                ent.refs -= 1

    # ---------------------------------------------------------- workers
    def _worker(self, wi):
        stream = self.streams[wi]
        torch = self.torch
        while True:
            with self.cv:
                while not self.queue and not self.stop:
                    self.cv.wait()
                if not self.queue and self.stop:
                    return
                batch = [self.queue.popleft()
                         for _ in range(min(self.max_batch, len(self.queue)))]
            t0 = time.perf_counter()
            for r in batch:
                r.start = t0
            acquired = []
            try:
                with torch.cuda.stream(stream):
                    handles = []
                    for r in batch:
                        # a graph that cannot be prepared fails its own request only:
                        # its slot goes to the batch count as NULL, which the library
                        # reports per graph while it counts the others
                        try:
                            handles.append(self._acquire(r.key, stream).handle)
                            acquired.append(r.key)
                        except Exception as exc:
                            self._note_error(exc)
                            handles.append(None)
                    opts = make_opts(p=self.p, kernel=self.kernel, stream=stream)
                    counts, stats = bbtc_count_batch(handles, opts)
            except Exception as exc:  # the count failed: the batch fails, the server keeps running
                self._note_error(exc)
                counts = np.zeros(len(batch), dtype=np.uint64)
                stats = np.full(len(batch), 6, dtype=np.int32)
            t1 = time.perf_counter()
            for r, c, s in zip(batch, counts, stats):
                r.count, r.status, r.finish, r.batch_size = int(c), int(s), t1, len(batch)
            for k in acquired:
                self._release(k)
            with self.cv:
                self.done.extend(batch)
                self.cv.notify_all()

    # ------------------------------------------------------------- API
    def submit(self, req: Request):
        with self.cv:
            self.queue.append(req)
            self.cv.notify()

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
