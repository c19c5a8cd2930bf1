"""Autotuner for the counting step's free parameters.

bbTC leaves three choices open: the number of blocks per side p (Sec. 7.3
suggests p near the average degree for a CPU; on one GPU with the graph
resident the best p is smaller), the per-task kernel (the isDense choice of
Alg. 7, here a threshold on the mean staged-list length), and how much of a
task one warp takes at a time (in-edges per work item). None of them changes
a count; they change only time.

The tuner measures the counting kernel with the library's CUDA-event timings
(bbtc_graph_get_timings) on a handle, searches the choices one at a time
(p, then kernel/threshold, then chunk), and caches the winner per graph-size
class in a JSON file so later graphs of the same class reuse it.
"""
from __future__ import annotations

import json
import math
import os
import threading

from . import Graph, bbtc_count, bbtc_graph_get_info, bbtc_graph_get_timings, make_opts

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build",
                             "autotune.json")

P_CHOICES = (1, 2, 4, 8, 16)
KERNEL_CHOICES = (("intersect", 0), ("hashmap", 0), ("auto", 8), ("auto", 32))
CHUNK_CHOICES = (0, 256, 1024, 4096)


def size_class(info: dict) -> str:
    """Graphs whose edge count and average degree round to the same powers of two."""
    m = max(int(info["m"]), 1)
    n = max(int(info["n"]), 1)
    return f"m2^{round(math.log2(m))}_d2^{round(math.log2(max(2.0 * m / n, 1.0)))}"


class Autotuner:
    def __init__(self, cache_path: str | None = DEFAULT_CACHE, repeats: int = 2):
        self.cache_path = cache_path
        self.repeats = repeats
        self._lock = threading.Lock()
        self.cache: dict[str, dict] = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.cache = json.load(f)

    def _save(self):
        if not self.cache_path:
            return
        os.makedirs(os.path.dirname(self.cache_path), exist_ok=True)
        tmp = f"{self.cache_path}.{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(self.cache, f, indent=1, sort_keys=True)
        os.replace(tmp, self.cache_path)

    def measure(self, handle: int, cfg: dict) -> float:
        """Best counting-kernel time (ms) of `repeats` runs with cfg (plan built first)."""
        opts = make_opts(p=cfg["p"], kernel=cfg["kernel"], hash_threshold=cfg["hash_threshold"],
                         chunk=cfg["chunk"])
        bbtc_count(handle, opts)  # builds the plan for cfg
        best = float("inf")
        for _ in range(self.repeats):
            bbtc_count(handle, opts)
            best = min(best, bbtc_graph_get_timings(handle)["count_ms"])
        return best

    def tune(self, graph, p_choices=P_CHOICES) -> dict:
        """Search p, then kernel/threshold, then chunk on this graph; cache the winner."""
        handle = graph.handle if isinstance(graph, Graph) else int(graph)
        info = bbtc_graph_get_info(handle)
        cfg = {"p": 1, "kernel": "hashmap", "hash_threshold": 0, "chunk": 0}
        trials = []

        def run(c):
            ms = self.measure(handle, c)
            trials.append((dict(c), ms))
            return ms

        best_ms = float("inf")
        for p in p_choices:
            c = dict(cfg, p=p)
            ms = run(c)
            if ms < best_ms:
                best_ms, cfg = ms, c
        for kernel, thr in KERNEL_CHOICES:
            c = dict(cfg, kernel=kernel, hash_threshold=thr)
            if c == cfg:
                continue
            ms = run(c)
            if ms < best_ms:
                best_ms, cfg = ms, c
        for chunk in CHUNK_CHOICES:
            c = dict(cfg, chunk=chunk)
            if c == cfg:
                continue
            ms = run(c)
            if ms < best_ms:
                best_ms, cfg = ms, c
        result = dict(cfg, count_ms=best_ms, size_class=size_class(info), trials=len(trials))
        with self._lock:
            self.cache[size_class(info)] = result
            self._save()
        return result

    def choice(self, graph, tune_if_missing: bool = True) -> dict:
        """The cached choice for the graph's size class (tuning it first if allowed)."""
        handle = graph.handle if isinstance(graph, Graph) else int(graph)
        key = size_class(bbtc_graph_get_info(handle))
        with self._lock:
            hit = self.cache.get(key)
        if hit is not None:
            return hit
        if not tune_if_missing:
            return {"p": 0, "kernel": "auto", "hash_threshold": 0, "chunk": 0}
        return self.tune(graph)

    @staticmethod
    def opts(choice: dict, **extra):
        return make_opts(p=choice["p"], kernel=choice["kernel"],
                         hash_threshold=choice["hash_threshold"], chunk=choice["chunk"], **extra)
