"""Seeded synthetic graph inputs shared by the CUDA library's tests/benchmark and the oracle.

This module draws graphs; it performs no step of triangle counting. Every
generator returns ``(n, rowptr, colidx)``: a symmetrised CSR (int64 rowptr of
n+1 entries, int32 colidx) in which each drawn pair (a, b) is listed under both
endpoints, duplicates and self-loops kept exactly as drawn. Removing them is the
first step of the counting method itself.

Randomness is SplitMix64 used as a counter-based generator (see graphgen.c), so
a graph depends only on its parameters and seed, never on the thread count.

Workload recipes (synthetic stand-ins for the paper's datasets):

* ``rmat(scale, edge_factor, seed)`` -- R-MAT with (a, b, c, d) = (.57, .19, .19, .05),
  ``edge_factor * 2**scale`` pairs, no noise, no relabelling.
* ``gnm(n, pairs, seed)`` -- Erdos-Renyi G(n, m) drawn with replacement.
* ``chunglu(n, gamma, wmax, weight_sum, pairs, seed)`` -- Chung-Lu expected degree
  graph, weights ``min(wmax, C (i+1)^(-1/(gamma-1)))`` summing to ``weight_sum``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libgraphgen.so")
_lib = None
_lock = threading.Lock()

RMAT_ABC = (0.57, 0.19, 0.19)


def build(force: bool = False) -> str:
    """Compile graphgen.c into a shared library (gcc, OpenMP). Returns its path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = f"{_LIB_PATH}.{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                    "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        lib.gg_draw.argtypes = [u64, u64, u64]
        lib.gg_draw.restype = u64
        lib.gg_rmat_pairs.argtypes = [i32, i64, f64, f64, f64, u64, P, P]
        lib.gg_gnm_pairs.argtypes = [i64, i64, u64, P, P]
        lib.gg_chunglu_weights.argtypes = [i64, f64, f64, f64, P]
        lib.gg_chunglu_weights.restype = f64
        lib.gg_alias_build.argtypes = [i64, P, P, P]
        lib.gg_chunglu_pairs.argtypes = [i64, i64, P, P, u64, P, P]
        lib.gg_pairs_to_csr.argtypes = [i64, i64, P, P, P, P]
        lib.gg_num_threads.restype = ctypes.c_int
        lib.gg_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
        return lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def draw(seed: int, stream: int, index: int) -> int:
    """The counter-based 64-bit draw (seed, stream, index)."""
    return int(_load().gg_draw(seed, stream, index))


def pairs_to_csr(n: int, src: np.ndarray, dst: np.ndarray):
    """Symmetrised CSR of the pairs (src[e], dst[e]); duplicates/self-loops kept."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    assert src.shape == dst.shape
    M = src.shape[0]
    rowptr = np.empty(n + 1, dtype=np.int64)
    colidx = np.empty(2 * M, dtype=np.int32)
    _load().gg_pairs_to_csr(n, M, _ptr(src), _ptr(dst), _ptr(rowptr), _ptr(colidx))
    return n, rowptr, colidx


def rmat_pairs(scale: int, edge_factor: int, seed: int, abc=RMAT_ABC):
    M = edge_factor * (1 << scale)
    src = np.empty(M, dtype=np.int32)
    dst = np.empty(M, dtype=np.int32)
    a, b, c = abc
    _load().gg_rmat_pairs(scale, M, a, b, c, seed, _ptr(src), _ptr(dst))
    return 1 << scale, src, dst


def rmat(scale: int, edge_factor: int, seed: int, abc=RMAT_ABC):
    n, src, dst = rmat_pairs(scale, edge_factor, seed, abc)
    return pairs_to_csr(n, src, dst)


def gnm_pairs(n: int, pairs: int, seed: int):
    src = np.empty(pairs, dtype=np.int32)
    dst = np.empty(pairs, dtype=np.int32)
    _load().gg_gnm_pairs(n, pairs, seed, _ptr(src), _ptr(dst))
    return n, src, dst


def gnm(n: int, pairs: int, seed: int):
    return pairs_to_csr(*gnm_pairs(n, pairs, seed))


def chunglu_pairs(n: int, gamma: float, wmax: float, weight_sum: float, pairs: int, seed: int):
    lib = _load()
    w = np.empty(n, dtype=np.float64)
    lib.gg_chunglu_weights(n, gamma, wmax, weight_sum, _ptr(w))
    prob = np.empty(n, dtype=np.uint32)
    alias = np.empty(n, dtype=np.int32)
    lib.gg_alias_build(n, _ptr(w), _ptr(prob), _ptr(alias))
    del w
    src = np.empty(pairs, dtype=np.int32)
    dst = np.empty(pairs, dtype=np.int32)
    lib.gg_chunglu_pairs(n, pairs, _ptr(prob), _ptr(alias), seed, _ptr(src), _ptr(dst))
    return n, src, dst


def chunglu(n: int, gamma: float, wmax: float, weight_sum: float, pairs: int, seed: int):
    return pairs_to_csr(*chunglu_pairs(n, gamma, wmax, weight_sum, pairs, seed))


def num_threads() -> int:
    return int(_load().gg_num_threads())


# ---------------------------------------------------------------------------
# Named workloads (sizes of the benchmark and parity configurations)
# ---------------------------------------------------------------------------

def rmat_s14():
    """R-MAT scale 14, edge factor 16, seed 1 (16,384 vertices, 262,144 pairs)."""
    return rmat(14, 16, 1)


def rmat_s23():
    """R-MAT scale 23, edge factor 16, seed 2 (8.4M vertices, 134M pairs)."""
    return rmat(23, 16, 2)


FRIENDSTER_N = 65_608_366
FRIENDSTER_M = 1_806_067_135


def chunglu_friendster(scale_down: int = 1):
    """Friendster-shaped Chung-Lu graph: gamma 2.1, weights capped at 5,000, seed 3.

    ``scale_down`` > 1 divides n and the pair count (same exponent and cap) for
    smaller stand-ins of the same shape.
    """
    n = FRIENDSTER_N // scale_down
    pairs = FRIENDSTER_M // scale_down
    return chunglu(n, 2.1, 5000.0, 2.0 * pairs, pairs, 3)


def batch_spec(g: int):
    """Parameters of graph g (0..4095) of the batched workload, from seed 100+g.

    Target pair count m log-uniform in [1e3, 2e6]. Even g: G(n,m) with average
    degree uniform in [8, 64], n = ceil(2m/deg). Odd g: R-MAT (a=.57) with edge
    factor uniform in [8, 32] and scale = round(log2(m/ef)).
    """
    seed = 100 + g
    u0 = (draw(seed, 7, 0) >> 11) * (1.0 / (1 << 53))
    u1 = (draw(seed, 7, 1) >> 11) * (1.0 / (1 << 53))
    m = int(round(math.exp(math.log(1e3) + u0 * (math.log(2e6) - math.log(1e3)))))
    if g % 2 == 0:
        deg = 8.0 + 56.0 * u1
        n = max(2, int(math.ceil(2.0 * m / deg)))
        return {"kind": "gnm", "n": n, "pairs": m, "seed": seed}
    ef = 8 + int(u1 * 25) if u1 < 1.0 else 32
    scale = max(1, int(round(math.log2(max(m / ef, 2.0)))))
    return {"kind": "rmat", "scale": scale, "edge_factor": ef, "seed": seed}


def batch_graph(g: int):
    s = batch_spec(g)
    if s["kind"] == "gnm":
        return gnm(s["n"], s["pairs"], s["seed"])
    return rmat(s["scale"], s["edge_factor"], s["seed"])


def batch_graphs(count: int = 4096, workers: int | None = None):
    """The batched workload's graphs 0..count-1 (see batch_spec), generated by a
    pool of host threads with one OpenMP thread each (the result does not depend
    on either)."""
    import concurrent.futures
    workers = workers or max(1, os.cpu_count() or 1)
    lib = _load()

    def one(g):
        lib.gg_set_threads(1)
        return batch_graph(g)

    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        return list(ex.map(one, range(count)))
