"""TEST INFRASTRUCTURE ONLY: the CPU oracle for block-based triangle counting.

A plain, slow, single-threaded restatement (bbtc_oracle.c) of what the CUDA
library computes, following the paper's steps in order: canonical simple edge
set (Sec. 2), degree and non-decreasing degree order (Sec. 4.1), orientation
u < v (Sec. 2), contiguous partition into p parts (Sec. 2, Sec. 4.1; balanced on
edges, or probe-based to bound the largest block, Sec. 4.4), task
composition (Alg. 4), task estimate and order (Sec. 5), per-task counting with
bbTC-Intersect (Alg. 5) or bbTC-HMap (Alg. 6), and the whole-graph counts of
Alg. 2 / Alg. 3.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package. It shares no code with the CUDA library.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bbtc_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libbbtc_oracle.so")
_lib = None
_lock = threading.Lock()


def compile_source(src: str, out: str) -> str:
    """Compile one oracle C source into a shared library at ``out``."""
    tmp = f"{out}.{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, src],
                   check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle (plain gcc -O2, no OpenMP). Returns the library path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    return compile_source(_SRC, _LIB_PATH)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
        return _lib


@contextlib.contextmanager
def using_library(path: str):
    """Temporarily route every oracle call to another build of bbtc_oracle.c.

    Used by the pin tests to check that deliberately broken copies of the
    oracle fail them.
    """
    global _lib
    saved = _load()
    _lib = _declare(ctypes.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


def _declare(lib):
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    u64 = ctypes.c_uint64
    lib.orc_canonical_edges.argtypes = [i64, P, P, P]
    lib.orc_canonical_edges.restype = i64
    lib.orc_degree.argtypes = [i64, i64, P, P]
    lib.orc_order_by_degree.argtypes = [i64, P, P, P]
    lib.orc_orient.argtypes = [i64, i64, P, P, P, P]
    lib.orc_n_intersect.argtypes = [P, i64, P, i64]
    lib.orc_n_intersect.restype = u64
    lib.orc_tc_intersect.argtypes = [i64, P, P]
    lib.orc_tc_intersect.restype = u64
    lib.orc_tc_hmap.argtypes = [i64, P, P]
    lib.orc_tc_hmap.restype = u64
    lib.orc_per_vertex.argtypes = [i64, P, P, P, P]
    lib.orc_edge_support.argtypes = [i64, P, P, P]
    lib.orc_cuts.argtypes = [i64, P, i32, P]
    lib.orc_block_nnz.argtypes = [i64, P, P, i32, P, P]
    lib.orc_pbd_grains.argtypes = [i32]
    lib.orc_pbd_grains.restype = i32
    lib.orc_pbd_grain_bounds.argtypes = [i64, P, P, i32, P]
    lib.orc_pbd_prefix.argtypes = [i64, P, P, i32, P, P]
    lib.orc_pbd_load.argtypes = [i32, P, i32, i32, i32, i32]
    lib.orc_pbd_load.restype = i64
    lib.orc_pbd_probe.argtypes = [i32, P, i32, i64, P]
    lib.orc_pbd_probe.restype = i32
    lib.orc_pbd_cuts.argtypes = [i64, P, P, i32, P]
    lib.orc_pbd_cuts.restype = i64
    lib.orc_num_tasks.argtypes = [i32]
    lib.orc_num_tasks.restype = i64
    lib.orc_task_list.argtypes = [i32, P, P, P]
    lib.orc_task_list.restype = i64
    lib.orc_exec_time.argtypes = [i32, P, P, P]
    lib.orc_order_tasks.argtypes = [i64, P, P]
    lib.orc_bbtc_intersect_task.argtypes = [i64, P, P, P, i32, i32, i32]
    lib.orc_bbtc_intersect_task.restype = u64
    lib.orc_bbtc_hmap_task.argtypes = [i64, P, P, P, i32, i32, i32]
    lib.orc_bbtc_hmap_task.restype = u64
    lib.orc_classify_triangles.argtypes = [i64, P, P, i32, P, P]
    lib.orc_work_figures.argtypes = [i64, P, P, P, P, P]
    lib.orc_vertex_triangles.argtypes = [i64, P, P, i64]
    lib.orc_vertex_triangles.restype = u64
    return lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ------------------------------------------------------------------- steps

def canonical_edges(n: int, rowptr, colidx, compact: bool = True) -> np.ndarray:
    """Sorted unique keys (a << 32) | b, a < b, of the simple undirected edge set.

    compact=False returns a view into the rowptr[n]-entry work buffer instead of
    a copy of its first m entries (the caller then decides when to copy, e.g.
    after freeing the input of a graph too large to hold twice).
    """
    rowptr, colidx = _c(rowptr, np.int64), _c(colidx, np.int32)
    keys = np.empty(max(int(rowptr[n]), 1), dtype=np.uint64)
    m = _load().orc_canonical_edges(n, _p(rowptr), _p(colidx), _p(keys))
    return keys[:m].copy() if compact else keys[:m]


def degree(n: int, keys) -> np.ndarray:
    keys = _c(keys, np.uint64)
    deg = np.empty(max(n, 1), dtype=np.int64)
    _load().orc_degree(n, keys.shape[0], _p(keys), _p(deg))
    return deg[:n]


def order_by_degree(n: int, deg):
    """(rank, perm): rank[v] = position of v in (degree, id) order; perm = inverse."""
    deg = _c(deg, np.int64)
    rank = np.empty(max(n, 1), dtype=np.int32)
    perm = np.empty(max(n, 1), dtype=np.int32)
    _load().orc_order_by_degree(n, _p(deg), _p(rank), _p(perm))
    return rank[:n], perm[:n]


def orient(n: int, keys, rank):
    """Oriented CSR (rowptr int64[n+1], colidx int32[m]) in degree-order positions."""
    keys, rank = _c(keys, np.uint64), _c(rank, np.int32)
    m = keys.shape[0]
    rp = np.empty(n + 1, dtype=np.int64)
    ci = np.empty(max(m, 1), dtype=np.int32)
    _load().orc_orient(n, m, _p(keys), _p(rank), _p(rp), _p(ci))
    return rp, ci[:m]


def n_intersect(A, B) -> int:
    """Alg. 1: number of common elements of two sorted lists."""
    A, B = _c(A, np.int32), _c(B, np.int32)
    return int(_load().orc_n_intersect(_p(A), A.shape[0], _p(B), B.shape[0]))


def tc_intersect(n: int, rp, ci) -> int:
    """Alg. 2 over an oriented CSR."""
    rp, ci = _c(rp, np.int64), _c(ci, np.int32)
    return int(_load().orc_tc_intersect(n, _p(rp), _p(ci)))


def tc_hmap(n: int, rp, ci) -> int:
    """Alg. 3 over an oriented CSR."""
    rp, ci = _c(rp, np.int64), _c(ci, np.int32)
    return int(_load().orc_tc_hmap(n, _p(rp), _p(ci)))


def per_vertex(n: int, rp, ci, perm) -> np.ndarray:
    """Triangles at each vertex, in original ids."""
    rp, ci, perm = _c(rp, np.int64), _c(ci, np.int32), _c(perm, np.int32)
    out = np.empty(max(n, 1), dtype=np.uint64)
    _load().orc_per_vertex(n, _p(rp), _p(ci), _p(perm), _p(out))
    return out[:n]


def edge_support(n: int, rp, ci) -> np.ndarray:
    """Triangles containing each oriented edge, by oriented-CSR position."""
    rp = _c(rp, np.int64)
    ci = _c(ci, np.int32)
    out = np.zeros(max(int(rp[n]), 1), dtype=np.uint32)
    _load().orc_edge_support(n, _p(rp), _p(ci), _p(out))
    return out[:int(rp[n])]


def cuts(n: int, rp, p: int) -> np.ndarray:
    rp = _c(rp, np.int64)
    c = np.empty(p + 1, dtype=np.int32)
    _load().orc_cuts(n, _p(rp), p, _p(c))
    return c


def pbd_grains(p: int) -> int:
    """Number of grains G of the probe-based partition for p parts."""
    return int(_load().orc_pbd_grains(p))


def pbd_grain_bounds(n: int, rp, ci, G: int) -> np.ndarray:
    """Grain boundaries b[0..G], balanced on undirected degree."""
    rp, ci = _c(rp, np.int64), _c(ci, np.int32)
    b = np.empty(G + 1, dtype=np.int32)
    _load().orc_pbd_grain_bounds(n, _p(rp), _p(ci), G, _p(b))
    return b


def pbd_prefix(n: int, rp, ci, G: int, b) -> np.ndarray:
    """(G+1) x (G+1) int64 table: S[r][c] = edges from grains [0,r) into grains [0,c)."""
    rp, ci, b = _c(rp, np.int64), _c(ci, np.int32), _c(b, np.int32)
    S = np.empty((G + 1) * (G + 1), dtype=np.int64)
    _load().orc_pbd_prefix(n, _p(rp), _p(ci), G, _p(b), _p(S))
    return S.reshape(G + 1, G + 1)


def pbd_load(S, r0: int, r1: int, c0: int, c1: int) -> int:
    """Edges from grains [r0, r1) into grains [c0, c1), through the oracle's table."""
    S = _c(S, np.int64)
    return int(_load().orc_pbd_load(S.shape[0] - 1, _p(S), r0, r1, c0, c1))


def pbd_probe(S, p: int, B: int):
    """Probe(B): (passed, grain cuts x[0..p])."""
    S = _c(S, np.int64)
    x = np.zeros(p + 1, dtype=np.int32)
    ok = _load().orc_pbd_probe(S.shape[0] - 1, _p(S), p, B, _p(x))
    return bool(ok), x


def pbd_cuts(n: int, rp, ci, p: int):
    """(cuts c[0..p], B*) of the probe-based symmetric partition."""
    rp, ci = _c(rp, np.int64), _c(ci, np.int32)
    c = np.empty(p + 1, dtype=np.int32)
    bstar = _load().orc_pbd_cuts(n, _p(rp), _p(ci), p, _p(c))
    return c, int(bstar)


def block_nnz(n: int, rp, ci, p: int, c) -> np.ndarray:
    """|G_ij| as a p x p int64 array (row-major)."""
    rp, ci, c = _c(rp, np.int64), _c(ci, np.int32), _c(c, np.int32)
    out = np.empty(p * p, dtype=np.int64)
    _load().orc_block_nnz(n, _p(rp), _p(ci), p, _p(c), _p(out))
    return out.reshape(p, p)


def num_tasks(p: int) -> int:
    return int(_load().orc_num_tasks(p))


def task_list(p: int) -> np.ndarray:
    """Alg. 4: (|T|, 3) int32 array of (i, j, k)."""
    nt = num_tasks(p)
    ti = np.empty(max(nt, 1), dtype=np.int32)
    tj = np.empty(max(nt, 1), dtype=np.int32)
    tk = np.empty(max(nt, 1), dtype=np.int32)
    _load().orc_task_list(p, _p(ti), _p(tj), _p(tk))
    return np.stack([ti[:nt], tj[:nt], tk[:nt]], axis=1)


def exec_time(p: int, c, nnz) -> np.ndarray:
    """Sec. 5 ExecTime of each task, in Alg. 4 order (float64)."""
    c, nnz = _c(c, np.int32), _c(nnz, np.int64).reshape(-1)
    est = np.empty(max(num_tasks(p), 1), dtype=np.float64)
    _load().orc_exec_time(p, _p(c), _p(nnz), _p(est))
    return est[:num_tasks(p)]


def order_tasks(est) -> np.ndarray:
    est = _c(est, np.float64)
    order = np.empty(max(est.shape[0], 1), dtype=np.int32)
    _load().orc_order_tasks(est.shape[0], _p(est), _p(order))
    return order[:est.shape[0]]


def bbtc_task(n: int, rp, ci, c, i: int, j: int, k: int, method: str = "intersect") -> int:
    """Alg. 5 (method='intersect') or Alg. 6 (method='hmap') for task (i,j,k)."""
    rp, ci, c = _c(rp, np.int64), _c(ci, np.int32), _c(c, np.int32)
    fn = _load().orc_bbtc_intersect_task if method == "intersect" else _load().orc_bbtc_hmap_task
    return int(fn(n, _p(rp), _p(ci), _p(c), i, j, k))


def classify_triangles(n: int, rp, ci, p: int, c) -> np.ndarray:
    """Per-task counts from classifying every triangle into its task."""
    rp, ci, c = _c(rp, np.int64), _c(ci, np.int32), _c(c, np.int32)
    out = np.empty(max(num_tasks(p), 1), dtype=np.uint64)
    _load().orc_classify_triangles(n, _p(rp), _p(ci), p, _p(c), _p(out))
    return out[:num_tasks(p)]


def work_figures(n: int, rp, ci) -> dict:
    """Algorithmic bytes of the counting step: wmin, wmerge (bytes), wedges (count)."""
    rp, ci = _c(rp, np.int64), _c(ci, np.int32)
    a = np.zeros(3, dtype=np.uint64)
    _load().orc_work_figures(n, _p(rp), _p(ci), _p(a[0:]), _p(a[1:]), _p(a[2:]))
    return {"wmin": int(a[0]), "wmerge": int(a[1]), "wedges": int(a[2])}


def vertex_triangles(n: int, rowptr, colidx, x: int) -> int:
    """Triangles containing original vertex x, from a symmetric input CSR."""
    rowptr, colidx = _c(rowptr, np.int64), _c(colidx, np.int32)
    return int(_load().orc_vertex_triangles(n, _p(rowptr), _p(colidx), x))


# ---------------------------------------------------------- full pipeline

def prepare(n: int, rowptr, colidx) -> dict:
    """Canonical edges -> degree -> order -> oriented CSR (Sec. 2, Sec. 4.1)."""
    keys = canonical_edges(n, rowptr, colidx)
    deg = degree(n, keys)
    rank, perm = order_by_degree(n, deg)
    rp, ci = orient(n, keys, rank)
    return {"n": n, "m": int(keys.shape[0]), "keys": keys, "deg": deg, "rank": rank,
            "perm": perm, "rowptr": rp, "colidx": ci}


def bbtc(n: int, rowptr, colidx, p: int = 1, method: str = "intersect",
         prep: dict | None = None, want_per_vertex: bool = False,
         partition: str = "edges") -> dict:
    """The whole bbTC pipeline in the paper's order, sequentially.

    partition: "edges" (contiguous parts balanced on oriented edges) or "probe"
    (the probe-based partition that bounds the largest block).
    Returns the oriented CSR, cuts, block sizes, task list, estimates and order,
    per-task counts (Alg. 5 or Alg. 6, one task at a time in the estimate's
    order), the total, and optionally per-vertex counts.
    """
    pr = prep if prep is not None else prepare(n, rowptr, colidx)
    rp, ci = pr["rowptr"], pr["colidx"]
    c = cuts(n, rp, p) if partition == "edges" else pbd_cuts(n, rp, ci, p)[0]  # "probe"
    nnz = block_nnz(n, rp, ci, p, c)
    tasks = task_list(p)
    est = exec_time(p, c, nnz)
    order = order_tasks(est)
    per_task = np.zeros(tasks.shape[0], dtype=np.uint64)
    for t in order:
        i, j, k = (int(x) for x in tasks[t])
        per_task[t] = bbtc_task(n, rp, ci, c, i, j, k, method)
    out = dict(pr)
    out.update({"p": p, "cuts": c, "block_nnz": nnz, "tasks": tasks, "exec_time": est,
                "order": order, "per_task": per_task, "total": int(per_task.sum())})
    if want_per_vertex:
        out["per_vertex"] = per_vertex(n, rp, ci, pr["perm"])
    return out
