"""Python binding of libbbtc, the block-based triangle counting library (sm_103a).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels behind the C ABI of ``include/bbtc.h``. The functions carry the C
names (``bbtc_graph_create``, ``bbtc_count``, ...); ``Graph`` wraps a handle.

Arrays may be numpy arrays (host) or CUDA tensors (device; any object with
``data_ptr()`` and ``is_cuda``). There is no CPU fallback: if the library
cannot be built or loaded, importing the binding's functions raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

__all__ = [
    "BbtcError", "Graph", "bbtc_graph_create", "bbtc_graph_create_async", "bbtc_count",
    "bbtc_count_batch", "bbtc_graph_plan", "bbtc_graph_destroy", "bbtc_last_error", "bbtc_num_tasks",
    "bbtc_opts_init", "bbtc_graph_get_info", "bbtc_graph_get_oriented", "bbtc_graph_get_plan",
    "bbtc_graph_get_timings", "bbtc_kernel_launches", "bbtc_count_noalloc",
    "bbtc_graph_create_batch", "bbtc_count_async", "bbtc_device_memory", "BatchGraph",
    "library_path", "load",
]

STATUS = {0: "BBTC_OK", 1: "BBTC_EINVAL", 2: "BBTC_ENOMEM", 3: "BBTC_ECUDA",
          4: "BBTC_ETIMEOUT", 5: "BBTC_ECANCELLED", 6: "BBTC_EINTERNAL"}
KERNELS = {"auto": 0, "intersect": 1, "hashmap": 2}
PARTITIONS = {"edges": 0, "probe": 1}

INPUT_DEVICE = 0x1
INPUT_SYMMETRIC = 0x2
OUT_DEVICE = 0x1


class BbtcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class bbtc_opts(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("p", ctypes.c_int32),
        ("kernel", ctypes.c_int32),
        ("timeout_ms", ctypes.c_uint32),
        ("device_budget_bytes", ctypes.c_uint64),
        ("per_vertex_out", ctypes.c_void_p),
        ("per_task_out", ctypes.c_void_p),
        ("stream", ctypes.c_void_p),
        ("flags", ctypes.c_uint32),
        ("hash_threshold", ctypes.c_int32),
        ("per_graph_out", ctypes.c_void_p),
        ("chunk", ctypes.c_int32),
        ("partition", ctypes.c_int32),
        ("per_task_cycles_out", ctypes.c_void_p),
        ("per_edge_out", ctypes.c_void_p),
        ("task_mask", ctypes.c_void_p),
    ]


class bbtc_graph_info(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("m", ctypes.c_int64),
        ("dplus_max", ctypes.c_int64),
        ("deg_max", ctypes.c_int64),
        ("device_bytes", ctypes.c_uint64),
        ("wedges_in", ctypes.c_uint64),
        ("wedges_out", ctypes.c_uint64),
        ("num_graphs", ctypes.c_int64),
    ]


class bbtc_timings(ctypes.Structure):
    _fields_ = [
        ("prep_ms", ctypes.c_double),
        ("plan_ms", ctypes.c_double),
        ("count_ms", ctypes.c_double),
        ("work_items", ctypes.c_int64),
        ("stream_rounds", ctypes.c_int64),
        ("stream_h2d_bytes", ctypes.c_uint64),
        ("stream_copy_ms", ctypes.c_double),
        ("stream_block_bytes", ctypes.c_uint64),
        ("stream_device_peak_bytes", ctypes.c_uint64),
        ("stream_mode", ctypes.c_int32),
    ]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB_PATH


def load():
    """Load libbbtc (building it from csrc/ first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        lib = ctypes.CDLL(path)
        P, i32, i64, u32, u64 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                 ctypes.c_uint32, ctypes.c_uint64)
        st = ctypes.c_int
        lib.bbtc_opts_init.argtypes = [ctypes.POINTER(bbtc_opts)]
        lib.bbtc_opts_init.restype = None
        lib.bbtc_graph_create.argtypes = [i64, P, P, u32, ctypes.POINTER(P)]
        lib.bbtc_graph_create.restype = st
        lib.bbtc_graph_create_async.argtypes = [i64, P, P, u32, P, ctypes.POINTER(P)]
        lib.bbtc_graph_create_async.restype = st
        lib.bbtc_count.argtypes = [P, ctypes.POINTER(bbtc_opts), ctypes.POINTER(u64)]
        lib.bbtc_count.restype = st
        lib.bbtc_count_batch.argtypes = [P, i32, ctypes.POINTER(bbtc_opts), P, P]
        lib.bbtc_count_batch.restype = st
        lib.bbtc_graph_plan.argtypes = [P, ctypes.POINTER(bbtc_opts)]
        lib.bbtc_graph_plan.restype = st
        lib.bbtc_graph_destroy.argtypes = [P]
        lib.bbtc_graph_destroy.restype = None
        lib.bbtc_last_error.argtypes = []
        lib.bbtc_last_error.restype = ctypes.c_char_p
        lib.bbtc_num_tasks.argtypes = [i32]
        lib.bbtc_num_tasks.restype = u64
        lib.bbtc_graph_get_info.argtypes = [P, ctypes.POINTER(bbtc_graph_info)]
        lib.bbtc_graph_get_info.restype = st
        lib.bbtc_graph_get_oriented.argtypes = [P, P, P, P, P]
        lib.bbtc_graph_get_oriented.restype = st
        lib.bbtc_graph_get_plan.argtypes = [P, i32, P, P, P, P, P]
        lib.bbtc_graph_get_plan.restype = st
        lib.bbtc_graph_get_timings.argtypes = [P, ctypes.POINTER(bbtc_timings)]
        lib.bbtc_graph_get_timings.restype = st
        lib.bbtc_kernel_launches.argtypes = []
        lib.bbtc_kernel_launches.restype = u64
        lib.bbtc_count_noalloc.argtypes = [P, i32, P, P, P]
        lib.bbtc_count_noalloc.restype = st
        lib.bbtc_graph_create_batch.argtypes = [i32, P, P, P, u32, P, ctypes.POINTER(P)]
        lib.bbtc_graph_create_batch.restype = st
        lib.bbtc_count_async.argtypes = [P, ctypes.POINTER(bbtc_opts), P]
        lib.bbtc_count_async.restype = st
        lib.bbtc_device_memory.argtypes = [i32, P, P, P, P]
        lib.bbtc_device_memory.restype = st
        _lib = lib
        return lib


def _check(status: int):
    if status != 0:
        raise BbtcError(status, load().bbtc_last_error().decode(errors="replace"))


def _ptr(a) -> tuple[int, bool]:
    """(address, is_device) of a numpy array or a CUDA tensor-like object."""
    if a is None:
        return 0, False
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        return int(a.data_ptr()), bool(a.is_cuda)
    if isinstance(a, np.ndarray):
        return int(a.ctypes.data), False
    raise TypeError(f"unsupported array type {type(a)!r}")


def _stream_ptr(stream) -> int:
    if stream is None:
        return 0
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


# ------------------------------------------------------------ C-named calls

def bbtc_opts_init() -> bbtc_opts:
    o = bbtc_opts()
    load().bbtc_opts_init(ctypes.byref(o))
    return o


def bbtc_num_tasks(p: int) -> int:
    return int(load().bbtc_num_tasks(p))


def bbtc_last_error() -> str:
    return load().bbtc_last_error().decode(errors="replace")


def bbtc_graph_create_async(n: int, rowptr, colidx, flags: int = 0, stream=None) -> int:
    """Create a handle from a CSR. Host numpy arrays, or CUDA tensors (sets INPUT_DEVICE)."""
    rp, rp_dev = _ptr(rowptr)
    ci, ci_dev = _ptr(colidx)
    if rp_dev or ci_dev:
        if not (rp_dev and (ci_dev or ci == 0)):
            raise ValueError("rowptr and colidx must both be host or both be device arrays")
        flags |= INPUT_DEVICE
    else:
        if isinstance(rowptr, np.ndarray) and (rowptr.dtype != np.int64 or not rowptr.flags.c_contiguous):
            raise TypeError("rowptr must be a contiguous int64 array")
        if isinstance(colidx, np.ndarray) and (colidx.dtype != np.int32 or not colidx.flags.c_contiguous):
            raise TypeError("colidx must be a contiguous int32 array")
    h = ctypes.c_void_p()
    _check(load().bbtc_graph_create_async(n, rp or None, ci or None, flags,
                                          _stream_ptr(stream) or None, ctypes.byref(h)))
    return h.value


def bbtc_graph_create(n: int, rowptr, colidx, flags: int = 0) -> int:
    return bbtc_graph_create_async(n, rowptr, colidx, flags, None)


def bbtc_graph_destroy(handle: int) -> None:
    if handle:
        load().bbtc_graph_destroy(handle)


def make_opts(p: int = 0, kernel: str | int = "auto", timeout_ms: int = 0,
              device_budget_bytes: int = 0, per_vertex_out=None, per_task_out=None,
              stream=None, hash_threshold: int = 0, per_graph_out=None,
              chunk: int = 0, per_task_cycles_out=None, per_edge_out=None,
              partition: str | int = "edges", task_mask=None) -> bbtc_opts:
    o = bbtc_opts_init()
    o.partition = PARTITIONS[partition] if isinstance(partition, str) else int(partition)
    o.p = p
    o.kernel = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    o.timeout_ms = timeout_ms
    o.device_budget_bytes = device_budget_bytes
    o.hash_threshold = hash_threshold
    o.chunk = chunk
    outs = [(_ptr(a), a is not None)
            for a in (per_vertex_out, per_task_out, per_graph_out, per_task_cycles_out,
                      per_edge_out)]
    kinds = {dev for (addr, dev), given in outs if given}
    if len(kinds) > 1:
        raise ValueError("optional outputs must all be host arrays or all device arrays")
    o.per_vertex_out = outs[0][0][0] or None
    o.per_task_out = outs[1][0][0] or None
    o.per_graph_out = outs[2][0][0] or None
    o.per_task_cycles_out = outs[3][0][0] or None
    o.per_edge_out = outs[4][0][0] or None
    o.flags = OUT_DEVICE if kinds == {True} else 0
    o.stream = _stream_ptr(stream) or None
    if task_mask is not None:  # host bytes, one per task in Alg. 4 order
        task_mask = np.ascontiguousarray(task_mask, dtype=np.uint8)
        o.task_mask = task_mask.ctypes.data
    # the struct holds raw pointers: keep the output arrays (and the stream) alive
    # for as long as the options are, so a temporary passed here is not freed
    # before the library writes into it
    o._keep = (per_vertex_out, per_task_out, per_graph_out, per_task_cycles_out,
               per_edge_out, stream, task_mask)
    return o


def bbtc_count(handle: int, opts: bbtc_opts | None = None) -> int:
    c = ctypes.c_uint64()
    _check(load().bbtc_count(handle, ctypes.byref(opts) if opts is not None else None,
                             ctypes.byref(c)))
    return int(c.value)


def bbtc_graph_create_batch(vertex_offsets, rowptr, colidx, flags: int = 0, stream=None) -> int:
    """One handle for a batch: vertex_offsets (host int64, ng+1), union rowptr, LOCAL colidx."""
    voff = np.ascontiguousarray(vertex_offsets, dtype=np.int64)
    ng = voff.shape[0] - 1
    rp, rp_dev = _ptr(rowptr)
    ci, ci_dev = _ptr(colidx)
    if rp_dev or ci_dev:
        flags |= INPUT_DEVICE
    h = ctypes.c_void_p()
    _check(load().bbtc_graph_create_batch(ng, voff.ctypes.data, rp or None, ci or None, flags,
                                          _stream_ptr(stream) or None, ctypes.byref(h)))
    return h.value


def bbtc_count_async(handle: int, opts: bbtc_opts, total_dev) -> None:
    """Enqueue a count into device buffers (no allocation, no wait; capturable)."""
    t, t_dev = _ptr(total_dev)
    if not t_dev:
        raise ValueError("bbtc_count_async writes device buffers only")
    _check(load().bbtc_count_async(handle, ctypes.byref(opts), t))


def bbtc_count_noalloc(handle: int, p: int, count_dev, per_task_dev=None, stream=None) -> None:
    """Allocation-free count into device buffers (see include/bbtc.h)."""
    c, c_dev = _ptr(count_dev)
    t, t_dev = _ptr(per_task_dev)
    if not c_dev or (per_task_dev is not None and not t_dev):
        raise ValueError("bbtc_count_noalloc writes device buffers only")
    _check(load().bbtc_count_noalloc(handle, p, c, t or None, _stream_ptr(stream) or None))


def bbtc_graph_plan(handle: int, opts: bbtc_opts | None = None) -> None:
    """Build (or keep) the handle's resident plan for the options, without counting."""
    _check(load().bbtc_graph_plan(handle, ctypes.byref(opts) if opts is not None else None))


def bbtc_count_batch(handles, opts: bbtc_opts | None = None):
    """Counts of several handles; returns (counts uint64 array, statuses int32 array)."""
    ng = len(handles)
    arr = (ctypes.c_void_p * max(ng, 1))(*handles)
    counts = np.zeros(max(ng, 1), dtype=np.uint64)
    stats = np.zeros(max(ng, 1), dtype=np.int32)
    st = load().bbtc_count_batch(arr, ng, ctypes.byref(opts) if opts is not None else None,
                                 counts.ctypes.data, stats.ctypes.data)
    if st != 0 and not np.any(stats[:ng] != 0):
        _check(st)
    return counts[:ng], stats[:ng]


def bbtc_graph_get_info(handle: int) -> dict:
    info = bbtc_graph_info()
    _check(load().bbtc_graph_get_info(handle, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in bbtc_graph_info._fields_}


def bbtc_graph_get_oriented(handle: int) -> dict:
    info = bbtc_graph_get_info(handle)
    n, m = info["n"], info["m"]
    rowptr = np.empty(n + 1, dtype=np.int64)
    colidx = np.empty(max(m, 1), dtype=np.int32)
    perm = np.empty(max(n, 1), dtype=np.int32)
    degree = np.empty(max(n, 1), dtype=np.int64)
    _check(load().bbtc_graph_get_oriented(handle, rowptr.ctypes.data, colidx.ctypes.data,
                                          perm.ctypes.data, degree.ctypes.data))
    return {"rowptr": rowptr, "colidx": colidx[:m], "perm": perm[:n], "degree": degree[:n]}


def bbtc_graph_get_plan(handle: int, p: int) -> dict:
    nt = bbtc_num_tasks(p)
    cuts = np.empty(p + 1, dtype=np.int32)
    nnz = np.empty(p * p, dtype=np.int64)
    tasks = np.empty(3 * nt, dtype=np.int32)
    est = np.empty(nt, dtype=np.float64)
    order = np.empty(nt, dtype=np.int32)
    _check(load().bbtc_graph_get_plan(handle, p, cuts.ctypes.data, nnz.ctypes.data,
                                      tasks.ctypes.data, est.ctypes.data, order.ctypes.data))
    return {"cuts": cuts, "block_nnz": nnz.reshape(p, p), "tasks": tasks.reshape(nt, 3),
            "exec_time": est, "order": order}


def bbtc_graph_get_timings(handle: int) -> dict:
    t = bbtc_timings()
    _check(load().bbtc_graph_get_timings(handle, ctypes.byref(t)))
    return {f: getattr(t, f) for f, _ in bbtc_timings._fields_}


def bbtc_kernel_launches() -> int:
    return int(load().bbtc_kernel_launches())


def bbtc_device_memory(device: int = 0) -> dict:
    """Device memory the library can still use on `device` (driver free bytes plus
    the unused part of its stream-ordered pool), with the total and the pool's
    reserved and used bytes."""
    out = np.zeros(4, dtype=np.uint64)
    p = out.ctypes.data
    _check(load().bbtc_device_memory(device, p, p + 8, p + 16, p + 24))
    return {"available": int(out[0]), "total": int(out[1]), "pool_reserved": int(out[2]),
            "pool_used": int(out[3])}


# ------------------------------------------------------------- convenience

class Graph:
    """A bbTC graph handle: the device-resident oriented CSR of one graph."""

    def __init__(self, n: int, rowptr, colidx, symmetric: bool = False, stream=None):
        flags = INPUT_SYMMETRIC if symmetric else 0
        self.handle = bbtc_graph_create_async(n, rowptr, colidx, flags, stream)
        self.n = n

    def count(self, p: int = 0, kernel: str = "auto", per_vertex: bool = False,
              per_task: bool = False, timeout_ms: int = 0, device_budget_bytes: int = 0,
              stream=None, hash_threshold: int = 0, per_graph: bool = False, chunk: int = 0,
              per_task_cycles: bool = False, per_edge: bool = False,
              partition: str = "edges"):
        """Total triangle count, or a dict with per-task / per-vertex / per-graph counts
        (with per_task_cycles, the SM cycles spent on each task; with per_edge, the
        support of each oriented edge in the order of get_oriented()'s colidx)."""
        pt = np.zeros(max(bbtc_num_tasks(p), 1), dtype=np.uint64) if per_task and p > 0 else None
        if per_task and p == 0:
            raise ValueError("per_task needs an explicit p")
        pv = np.zeros(max(self.n, 1), dtype=np.uint64) if per_vertex else None
        ng = self.info()["num_graphs"] if per_graph else 0
        pg = np.zeros(max(ng, 1), dtype=np.uint64) if per_graph else None
        if per_task_cycles and p == 0:
            raise ValueError("per_task_cycles needs an explicit p")
        cyc = np.zeros(max(bbtc_num_tasks(p), 1), dtype=np.uint64) if per_task_cycles else None
        m = self.info()["m"] if per_edge else 0
        pe = np.zeros(max(m, 1), dtype=np.uint32) if per_edge else None
        opts = make_opts(p, kernel, timeout_ms, device_budget_bytes, pv, pt, stream,
                         hash_threshold, pg, chunk, cyc, pe, partition)
        total = bbtc_count(self.handle, opts)
        if not (per_task or per_vertex or per_graph or per_task_cycles or per_edge):
            return total
        out = {"total": total}
        if per_task:
            out["per_task"] = pt[:bbtc_num_tasks(p)]
        if per_vertex:
            out["per_vertex"] = pv[:self.n]
        if per_graph:
            out["per_graph"] = pg[:ng]
        if per_task_cycles:
            out["per_task_cycles"] = cyc[:bbtc_num_tasks(p)]
        if per_edge:
            out["per_edge"] = pe[:m]
        return out

    def info(self) -> dict:
        return bbtc_graph_get_info(self.handle)

    def edge_support(self, p: int = 0, kernel: str = "auto"):
        """Support of every edge (the number of triangles containing it, the input of
        k-truss): arrays (u, v, support) with u, v original vertex ids."""
        sup = self.count(p=p, kernel=kernel, per_edge=True)["per_edge"]
        o = self.oriented()
        src = np.repeat(np.arange(len(o["perm"]), dtype=np.int64), np.diff(o["rowptr"]))
        return o["perm"][src], o["perm"][o["colidx"]], sup

    def oriented(self) -> dict:
        return bbtc_graph_get_oriented(self.handle)

    def plan(self, p: int, partition: str | None = None) -> dict:
        """The plan for p: the handle's current one for p, or first built with
        `partition` when given."""
        if partition is not None:
            bbtc_graph_plan(self.handle, make_opts(p=p, partition=partition))
        return bbtc_graph_get_plan(self.handle, p)

    def timings(self) -> dict:
        return bbtc_graph_get_timings(self.handle)

    def close(self):
        if self.handle:
            bbtc_graph_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_csr(graphs):
    """Concatenate [(n, rowptr, colidx), ...] into (vertex_offsets, rowptr, colidx) with
    colidx left local to each graph (the form bbtc_graph_create_batch takes)."""
    ns = [int(g[0]) for g in graphs]
    voff = np.zeros(len(graphs) + 1, dtype=np.int64)
    voff[1:] = np.cumsum(ns)
    nnz = [int(g[1][g[0]]) for g in graphs]
    eoff = np.zeros(len(graphs) + 1, dtype=np.int64)
    eoff[1:] = np.cumsum(nnz)
    rowptr = np.empty(int(voff[-1]) + 1, dtype=np.int64)
    colidx = np.empty(int(eoff[-1]), dtype=np.int32)
    for i, (n, rp, ci) in enumerate(graphs):
        rowptr[voff[i]:voff[i] + n] = np.asarray(rp[:n], dtype=np.int64) + eoff[i]
        colidx[eoff[i]:eoff[i + 1]] = ci[:nnz[i]]
    rowptr[-1] = eoff[-1]
    return voff, rowptr, colidx


class BatchGraph(Graph):
    """A batch handle: several independent graphs prepared and counted as one union."""

    def __init__(self, graphs=None, vertex_offsets=None, rowptr=None, colidx=None,
                 symmetric: bool = False, stream=None):
        if graphs is not None:
            vertex_offsets, rowptr, colidx = batch_csr(graphs)
        flags = INPUT_SYMMETRIC if symmetric else 0
        self.handle = bbtc_graph_create_batch(vertex_offsets, rowptr, colidx, flags, stream)
        self.n = int(np.asarray(vertex_offsets)[-1])
        self.num_graphs = len(vertex_offsets) - 1
