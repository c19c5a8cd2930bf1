"""The C ABI library loads and exports every declared entry point (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2009_12457_gb300 as bb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "bbtc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(bbtc_[a-z_0-9]+)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("bbtc_graph_create", "bbtc_count", "bbtc_count_batch",
                     "bbtc_graph_destroy", "bbtc_last_error", "bbtc_num_tasks"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(bb._build.build())
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_struct_layout_matches_c():
    o = bb.bbtc_opts_init()
    assert o.struct_size == ctypes.sizeof(bb.bbtc_opts)
    assert o.kernel == 0 and o.p == 0 and o.device_budget_bytes == 0


def test_num_tasks():
    assert [bb.bbtc_num_tasks(p) for p in range(0, 5)] == [0, 1, 4, 10, 20]
    assert bb.bbtc_num_tasks(36) == 8436
    assert bb.bbtc_num_tasks(-3) == 0


def test_argument_errors_without_touching_the_gpu():
    lib = bb.load()
    h = ctypes.c_void_p()
    rp = np.zeros(2, dtype=np.int64)
    assert lib.bbtc_graph_create(-1, rp.ctypes.data, None, 0, ctypes.byref(h)) == 1
    assert "outside" in bb.bbtc_last_error()
    assert lib.bbtc_graph_create(1, rp.ctypes.data, None, 0, None) == 1
    assert lib.bbtc_graph_create(1, None, None, 0, ctypes.byref(h)) == 1
    assert lib.bbtc_graph_create(1, rp.ctypes.data, None, 0x80, ctypes.byref(h)) == 1
    assert lib.bbtc_graph_create(1 << 31, rp.ctypes.data, None, 0, ctypes.byref(h)) == 1
    c = ctypes.c_uint64()
    assert lib.bbtc_count(None, None, ctypes.byref(c)) == 1
    bad = bb.bbtc_opts_init()
    bad.struct_size = 8
    assert lib.bbtc_count_batch(None, -1, ctypes.byref(bad), None, None) == 1
    lib.bbtc_graph_destroy(None)  # accepted


def test_python_binding_rejects_bad_dtypes():
    with pytest.raises(TypeError):
        bb.bbtc_graph_create(2, np.zeros(3, dtype=np.int32), np.zeros(0, dtype=np.int32))


def _c_struct_fields(name):
    """Field names of a typedef'd struct in include/bbtc.h, in declaration order."""
    text = open(os.path.join(ROOT, "include", "bbtc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", text).group(1)
    return re.findall(r"([A-Za-z_][A-Za-z0-9_]*)\s*;", body)


def test_python_structs_mirror_the_header():
    assert [f for f, _ in bb.bbtc_opts._fields_] == _c_struct_fields("bbtc_opts")
    assert [f for f, _ in bb.bbtc_graph_info._fields_] == _c_struct_fields("bbtc_graph_info")
    assert [f for f, _ in bb.bbtc_timings._fields_] == _c_struct_fields("bbtc_timings")


def test_partition_option():
    assert bb.bbtc_opts_init().partition == 0           # edge-balanced by default
    assert bb.make_opts(p=4, partition="probe").partition == 1
    assert bb.make_opts(p=4, partition="edges").partition == 0
    text = open(os.path.join(ROOT, "include", "bbtc.h")).read()
    assert "BBTC_PARTITION_EDGES = 0" in text and "BBTC_PARTITION_PROBE = 1" in text


def test_python_struct_offsets_match_the_c_compiler(tmp_path):
    """Offsets and sizes of the three public structs as gcc lays them out from
    include/bbtc.h, against the ctypes mirrors the binding passes to the library."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = ("bbtc_opts", "bbtc_graph_info", "bbtc_timings")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bbtc.h"', "int main(void) {"]
    for s in structs:
        lines.append(f'  printf("{s} sizeof %zu\\n", sizeof({s}));')
        for f in _c_struct_fields(s):
            lines.append(f'  printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True,
                               text=True).stdout.splitlines():
        s, f, v = line.split()
        got[(s, f)] = int(v)
    for s in structs:
        cls = getattr(bb, s)
        assert got[(s, "sizeof")] == ctypes.sizeof(cls), s
        for f, _ in cls._fields_:
            assert got[(s, f)] == getattr(cls, f).offset, (s, f)
