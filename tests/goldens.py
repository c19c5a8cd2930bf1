"""Readers of the stored expected values under tests/golden/ (all written by
tests/golden/make_golden.py from graphgen inputs and the CPU oracle alone)."""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                yield line.split()


def config_counts() -> dict:
    """name -> {n, m, triangles, wedges, wmin} (config_counts.txt)."""
    out = {}
    for k, n, m, T, wedges, wmin in _rows("config_counts.txt"):
        out[k] = {"n": int(n), "m": int(m), "triangles": int(T), "wedges": int(wedges),
                  "wmin": int(wmin)}
    return out


def rmat_s23_per_task() -> dict:
    """p -> (total, per-task counts in Alg. 4 order) of R-MAT scale 23, edge-balanced cuts."""
    out = {}
    for row in _rows("rmat_s23_per_task.txt"):
        p, total = int(row[0]), int(row[1])
        out[p] = (total, np.array([int(x) for x in row[2:]], dtype=np.uint64))
    return out


def batch4096() -> np.ndarray:
    """(4096, 4) int64: g, n, m, triangles of each graph of the batched workload."""
    return np.array([[int(x) for x in row] for row in _rows("batch4096_counts.txt")],
                    dtype=np.int64)


def chunglu_friendster_vertices() -> dict:
    """original vertex id -> triangles at it, for the sampled vertices."""
    return {int(x): int(t) for x, t in _rows("chunglu_friendster_vertices.txt")}
