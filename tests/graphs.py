"""Small test graphs with known triangle counts, and brute-force counters.

Graphs are returned as ``(n, rowptr, colidx)`` CSR arrays listing every edge in
both directions. The brute-force counters work on a dense 0/1 adjacency matrix
built straight from the CSR, independently of the oracle's code.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def csr_from_edges(n: int, edges, both_directions: bool = True):
    rows = [[] for _ in range(n)]
    for a, b in edges:
        rows[a].append(b)
        if both_directions:
            rows[b].append(a)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    for v in range(n):
        rowptr[v + 1] = rowptr[v] + len(rows[v])
    colidx = np.array([x for r in rows for x in r], dtype=np.int32)
    return n, rowptr, colidx


def complete(n):
    return csr_from_edges(n, itertools.combinations(range(n), 2))


def cycle(n):
    return csr_from_edges(n, [(i, (i + 1) % n) for i in range(n)])


def wheel(n):
    """Hub 0 joined to every vertex of the cycle 1..n."""
    rim = [(1 + i, 1 + (i + 1) % n) for i in range(n)]
    spokes = [(0, 1 + i) for i in range(n)]
    return csr_from_edges(n + 1, rim + spokes)


def friendship(k):
    """k triangles sharing the single vertex 0."""
    edges = []
    for t in range(k):
        a, b = 1 + 2 * t, 2 + 2 * t
        edges += [(0, a), (0, b), (a, b)]
    return csr_from_edges(2 * k + 1, edges)


def complete_multipartite(sizes):
    starts = np.cumsum([0] + list(sizes))
    part = np.repeat(np.arange(len(sizes)), sizes)
    n = int(starts[-1])
    edges = [(a, b) for a in range(n) for b in range(a + 1, n) if part[a] != part[b]]
    return csr_from_edges(n, edges)


def grid(r, c):
    edges = []
    for i in range(r):
        for j in range(c):
            v = i * c + j
            if j + 1 < c:
                edges.append((v, v + 1))
            if i + 1 < r:
                edges.append((v, v + c))
    return csr_from_edges(r * c, edges)


def random_tree(n, rng):
    return csr_from_edges(n, [(v, int(rng.integers(0, v))) for v in range(1, n)])


def gnp(n, prob, rng):
    upper = np.triu(rng.random((n, n)) < prob, 1)
    a, b = np.nonzero(upper)
    return csr_from_edges(n, list(zip(a.tolist(), b.tolist())))


def dense_adjacency(n, rowptr, colidx):
    """Simple undirected 0/1 adjacency (symmetrised, no self-loops)."""
    A = np.zeros((n, n), dtype=np.int64)
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    A[rows, colidx] = 1
    A[colidx, rows] = 1
    np.fill_diagonal(A, 0)
    return A


def brute_force_triangles(n, rowptr, colidx):
    """Count vertex triples a < b < c with all three edges present, one by one."""
    A = dense_adjacency(n, rowptr, colidx)
    t = 0
    for a in range(n):
        for b in range(a + 1, n):
            if not A[a, b]:
                continue
            for c in range(b + 1, n):
                if A[a, c] and A[b, c]:
                    t += 1
    return t


def trace_cubed_over_six(n, rowptr, colidx):
    """trace(A^3)/6 with exact float64 products (entries stay far below 2^53)."""
    A = dense_adjacency(n, rowptr, colidx).astype(np.float64)
    A2 = A @ A
    tr = float(np.einsum("ij,ji->", A2, A))
    return int(round(tr)) // 6


def per_vertex_dense(n, rowptr, colidx):
    """Triangles at each vertex: (A^3)_vv / 2."""
    A = dense_adjacency(n, rowptr, colidx).astype(np.float64)
    d = np.einsum("ij,ji->i", A @ A, A)
    return np.rint(d / 2).astype(np.uint64)


def choose(n, k):
    return math.comb(n, k)
