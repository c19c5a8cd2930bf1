"""Write the stored expected values of the seeded workloads, computed by the CPU
oracle alone (graphgen inputs + oracle; nothing from the CUDA library).

Run from the repository root:  python tests/golden/make_golden.py [jobs...]

Jobs and the files they write (all under tests/golden/):

* ``rmat_s14_ef16_seed1``, ``rmat_s23_ef16_seed2``, ``chunglu_friendster_seed3``:
  one row each of config_counts.txt -- n, m, the triangle count and the work
  figures of the oriented graph. The Friendster-shaped graph (3.6 G input
  entries) is prepared stage by stage, freeing each stage's input, so that it
  fits in about 55 GB of host memory; it takes tens of minutes.
* ``chunglu_friendster_vertices``: chunglu_friendster_vertices.txt -- the
  triangles at a seeded sample of original vertices (the four heaviest ids and
  44 drawn ones), each from its definition on the input CSR.
* ``rmat_s23_per_task``: rmat_s23_per_task.txt -- per-task counts of R-MAT
  scale 23 for p = 4, 8 and 16 with the edge-balanced cuts, every triangle
  placed in its task (i, j, k) (Sec. 4.2), tasks in Alg. 4 order.
* ``batch4096``: batch4096_counts.txt -- n, m and the triangle count of each of
  the 4096 graphs of the batched workload, one process per host core.
"""
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import graphgen  # noqa: E402
import oracle  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
COUNTS = os.path.join(HERE, "config_counts.txt")
PER_TASK = os.path.join(HERE, "rmat_s23_per_task.txt")
BATCH = os.path.join(HERE, "batch4096_counts.txt")
VERTICES = os.path.join(HERE, "chunglu_friendster_vertices.txt")
PER_TASK_P = (4, 8, 16)
VERTEX_SAMPLE = 44


def _prepare_lean(n, rp, ci):
    """oracle.prepare, one stage at a time, dropping each stage's input."""
    keys = oracle.canonical_edges(n, rp, ci, compact=False)
    del rp, ci
    keys = keys.copy()  # frees the rowptr[n]-entry work buffer
    deg = oracle.degree(n, keys)
    rank, perm = oracle.order_by_degree(n, deg)
    del deg
    orp, oci = oracle.orient(n, keys, rank)
    return int(keys.shape[0]), orp, oci


def _count_row(name, gen, lean=False):
    n, rp, ci = gen()
    if lean:
        m, orp, oci = _prepare_lean(n, rp, ci)
        T = oracle.tc_intersect(n, orp, oci)
    else:
        pr = oracle.prepare(n, rp, ci)
        m, orp, oci = pr["m"], pr["rowptr"], pr["colidx"]
        T = oracle.tc_hmap(n, orp, oci)
    wf = oracle.work_figures(n, orp, oci)
    return [str(n), str(m), str(T), str(wf["wedges"]), str(wf["wmin"])]


COUNT_JOBS = {
    "rmat_s14_ef16_seed1": (graphgen.rmat_s14, False),
    "rmat_s23_ef16_seed2": (graphgen.rmat_s23, False),
    "chunglu_friendster_seed3": (graphgen.chunglu_friendster, True),
}


def write_counts(names):
    rows = {}
    if os.path.exists(COUNTS):
        for line in open(COUNTS):
            if line.strip() and not line.startswith("#"):
                k, *vals = line.split()
                rows[k] = vals
    for name in names:
        t0 = time.time()
        gen, lean = COUNT_JOBS[name]
        rows[name] = _count_row(name, gen, lean)
        print(name, rows[name], f"{time.time() - t0:.1f}s", flush=True)
        with open(COUNTS, "w") as f:
            f.write("# Exact counts of the seeded workloads, written by tests/golden/make_golden.py\n")
            f.write("# from graphgen inputs and the CPU oracle only (Alg. 3, or Alg. 2 for the\n")
            f.write("# Friendster-shaped graph, over the oriented CSR).\n")
            f.write("# name n m triangles wedges(sum d+(v) over edges) wmin_bytes\n")
            for k in sorted(rows):
                f.write(" ".join([k] + rows[k]) + "\n")


def vertex_sample_ids(n):
    """The four heaviest ids of the Chung-Lu recipe (weights fall with the id) and
    VERTEX_SAMPLE ids drawn from stream 99 of seed 3."""
    ids = [0, 1, 2, 3] + [graphgen.draw(3, 99, i) % n for i in range(VERTEX_SAMPLE)]
    return sorted(set(int(x) for x in ids))


def write_vertices():
    t0 = time.time()
    n, rp, ci = graphgen.chunglu_friendster()
    ids = vertex_sample_ids(n)
    with open(VERTICES, "w") as f:
        f.write("# Triangles at sampled original vertices of the Friendster-shaped Chung-Lu\n")
        f.write("# graph (seed 3), each counted from its definition on the input CSR\n")
        f.write("# (oracle.vertex_triangles); written by tests/golden/make_golden.py.\n")
        f.write("# vertex triangles\n")
        for x in ids:
            f.write(f"{x} {oracle.vertex_triangles(n, rp, ci, x)}\n")
    print("vertices", len(ids), f"{time.time() - t0:.1f}s", flush=True)


def _per_task_one(p):
    n, rp, ci = graphgen.rmat_s23()
    pr = oracle.prepare(n, rp, ci)
    c = oracle.cuts(n, pr["rowptr"], p)
    return p, oracle.classify_triangles(n, pr["rowptr"], pr["colidx"], p, c)


def write_per_task():
    t0 = time.time()
    with mp.get_context("spawn").Pool(len(PER_TASK_P)) as pool:
        res = dict(pool.map(_per_task_one, PER_TASK_P))
    with open(PER_TASK, "w") as f:
        f.write("# Per-task triangle counts of R-MAT scale 23 (ef 16, seed 2), edge-balanced\n")
        f.write("# cuts, tasks in Alg. 4 order; each triangle placed in its task (Sec. 4.2)\n")
        f.write("# by oracle.classify_triangles. Written by tests/golden/make_golden.py.\n")
        f.write("# p total count_0 ... count_{T-1}\n")
        for p in PER_TASK_P:
            v = res[p]
            f.write(" ".join([str(p), str(int(v.sum()))] + [str(int(x)) for x in v]) + "\n")
    print("per_task", {p: int(res[p].sum()) for p in PER_TASK_P}, f"{time.time() - t0:.1f}s",
          flush=True)


def _batch_one(g):
    graphgen._load().gg_set_threads(1)
    n, rp, ci = graphgen.batch_graph(g)
    pr = oracle.prepare(n, rp, ci)
    return g, n, pr["m"], oracle.tc_intersect(n, pr["rowptr"], pr["colidx"])


def write_batch(count=4096):
    t0 = time.time()
    with mp.get_context("spawn").Pool(os.cpu_count() or 1) as pool:
        rows = sorted(pool.map(_batch_one, range(count), chunksize=8))
    with open(BATCH, "w") as f:
        f.write(f"# The {count} graphs of the batched workload (graphgen.batch_spec, seeds\n")
        f.write(f"# 100-{99 + count}): n, simple edges m and triangles from the CPU oracle\n")
        f.write("# (Alg. 2 over the oriented CSR). Written by tests/golden/make_golden.py.\n")
        f.write("# g n m triangles\n")
        for g, n, m, T in rows:
            f.write(f"{g} {n} {m} {T}\n")
    print("batch", count, sum(r[3] for r in rows), f"{time.time() - t0:.1f}s", flush=True)


def main(jobs):
    for job in jobs:
        if job in COUNT_JOBS:
            write_counts([job])
        elif job == "chunglu_friendster_vertices":
            write_vertices()
        elif job == "rmat_s23_per_task":
            write_per_task()
        elif job == "batch4096":
            write_batch()
        else:
            raise SystemExit(f"unknown job {job}")


if __name__ == "__main__":
    main(sys.argv[1:] or ["rmat_s14_ef16_seed1", "rmat_s23_ef16_seed2", "rmat_s23_per_task",
                          "batch4096", "chunglu_friendster_vertices",
                          "chunglu_friendster_seed3"])
