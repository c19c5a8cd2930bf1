"""Task workload estimates (Sec. 5) and how well they find the heavy tasks (Sec. 7.5).

The task order only needs to put heavy tasks first, not to predict time
exactly. Sec. 7.5 compares four estimates by the share of the task list,
taken in estimate order, that is needed to cover the x most time-consuming
tasks (lower is better):

* NNZ:     total nonzeros of the task's three blocks, |G_ij| + |G_jk| + |G_ik|
* Density: sum over the three blocks of their nonzeros per cell, |G_ab| / (|V_a| |V_b|)
* Degree:  sum over the three blocks of their average degree, |G_ab| / |V_a|
* bbTC:    ExecTime(t) = |G_ij| * max(delta(G_ik), delta(G_jk))

Here the measured cost of a task is the SM cycles the counting kernel's warps
spent on its work items (opts.per_task_cycles_out).
"""
from __future__ import annotations

import numpy as np

from . import Graph


def estimates(plan: dict) -> dict:
    """The four estimates of every task (Alg. 4 order) from a plan (Graph.plan(p))."""
    cuts = plan["cuts"].astype(np.float64)
    nnz = plan["block_nnz"].astype(np.float64)
    vsize = np.diff(cuts)
    t = plan["tasks"]
    i, j, k = t[:, 0], t[:, 1], t[:, 2]

    def safe_div(a, b):
        return np.where(b > 0, a / np.where(b > 0, b, 1.0), 0.0)

    blocks = ((i, j), (j, k), (i, k))
    out = {
        "nnz": sum(nnz[a, b] for a, b in blocks),
        "density": sum(safe_div(nnz[a, b], vsize[a] * vsize[b]) for a, b in blocks),
        "degree": sum(safe_div(nnz[a, b], vsize[a]) for a, b in blocks),
        "bbtc": plan["exec_time"].astype(np.float64),
    }
    return out


def coverage(estimate: np.ndarray, cost: np.ndarray, xs=(1, 2, 4, 8, 16, 32)) -> dict:
    """Share of tasks, taken in non-increasing estimate order (ties in Alg. 4 order),
    needed to include the x most costly tasks, for each x."""
    order = np.lexsort((np.arange(len(estimate)), -estimate))
    pos = np.empty(len(order), dtype=np.int64)
    pos[order] = np.arange(len(order))
    by_cost = np.argsort(-cost, kind="stable")
    out = {}
    for x in xs:
        if x > len(cost):
            break
        out[x] = float(pos[by_cost[:x]].max() + 1) / len(cost)
    return out


def spearman(a: np.ndarray, b: np.ndarray) -> float:
    """Rank correlation (average ranks for ties)."""
    def ranks(x):
        order = np.argsort(x, kind="stable")
        r = np.empty(len(x), dtype=np.float64)
        r[order] = np.arange(len(x), dtype=np.float64)
        xs = x[order]
        start = 0
        for end in range(1, len(x) + 1):
            if end == len(x) or xs[end] != xs[start]:
                r[order[start:end]] = (start + end - 1) / 2.0
                start = end
        return r
    ra, rb = ranks(np.asarray(a, dtype=np.float64)), ranks(np.asarray(b, dtype=np.float64))
    ra -= ra.mean()
    rb -= rb.mean()
    den = np.sqrt((ra * ra).sum() * (rb * rb).sum())
    return float((ra * rb).sum() / den) if den > 0 else 0.0


def study(graph: Graph, p: int, kernel: str = "auto", repeats: int = 3) -> dict:
    """Measure per-task cost on `graph` at p and score the four estimates."""
    cycles = None
    for _ in range(repeats):  # keep the smallest cycle count of each task
        out = graph.count(p=p, kernel=kernel, per_task_cycles=True)
        c = out["per_task_cycles"].astype(np.float64)
        cycles = c if cycles is None else np.minimum(cycles, c)
    plan = graph.plan(p)
    est = estimates(plan)
    worked = cycles > 0
    return {
        "p": p, "tasks": int(len(cycles)), "tasks_with_work": int(worked.sum()),
        "coverage": {name: coverage(e, cycles) for name, e in est.items()},
        "spearman": {name: spearman(e[worked], cycles[worked]) for name, e in est.items()},
    }


def main(argv=None):
    """Run the study on a seeded R-MAT graph and print one JSON line."""
    import argparse
    import json

    import graphgen

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--scale", type=int, default=21)
    ap.add_argument("--edge-factor", type=int, default=16)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--p", default="8,16")
    ap.add_argument("--kernel", default="auto")
    ap.add_argument("--repeats", type=int, default=3)
    a = ap.parse_args(argv)
    n, rp, ci = graphgen.rmat(a.scale, a.edge_factor, a.seed)
    with Graph(n, rp, ci, symmetric=True) as g:
        for p in (int(x) for x in a.p.split(",")):
            r = study(g, p, a.kernel, a.repeats)
            r.update({"graph": f"R-MAT scale {a.scale}, edge factor {a.edge_factor}, seed {a.seed}",
                      "kernel": a.kernel})
            print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
