"""Independent pins for the oracle: facts fixed by the paper or by mathematics.

``pin_battery()`` runs a compact set of checks against whatever oracle build is
active and returns the list of failures. The pin tests run it on the oracle
itself (expecting none) and on deliberately broken copies of it (expecting at
least one), so every pin below is shown to catch a plausible mistake.
"""
from __future__ import annotations

import os

import numpy as np

import oracle
from tests import graphs as G

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_table4_pairs():
    rows = []
    with open(os.path.join(GOLDEN, "table4_tiles_tasks.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                tiles, tasks = (int(x) for x in line.split())
                rows.append((tiles, tasks))
    return rows


def load_toy_tasks():
    out = []
    with open(os.path.join(GOLDEN, "toy_tasks_p3.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(tuple(int(x) for x in line.split()))
    return out


def positions_by_definition(n, rowptr, colidx):
    """(rank, perm, oriented out-degree) from the dense adjacency and Sec. 4.1's rule."""
    A = G.dense_adjacency(n, rowptr, colidx)
    deg = A.sum(axis=1)
    perm = np.lexsort((np.arange(n), deg))      # by degree, then id
    rank = np.empty(n, dtype=np.int64)
    rank[perm] = np.arange(n)
    ar, br = np.nonzero(np.triu(A, 1))
    lo = np.minimum(rank[ar], rank[br])
    outdeg = np.bincount(lo, minlength=n)
    return A, deg, rank, perm, outdeg


def cuts_by_definition(n, outdeg_by_position, p):
    rp = np.concatenate([[0], np.cumsum(outdeg_by_position)])
    m = int(rp[-1])
    c = [0]
    for i in range(1, p):
        target = -(-i * m // p)
        r = 0
        while r < n and rp[r] < target:
            r += 1
        c.append(r)
    c.append(n)
    return np.array(c, dtype=np.int64)


def per_task_brute(n, rowptr, colidx, p):
    """Per-task counts by enumerating vertex triples and placing each triangle."""
    A, deg, rank, perm, outdeg = positions_by_definition(n, rowptr, colidx)
    c = cuts_by_definition(n, outdeg[np.arange(n)], p)
    part = np.searchsorted(c, np.arange(n), side="right") - 1
    part = np.minimum(part, p - 1)
    index = {}
    for i in range(p):
        for j in range(i, p):
            for k in range(j, p):
                index[(i, j, k)] = len(index)
    out = np.zeros(len(index), dtype=np.uint64)
    for a in range(n):
        for b in range(a + 1, n):
            if not A[a, b]:
                continue
            for d in range(b + 1, n):
                if A[a, d] and A[b, d]:
                    x, y, z = sorted((rank[a], rank[b], rank[d]))
                    out[index[(int(part[x]), int(part[y]), int(part[z]))]] += 1
    return out


def position_adjacency(A, rank):
    """Dense adjacency in position space with every edge stored once, u < v (Sec. 2)."""
    Ar = np.zeros_like(A)
    ar, br = np.nonzero(np.triu(A, 1))
    Ar[np.minimum(rank[ar], rank[br]), np.maximum(rank[ar], rank[br])] = 1
    return Ar


def block_nnz_by_definition(Ar, c):
    """|G_ij| = edges (u, v), u < v, with u in V_i = [c_i, c_{i+1}) and v in V_j (Sec. 2),
    summed over the dense position-space adjacency; empty parts hold nothing."""
    p = len(c) - 1
    out = np.zeros((p, p), dtype=np.int64)
    for i in range(p):
        for j in range(p):
            out[i, j] = int(Ar[c[i]:c[i + 1], c[j]:c[j + 1]].sum())
    return out


def cuts_with_empty_parts(n, p, rng):
    """Random valid cuts c_0 = 0 <= ... <= c_p = n in which some parts are empty:
    the first, the last and one in the middle (when p allows)."""
    inner = np.sort(rng.integers(0, n + 1, p - 1)) if p > 1 else np.array([], dtype=np.int64)
    c = np.concatenate([[0], inner, [n]]).astype(np.int64)
    if p >= 2:
        c[1] = 0                     # part 0 empty
        c[p - 1] = n                 # part p-1 empty
    if p >= 4:
        c[2] = c[3]                  # part 2 empty
    return np.maximum.accumulate(c)


def with_noise(n, rowptr, colidx, rng, dup=0.3, loops=3):
    """Same simple graph, with duplicate entries and self-loops added."""
    rows = [list(colidx[rowptr[v]:rowptr[v + 1]]) for v in range(n)]
    for v in range(n):
        extra = [x for x in rows[v] if rng.random() < dup]
        rows[v] += extra
    for _ in range(loops):
        if n:
            v = int(rng.integers(0, n))
            rows[v].append(v)
    for v in range(n):
        rng.shuffle(rows[v])
    rp = np.zeros(n + 1, dtype=np.int64)
    for v in range(n):
        rp[v + 1] = rp[v] + len(rows[v])
    ci = np.array([x for r in rows for x in r], dtype=np.int32)
    return n, rp, ci


def pbd_pins(check, rng):
    """Pins of the probe-based partition, from the dense adjacency and by hand."""
    # two disjoint K_64 (ids 0-63 and 64-127), p = 2: every vertex has degree 63,
    # so grain t is vertex t and the order is the id order. Part 0 can hold clique
    # 0 plus vertex 64 (which adds no edge to it) within B = C(64,2) = 2016, and
    # part 1 then holds C(63,2) = 1953 edges with 63 edges in block (0,1). Any
    # B < 2016 leaves a whole clique's 2016 edges in one block.
    n2, rp2, ci2 = G.csr_from_edges(128, [(a + o, b + o) for o in (0, 64)
                                          for a in range(64) for b in range(a + 1, 64)])
    pr = oracle.prepare(n2, rp2, ci2)
    c, bstar = oracle.pbd_cuts(n2, pr["rowptr"], pr["colidx"], 2)
    check(bstar == 2016 and c.tolist() == [0, 65, 128], f"PBD two K_64: {bstar} {c.tolist()}")
    # p = 1: one part, B* = m
    c, bstar = oracle.pbd_cuts(n2, pr["rowptr"], pr["colidx"], 1)
    check(bstar == pr["m"] and c.tolist() == [0, 128], "PBD p=1")

    for trial in range(6):
        n = int(rng.integers(40, 260))
        g = G.gnp(n, float(rng.uniform(0.02, 0.3)), rng)
        # skew the degrees: a few hubs joined to many vertices
        A0 = G.dense_adjacency(*g)
        for h in rng.choice(n, size=3, replace=False):
            others = rng.random(n) < 0.6
            A0[h, others] = 1
            A0[others, h] = 1
        np.fill_diagonal(A0, 0)
        g = G.csr_from_edges(n, list(zip(*np.nonzero(np.triu(A0, 1)))))
        A, deg, rank, perm, outdeg = positions_by_definition(*g)
        pr = oracle.prepare(*g)
        m = pr["m"]
        Ar = np.zeros_like(A)                    # adjacency in position space, u < v
        ar, br = np.nonzero(np.triu(A, 1))
        lo_, hi_ = np.minimum(rank[ar], rank[br]), np.maximum(rank[ar], rank[br])
        Ar[lo_, hi_] = 1
        cum = np.zeros((n + 1, n + 1), dtype=np.int64)
        cum[1:, 1:] = Ar.cumsum(0).cumsum(1)

        def edges_in(u0, u1, v0, v1):
            return int(cum[u1, v1] - cum[u0, v1] - cum[u1, v0] + cum[u0, v0])

        for p in (2, 3, 5):
            Gn = oracle.pbd_grains(p)
            check(Gn == min(2048, 64 * p), f"grain count p={p}")
            b = oracle.pbd_grain_bounds(n, pr["rowptr"], pr["colidx"], Gn)
            # grains: b_t = min{ r : D(r) >= ceil(t*2m/G) }, D over undirected degree
            D = np.concatenate([[0], np.cumsum(deg[perm])])
            want = [0] + [int(np.searchsorted(D, -(-t * 2 * m // Gn), side="left"))
                          for t in range(1, Gn)] + [n]
            check(b.tolist() == want, f"PBD grain bounds p={p} trial {trial}")
            S = oracle.pbd_prefix(n, pr["rowptr"], pr["colidx"], Gn, b)
            for _ in range(30):
                r0, r1 = sorted(int(x) for x in rng.integers(0, Gn + 1, 2))
                c0, c1 = sorted(int(x) for x in rng.integers(0, Gn + 1, 2))
                check(oracle.pbd_load(S, r0, r1, c0, c1) == edges_in(b[r0], b[r1], b[c0], b[c1]),
                      f"PBD load ({r0},{r1},{c0},{c1}) trial {trial}")
            c, bstar = oracle.pbd_cuts(n, pr["rowptr"], pr["colidx"], p)
            nnz = oracle.block_nnz(n, pr["rowptr"], pr["colidx"], p, c)
            check(int(nnz.max()) <= bstar, f"PBD blocks above B* p={p} trial {trial}")
            check(c[0] == 0 and c[p] == n and np.all(np.diff(c) >= 0), f"PBD cuts valid p={p}")
            ok, x = oracle.pbd_probe(S, p, bstar)
            check(ok and np.array_equal(b[x], c), f"PBD probe(B*) p={p} trial {trial}")
            nb = p * (p + 1) // 2
            okm, _ = oracle.pbd_probe(S, p, bstar - 1)
            check(bstar == -(-m // nb) or not okm, f"PBD bisection not converged p={p}")
            # each closed part is maximal: one more grain breaks a block of its column
            for i in range(p):
                if x[i] == Gn or x[i + 1] == Gn:
                    continue
                t = int(x[i + 1]) + 1
                loads = [edges_in(b[x[i]], b[t], b[x[i]], b[t])]
                loads += [edges_in(b[x[k]], b[x[k + 1]], b[x[i]], b[t]) for k in range(i)]
                check(max(loads) > bstar, f"PBD part {i} not maximal p={p} trial {trial}")


def pin_battery() -> list[str]:
    fails: list[str] = []

    def check(cond, msg):
        if not cond:
            fails.append(msg)

    rng = np.random.default_rng(12345)

    # Alg. 1 against set intersection on random sorted lists
    for _ in range(200):
        A = np.unique(rng.integers(0, 40, rng.integers(0, 20)))
        B = np.unique(rng.integers(0, 40, rng.integers(0, 20)))
        check(oracle.n_intersect(A, B) == len(set(A.tolist()) & set(B.tolist())),
              f"Alg.1 on {A.tolist()} {B.tolist()}")
        if fails:
            break

    # task composition: Tab. 4 pairs and the toy example
    for tiles, tasks in load_table4_pairs():
        p = int(round(tiles ** 0.5))
        check(p * p == tiles and oracle.num_tasks(p) == tasks, f"|T| for tiles={tiles}")
        check(oracle.task_list(p).shape[0] == tasks, f"Alg.4 length for p={p}")
    check([tuple(t) for t in oracle.task_list(3).tolist()] == load_toy_tasks(), "toy task list")

    # closed forms
    for k in (3, 5, 8):
        r = oracle.bbtc(*G.complete(k), p=2, want_per_vertex=True)
        check(r["total"] == G.choose(k, 3), f"K_{k}")
        check(np.all(r["per_vertex"] == G.choose(k - 1, 2)), f"K_{k} per-vertex")
    for k in (4, 7):
        r = oracle.bbtc(*G.wheel(k), p=3, method="hmap", want_per_vertex=True)
        pv = r["per_vertex"]
        check(r["total"] == k and pv[0] == k and np.all(pv[1:] == 2), f"wheel W_{k}")
    r = oracle.bbtc(*G.complete_multipartite([2, 3, 4]), p=3)
    check(r["total"] == 24, "K_{2,3,4}")
    check(oracle.bbtc(*G.grid(4, 5), p=2)["total"] == 0, "grid")

    # random graphs with noise: brute force, trace(A^3)/6, per-vertex, per task
    for trial in range(12):
        n = int(rng.integers(6, 22))
        g = G.gnp(n, float(rng.uniform(0.2, 0.8)), rng)
        noisy = with_noise(*g, rng)
        T = G.brute_force_triangles(*g)
        check(G.trace_cubed_over_six(*g) == T, "brute vs trace (test helper)")
        pr = oracle.prepare(*noisy)
        check(pr["m"] == int(G.dense_adjacency(*g).sum() // 2), f"canonical edge count trial {trial}")
        check(oracle.tc_intersect(n, pr["rowptr"], pr["colidx"]) == T, f"Alg.2 trial {trial}")
        check(oracle.tc_hmap(n, pr["rowptr"], pr["colidx"]) == T, f"Alg.3 trial {trial}")
        pv = oracle.per_vertex(n, pr["rowptr"], pr["colidx"], pr["perm"])
        check(np.array_equal(pv, G.per_vertex_dense(*g)), f"per-vertex trial {trial}")
        # edge support: common neighbours of each edge's endpoints (dense A @ A)
        A2 = G.dense_adjacency(*g)
        common = A2 @ A2
        sup = oracle.edge_support(n, pr["rowptr"], pr["colidx"])
        src = np.repeat(np.arange(n), np.diff(pr["rowptr"]))
        a, b = pr["perm"][src], pr["perm"][pr["colidx"]]
        check(np.array_equal(sup.astype(np.int64), common[a, b]), f"edge support trial {trial}")
        # the order: degree non-decreasing along positions, ties by id, edges upward
        A, deg, rank, perm, outdeg = positions_by_definition(*g)
        check(np.array_equal(pr["perm"], perm), f"degree order trial {trial}")
        check(np.array_equal(np.diff(pr["rowptr"]), outdeg), f"out-degrees trial {trial}")
        # |G_ij| (Sec. 2) for the whole p x p matrix, against the dense adjacency:
        # on the edge-balanced cuts and on cuts with empty parts
        Ar = position_adjacency(A, rank)
        for p in (1, 2, 3, 5, 8):
            for c in (cuts_by_definition(n, outdeg, p), cuts_with_empty_parts(n, p, rng)):
                got = oracle.block_nnz(n, pr["rowptr"], pr["colidx"], p, c)
                check(np.array_equal(got, block_nnz_by_definition(Ar, c)),
                      f"block sizes p={p} cuts {c.tolist()} trial {trial}")
        for p in (1, 2, 3, 5):
            c = oracle.cuts(n, pr["rowptr"], p)
            check(np.array_equal(c, cuts_by_definition(n, outdeg, p)), f"cuts p={p} trial {trial}")
            brute = per_task_brute(*g, p)
            r5 = oracle.bbtc(*noisy, p=p, method="intersect", prep=pr)
            r6 = oracle.bbtc(*noisy, p=p, method="hmap", prep=pr)
            cls = oracle.classify_triangles(n, pr["rowptr"], pr["colidx"], p, c)
            check(np.array_equal(r5["per_task"], brute), f"Alg.5 per task p={p} trial {trial}")
            check(np.array_equal(r6["per_task"], brute), f"Alg.6 per task p={p} trial {trial}")
            check(np.array_equal(cls, brute), f"classified per task p={p} trial {trial}")
        if len(fails) > 20:
            break

    # probe-based partition
    pbd_pins(check, rng)

    # ExecTime on a hand-worked example: p=2, cuts [0,2,5],
    # |G_00|=3, |G_01|=4, |G_11|=6 -> delta(G_00)=1.5, delta(G_01)=2, delta(G_11)=2
    # tasks (0,0,0): 3*1.5=4.5 ; (0,0,1): 3*max(2,2)=6 ; (0,1,1): 4*max(2,2)=8 ;
    # (1,1,1): 6*2=12
    est = oracle.exec_time(2, np.array([0, 2, 5]), np.array([[3, 4], [0, 6]]))
    check(np.allclose(est, [4.5, 6.0, 8.0, 12.0]), f"ExecTime example {est.tolist()}")
    # p=2, cuts [0,4,5], |G_00|=2, |G_01|=1, |G_11|=3: delta = 0.5, 0.25, 3
    # -> (0,0,0)=2*0.5, (0,0,1)=2*0.25, (0,1,1)=1*max(0.25,3), (1,1,1)=3*3
    est = oracle.exec_time(2, np.array([0, 4, 5]), np.array([[2, 1], [0, 3]]))
    check(np.allclose(est, [2 * 0.5, 2 * 0.25, 1 * 3.0, 3 * 3.0]), f"ExecTime example 2 {est.tolist()}")
    order = oracle.order_tasks(np.array([1.0, 3.0, 3.0, 2.0]))
    check(order.tolist() == [1, 2, 3, 0], "task order: non-increasing, ties in Alg.4 order")

    # algorithmic-bytes figures on the triangle 0-1-2 with a pendant vertex 3 on 2,
    # by hand: degrees 2, 2, 3, 1 give the order 3, 0, 1, 2 (positions 0..3), the
    # oriented edges (0,3), (1,2), (1,3), (2,3) and out-degrees d+ = 1, 2, 1, 0.
    # wedges = sum over edges of d+(v) = 0 + 1 + 0 + 0 = 1; wmin = 4 * (4 + 1) = 20;
    # wmerge = 4 * sum over edges of (d+(u) + d+(v)) = 4 * (1 + 3 + 2 + 1) = 28.
    n, rp, ci = G.csr_from_edges(4, [(0, 1), (1, 2), (0, 2), (2, 3)])
    pr = oracle.prepare(n, rp, ci)
    wf = oracle.work_figures(n, pr["rowptr"], pr["colidx"])
    check((wf["wedges"], wf["wmin"], wf["wmerge"]) == (1, 20, 28), f"work figures by hand {wf}")
    # and on random graphs, from the dense position-space adjacency
    for trial in range(4):
        nn = int(rng.integers(8, 40))
        g = G.gnp(nn, float(rng.uniform(0.1, 0.6)), rng)
        A, deg, rank, perm, outdeg = positions_by_definition(*g)
        us, vs = np.nonzero(position_adjacency(A, rank))
        pr = oracle.prepare(*g)
        wf = oracle.work_figures(nn, pr["rowptr"], pr["colidx"])
        want = (int(outdeg[vs].sum()), 4 * (len(us) + int(outdeg[vs].sum())),
                4 * int((outdeg[us] + outdeg[vs]).sum()))
        check((wf["wedges"], wf["wmin"], wf["wmerge"]) == want, f"work figures trial {trial}")
    return fails
