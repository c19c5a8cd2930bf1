"""Pins of the CPU oracle against the paper and against mathematics (no GPU)."""
import itertools

import numpy as np
import pytest

import graphgen
import oracle
from tests import graphs as G
from tests import pins


def test_pin_battery_passes():
    assert pins.pin_battery() == []


@pytest.mark.parametrize("p", [1, 2, 3, 4, 7])
@pytest.mark.parametrize("method", ["intersect", "hmap"])
def test_closed_forms(p, method):
    cases = []
    for k in range(3, 11):
        cases.append((G.complete(k), G.choose(k, 3)))
    for k in range(4, 11):
        cases.append((G.wheel(k), k))
    for k in range(1, 6):
        cases.append((G.friendship(k), k))
    for sizes in ([1, 1, 1], [2, 2, 2], [1, 3, 5], [4, 2, 3]):
        a, b, c = sizes
        cases.append((G.complete_multipartite(sizes), a * b * c))
    cases.append((G.complete_multipartite([3, 4]), 0))     # complete bipartite
    cases.append((G.complete_multipartite([5, 5]), 0))
    cases.append((G.grid(5, 6), 0))
    cases.append((G.cycle(8), 0))
    cases.append((G.cycle(3), 1))
    cases.append((G.random_tree(30, np.random.default_rng(1)), 0))
    for g, expect in cases:
        r = oracle.bbtc(*g, p=p, method=method)
        assert r["total"] == expect
        assert int(r["per_task"].sum()) == expect


def test_per_vertex_closed_forms():
    for k in range(3, 12):
        r = oracle.bbtc(*G.complete(k), p=2, want_per_vertex=True)
        assert np.all(r["per_vertex"] == G.choose(k - 1, 2))
    for k in range(4, 12):
        pv = oracle.bbtc(*G.wheel(k), p=2, want_per_vertex=True)["per_vertex"]
        assert pv[0] == k and np.all(pv[1:] == 2)
    pv = oracle.bbtc(*G.friendship(4), p=3, want_per_vertex=True)["per_vertex"]
    assert pv[0] == 4 and np.all(pv[1:] == 1)


def test_brute_force_many_seeds():
    rng = np.random.default_rng(7)
    for seed in range(300):
        n = int(rng.integers(1, 30))
        g = G.gnp(n, float(rng.choice([0.05, 0.2, 0.5, 0.9])), rng)
        T = G.brute_force_triangles(*g)
        pr = oracle.prepare(*g)
        assert oracle.tc_intersect(n, pr["rowptr"], pr["colidx"]) == T
        assert oracle.tc_hmap(n, pr["rowptr"], pr["colidx"]) == T
        p = int(rng.integers(1, 6))
        assert oracle.bbtc(*g, p=p, method="intersect", prep=pr)["total"] == T


@pytest.mark.parametrize("n,prob", [(120, 0.3), (300, 0.1), (500, 0.05), (200, 0.9)])
def test_trace_a_cubed(n, prob):
    g = G.gnp(n, prob, np.random.default_rng(n))
    T = G.trace_cubed_over_six(*g)
    pr = oracle.prepare(*g)
    assert oracle.tc_intersect(n, pr["rowptr"], pr["colidx"]) == T
    assert oracle.tc_hmap(n, pr["rowptr"], pr["colidx"]) == T
    r = oracle.bbtc(*g, p=6, method="hmap", prep=pr, want_per_vertex=True)
    assert r["total"] == T
    assert np.array_equal(r["per_vertex"], G.per_vertex_dense(*g))
    assert int(r["per_vertex"].sum()) == 3 * T


def test_per_task_brute_force():
    rng = np.random.default_rng(3)
    for _ in range(20):
        n = int(rng.integers(5, 26))
        g = G.gnp(n, float(rng.uniform(0.15, 0.9)), rng)
        pr = oracle.prepare(*g)
        for p in range(1, 7):
            brute = pins.per_task_brute(*g, p)
            c = oracle.cuts(n, pr["rowptr"], p)
            for method in ("intersect", "hmap"):
                r = oracle.bbtc(*g, p=p, method=method, prep=pr)
                assert np.array_equal(r["per_task"], brute)
            assert np.array_equal(oracle.classify_triangles(n, pr["rowptr"], pr["colidx"], p, c), brute)


def test_task_composition():
    for tiles, tasks in pins.load_table4_pairs():
        p = int(round(tiles ** 0.5))
        assert p * p == tiles
        assert oracle.num_tasks(p) == tasks
        tl = oracle.task_list(p)
        assert tl.shape == (tasks, 3)
        assert len({tuple(t) for t in tl.tolist()}) == tasks
    assert [tuple(t) for t in oracle.task_list(3).tolist()] == pins.load_toy_tasks()
    for p in range(1, 20):
        expect = [(i, j, k) for i, j, k in itertools.product(range(p), repeat=3) if i <= j <= k]
        assert [tuple(t) for t in oracle.task_list(p).tolist()] == expect


def test_canonical_edges_and_noise_invariance():
    rng = np.random.default_rng(11)
    for _ in range(30):
        n = int(rng.integers(2, 40))
        g = G.gnp(n, 0.3, rng)
        noisy = pins.with_noise(*g, rng, dup=0.5, loops=5)
        keys = oracle.canonical_edges(*noisy)
        A = G.dense_adjacency(*g)
        a, b = np.nonzero(np.triu(A, 1))
        expect = np.sort((a.astype(np.uint64) << np.uint64(32)) | b.astype(np.uint64))
        assert np.array_equal(keys, expect)
        assert oracle.bbtc(*noisy, p=3)["total"] == G.brute_force_triangles(*g)


def test_one_direction_listing():
    rng = np.random.default_rng(5)
    g = G.gnp(40, 0.3, rng)
    A = G.dense_adjacency(*g)
    a, b = np.nonzero(np.triu(A, 1))
    flip = rng.random(a.shape[0]) < 0.5
    src = np.where(flip, a, b)
    dst = np.where(flip, b, a)
    one = G.csr_from_edges(40, list(zip(src.tolist(), dst.tolist())), both_directions=False)
    assert oracle.bbtc(*one, p=4)["total"] == G.brute_force_triangles(*g)


def test_relabel_and_disjoint_union():
    rng = np.random.default_rng(9)
    g = G.gnp(60, 0.2, rng)
    n, rp, ci = g
    T = oracle.bbtc(*g, p=3)["total"]
    perm = rng.permutation(n)
    A = G.dense_adjacency(*g)
    a, b = np.nonzero(np.triu(A, 1))
    relabelled = G.csr_from_edges(n, list(zip(perm[a].tolist(), perm[b].tolist())))
    assert oracle.bbtc(*relabelled, p=5)["total"] == T
    h = G.complete(7)
    edges = list(zip(a.tolist(), b.tolist())) + [(n + x, n + y) for x, y in itertools.combinations(range(7), 2)]
    union = G.csr_from_edges(n + 7, edges)
    assert oracle.bbtc(*union, p=4)["total"] == T + 35


def test_config1_two_oracles_agree():
    n, rp, ci = graphgen.rmat_s14()
    pr = oracle.prepare(n, rp, ci)
    T2 = oracle.tc_intersect(n, pr["rowptr"], pr["colidx"])
    T3 = oracle.tc_hmap(n, pr["rowptr"], pr["colidx"])
    assert T2 == T3
    for p in (2, 5):
        r5 = oracle.bbtc(n, rp, ci, p=p, method="intersect", prep=pr)
        r6 = oracle.bbtc(n, rp, ci, p=p, method="hmap", prep=pr)
        c = oracle.cuts(n, pr["rowptr"], p)
        cls = oracle.classify_triangles(n, pr["rowptr"], pr["colidx"], p, c)
        assert np.array_equal(r5["per_task"], r6["per_task"])
        assert np.array_equal(r5["per_task"], cls)
        assert r5["total"] == T2
    pv = oracle.per_vertex(n, pr["rowptr"], pr["colidx"], pr["perm"])
    assert int(pv.sum()) == 3 * T2


def test_vertex_triangles_sampled():
    rng = np.random.default_rng(21)
    for _ in range(10):
        n = int(rng.integers(3, 40))
        g = pins.with_noise(*G.gnp(n, 0.4, rng), rng)
        A = G.dense_adjacency(*g)
        expect = np.rint(np.einsum("ij,ji->i", A @ A, A) / 2).astype(np.int64)
        for x in range(n):
            assert oracle.vertex_triangles(*g, x) == expect[x]
    for k in range(3, 9):
        for x in range(k):
            assert oracle.vertex_triangles(*G.complete(k), x) == G.choose(k - 1, 2)


def _support_by_pair(g):
    """Oracle edge support keyed by the original endpoint pair (min, max)."""
    n = g[0]
    pr = oracle.prepare(*g)
    rp, ci, perm = pr["rowptr"], pr["colidx"], pr["perm"]
    sup = oracle.edge_support(n, rp, ci)
    out = {}
    for r in range(n):
        for e in range(int(rp[r]), int(rp[r + 1])):
            a, b = int(perm[r]), int(perm[ci[e]])
            out[(min(a, b), max(a, b))] = int(sup[e])
    return out, pr


def test_edge_support_closed_forms():
    for k in range(3, 10):
        sup, _ = _support_by_pair(G.complete(k))
        assert len(sup) == G.choose(k, 2) and set(sup.values()) == {k - 2}
    for k in range(4, 10):
        sup, _ = _support_by_pair(G.wheel(k))
        assert all(s == (2 if a == 0 else 1) for (a, b), s in sup.items())
    sup, _ = _support_by_pair(G.friendship(5))
    assert set(sup.values()) == {1}
    sizes = (2, 3, 4)
    part = np.repeat(np.arange(3), sizes)
    sup, _ = _support_by_pair(G.complete_multipartite(sizes))
    for (a, b), s in sup.items():
        third = 3 - part[a] - part[b]
        assert s == sizes[third]
    sup, _ = _support_by_pair(G.grid(4, 5))
    assert set(sup.values()) == {0}


def test_edge_support_brute_force():
    rng = np.random.default_rng(31)
    for _ in range(40):
        n = int(rng.integers(2, 30))
        g = pins.with_noise(*G.gnp(n, float(rng.uniform(0.1, 0.9)), rng), rng)
        A = G.dense_adjacency(*g)
        common = A @ A
        sup, pr = _support_by_pair(g)
        assert len(sup) == int(A.sum()) // 2
        for (a, b), s in sup.items():
            assert A[a, b] == 1 and s == common[a, b]
        T = oracle.tc_intersect(n, pr["rowptr"], pr["colidx"])
        assert sum(sup.values()) == 3 * T


@pytest.mark.parametrize("p", [2, 3, 6])
def test_pbd_pipeline_per_task(p):
    """Under the probe-based cuts, Alg. 5 and Alg. 6 per task equal the
    classification of every triangle into its task, and the total is unchanged."""
    rng = np.random.default_rng(40 + p)
    for _ in range(4):
        n = int(rng.integers(30, 120))
        g = G.gnp(n, float(rng.uniform(0.05, 0.4)), rng)
        T = G.brute_force_triangles(*g)
        r5 = oracle.bbtc(*g, p=p, method="intersect", partition="probe")
        r6 = oracle.bbtc(*g, p=p, method="hmap", partition="probe", prep=r5)
        c, _ = oracle.pbd_cuts(n, r5["rowptr"], r5["colidx"], p)
        assert np.array_equal(r5["cuts"], c)
        cls = oracle.classify_triangles(n, r5["rowptr"], r5["colidx"], p, c)
        assert r5["total"] == T and r6["total"] == T
        assert np.array_equal(r5["per_task"], cls) and np.array_equal(r6["per_task"], cls)


def test_pbd_lowers_imbalance_on_rmat():
    """Sec. 4.4: lambda = m_max / m_avg. On the skewed R-MAT scale-14 graph the
    probe-based partition must not be worse than the edge-balanced one."""
    n, rp, ci = graphgen.rmat(14, 16, 1)
    pr = oracle.prepare(n, rp, ci)
    for p in (2, 4, 8):
        ce = oracle.cuts(n, pr["rowptr"], p)
        cp, bstar = oracle.pbd_cuts(n, pr["rowptr"], pr["colidx"], p)
        me = oracle.block_nnz(n, pr["rowptr"], pr["colidx"], p, ce).max()
        mp = oracle.block_nnz(n, pr["rowptr"], pr["colidx"], p, cp).max()
        assert mp <= bstar and mp <= me
