"""Parity of the CUDA library with the CPU oracle, element by element (GPU).

All comparisons are exact: every quantity is an integer except the task
estimate, which both sides compute with the same IEEE double operations.
"""
import numpy as np
import pytest

import graphgen
import oracle
import paper_2009_12457_gb300 as bb
from tests import graphs as G
from tests import pins

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

KERNELS = ("intersect", "hashmap", "auto")


def check_against_oracle(g, ps, kernels=KERNELS, per_vertex=True):
    n, rp, ci = g
    ref = oracle.prepare(n, rp, ci)
    with bb.Graph(n, rp, ci) as dev:
        info = dev.info()
        assert info["n"] == n and info["m"] == ref["m"]
        ori = dev.oriented()
        assert np.array_equal(ori["rowptr"], ref["rowptr"])
        assert np.array_equal(ori["colidx"], ref["colidx"])
        assert np.array_equal(ori["perm"], ref["perm"])
        assert np.array_equal(ori["degree"], ref["deg"])
        total = oracle.tc_hmap(n, ref["rowptr"], ref["colidx"])
        pv_ref = oracle.per_vertex(n, ref["rowptr"], ref["colidx"], ref["perm"]) if per_vertex else None
        for p in ps:
            r = oracle.bbtc(n, rp, ci, p=p, prep=ref)
            plan = dev.plan(p)
            assert np.array_equal(plan["cuts"], r["cuts"])
            assert np.array_equal(plan["block_nnz"], r["block_nnz"])
            assert np.array_equal(plan["tasks"], r["tasks"])
            assert np.array_equal(plan["exec_time"], r["exec_time"])  # same IEEE ops
            assert np.array_equal(plan["order"], r["order"])
            for kern in kernels:
                out = dev.count(p=p, kernel=kern, per_task=True, per_vertex=per_vertex)
                assert out["total"] == total == r["total"]
                assert np.array_equal(out["per_task"], r["per_task"])
                if per_vertex:
                    assert np.array_equal(out["per_vertex"], pv_ref)
        return total


def test_closed_forms():
    cases = [(G.complete(k), G.choose(k, 3)) for k in (3, 4, 7, 12, 33)]
    cases += [(G.wheel(k), k) for k in (4, 9, 40)]
    cases += [(G.friendship(k), k) for k in (1, 3, 17)]
    cases += [(G.complete_multipartite([3, 4, 5]), 60), (G.complete_multipartite([6, 7]), 0),
              (G.grid(9, 11), 0), (G.cycle(10), 0), (G.cycle(3), 1),
              (G.random_tree(200, np.random.default_rng(4)), 0)]
    for g, expect in cases:
        with bb.Graph(*g) as dev:
            for p in (1, 2, 3, 5, 8):
                for kern in KERNELS:
                    out = dev.count(p=p, kernel=kern, per_task=True, per_vertex=True)
                    assert out["total"] == expect
                    assert int(out["per_task"].sum()) == expect
                    assert int(out["per_vertex"].sum()) == 3 * expect


def test_complete_graph_per_vertex():
    for k in (5, 20, 64):
        with bb.Graph(*G.complete(k)) as dev:
            pv = dev.count(p=3, per_vertex=True)["per_vertex"]
            assert np.all(pv == G.choose(k - 1, 2))


@pytest.mark.parametrize("seed", range(6))
def test_random_graphs_with_noise(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(5, 400))
    g = pins.with_noise(*G.gnp(n, float(rng.uniform(0.02, 0.5)), rng), rng, dup=0.2, loops=4)
    check_against_oracle(g, ps=(1, 2, 3, 4, 7))


def test_config1_rmat_scale14():
    """R-MAT scale 14, edge factor 16, seed 1 at p=2 (and other p), all kernels."""
    g = graphgen.rmat_s14()
    total = check_against_oracle(g, ps=(2, 1, 3, 8, 16))
    assert total == 2838931  # tests/golden/config_counts.txt


def test_p_up_to_64_and_empty_parts():
    g = graphgen.gnm(300, 900, 7)
    check_against_oracle(g, ps=(17, 64), kernels=("auto",))
    tiny = G.complete(5)
    check_against_oracle(tiny, ps=(8, 64), kernels=("intersect", "hashmap"))


def test_multi_tile_ragged_sizes():
    # entry counts that span several sort tiles (4096 keys) and end mid-tile
    for n, pairs in ((5000, 4096 * 3 + 17), (70000, 200003)):
        g = graphgen.gnm(n, pairs, pairs)
        check_against_oracle(g, ps=(1, 5), kernels=("auto",))


def test_degenerate_inputs():
    empty0 = (0, np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32))
    one = (1, np.zeros(2, dtype=np.int64), np.zeros(0, dtype=np.int32))
    isolated = (6, np.zeros(7, dtype=np.int64), np.zeros(0, dtype=np.int32))
    loops = G.csr_from_edges(4, [(0, 0), (1, 1), (2, 2)], both_directions=False)
    for g in (empty0, one, isolated, loops):
        with bb.Graph(*g) as dev:
            assert dev.info()["m"] == 0
            for p in (1, 4):
                out = dev.count(p=p, per_task=True, per_vertex=True)
                assert out["total"] == 0
                assert not out["per_task"].any() and not out["per_vertex"].any()


def test_one_direction_unsorted_and_symmetric_flag():
    rng = np.random.default_rng(8)
    base = G.gnp(120, 0.2, rng)
    T = G.trace_cubed_over_six(*base)
    A = G.dense_adjacency(*base)
    a, b = np.nonzero(np.triu(A, 1))
    flip = rng.random(a.shape[0]) < 0.5
    one = G.csr_from_edges(120, list(zip(np.where(flip, a, b).tolist(),
                                         np.where(flip, b, a).tolist())), both_directions=False)
    with bb.Graph(*one) as dev:
        assert dev.count(p=3) == T
    with bb.Graph(*base, symmetric=True) as dev:
        assert dev.count(p=3) == T
    noisy = pins.with_noise(*base, rng)
    with bb.Graph(*noisy) as dev:
        assert dev.count(p=2) == T


def test_device_input_matches_host_input():
    n, rp, ci = graphgen.rmat(12, 8, 3)
    with bb.Graph(n, rp, ci) as host:
        expect = host.count(p=4, per_task=True)
    drp = torch.from_numpy(rp).cuda()
    dci = torch.from_numpy(ci).cuda()
    with bb.Graph(n, drp, dci) as dev:
        got = dev.count(p=4, per_task=True)
    assert got["total"] == expect["total"]
    assert np.array_equal(got["per_task"], expect["per_task"])
    # device-resident outputs
    pt = torch.zeros(bb.bbtc_num_tasks(4), dtype=torch.int64, device="cuda")
    with bb.Graph(n, drp, dci) as dev:
        opts = bb.make_opts(p=4, per_task_out=pt)
        total = bb.bbtc_count(dev.handle, opts)
    assert total == expect["total"]
    assert np.array_equal(pt.cpu().numpy().astype(np.uint64), expect["per_task"])


def test_relabel_and_disjoint_union():
    rng = np.random.default_rng(12)
    n, rp, ci = graphgen.rmat(11, 8, 5)
    with bb.Graph(n, rp, ci) as dev:
        T = dev.count(p=3)
    perm = rng.permutation(n).astype(np.int32)
    rows = np.repeat(np.arange(n), np.diff(rp))
    relabelled = graphgen.pairs_to_csr(n, perm[rows], perm[ci])
    # every input entry becomes a pair listed under both endpoints: the simple
    # graph is the relabelled original
    with bb.Graph(*relabelled) as dev:
        assert dev.count(p=5) == T
    union = graphgen.pairs_to_csr(2 * n, np.concatenate([rows, rows + n]).astype(np.int32),
                                  np.concatenate([ci, ci + n]).astype(np.int32))
    with bb.Graph(*union) as dev:
        assert dev.count(p=4) == 2 * T


def test_invalid_inputs_are_rejected():
    rp = np.array([0, 2, 1, 3], dtype=np.int64)   # decreasing
    ci = np.array([1, 2, 0], dtype=np.int32)
    with pytest.raises(bb.BbtcError) as e:
        bb.Graph(3, rp, ci)
    assert e.value.status == 1
    rp = np.array([0, 1, 2, 3], dtype=np.int64)
    ci = np.array([1, 7, 0], dtype=np.int32)       # out of range
    with pytest.raises(bb.BbtcError) as e:
        bb.Graph(3, rp, ci)
    assert e.value.status == 1
    rp = np.array([1, 1, 2, 3], dtype=np.int64)    # rowptr[0] != 0 (rowptr[n] = 3 entries)
    ci = np.array([1, 2, 0], dtype=np.int32)
    with pytest.raises(bb.BbtcError):
        bb.Graph(3, rp, ci)
    with bb.Graph(*G.complete(4)) as dev:
        with pytest.raises(bb.BbtcError):
            dev.count(p=65)
        with pytest.raises(bb.BbtcError):
            dev.count(p=-1)
        with pytest.raises(bb.BbtcError) as e:
            dev.count(p=2, partition=2)                # not a bbtc_partition
        assert e.value.status == 1
        assert dev.count(p=2) == 4  # the handle still works after a rejected call


def test_symmetric_fast_path_matches_general_path():
    """Symmetric sorted rows take the per-row path; unsorted rows and the
    general path must give the byte-identical oriented CSR."""
    rng = np.random.default_rng(31)
    for n, rp, ci in (graphgen.rmat(13, 16, 8), graphgen.gnm(3000, 20000, 9),
                      pins.with_noise(*G.gnp(90, 0.2, rng), rng)):
        sym_sorted = (n, rp, np.concatenate([np.sort(ci[rp[v]:rp[v + 1]]) for v in range(n)]
                                            or [np.zeros(0, np.int32)]).astype(np.int32))
        shuffled = (n, rp, ci.copy())
        for v in range(n):
            rng.shuffle(shuffled[2][rp[v]:rp[v + 1]])
        ref = oracle.prepare(n, rp, ci)
        for g, sym in ((sym_sorted, True), (shuffled, True), ((n, rp, ci), False)):
            with bb.Graph(*g, symmetric=sym) as dev:
                ori = dev.oriented()
                assert np.array_equal(ori["rowptr"], ref["rowptr"])
                assert np.array_equal(ori["colidx"], ref["colidx"])
                assert np.array_equal(ori["perm"], ref["perm"])
                assert np.array_equal(ori["degree"], ref["deg"])
                assert dev.info()["dplus_max"] == int(np.diff(ref["rowptr"]).max(initial=0))


def test_rows_longer_than_the_shared_sort():
    # K_2100: equal degrees, ties by id, so vertex 0 has 2099 out-neighbours
    k = 2100
    with bb.Graph(*G.complete(k), symmetric=True) as dev:
        assert dev.info()["dplus_max"] == k - 1
        assert dev.count(p=3) == G.choose(k, 3)


@pytest.mark.parametrize("p", [1, 3, 8])
def test_per_edge_support_matches_oracle(p):
    cases = [graphgen.rmat(12, 16, 5), G.complete(9), G.wheel(11), graphgen.gnm(3000, 40000, 4)]
    for n, rp, ci in cases:
        pr = oracle.prepare(n, rp, ci)
        expect = oracle.edge_support(n, pr["rowptr"], pr["colidx"])
        with bb.Graph(n, rp, ci) as g:
            for kernel in ("auto", "intersect", "hashmap"):
                out = g.count(p=p, kernel=kernel, per_edge=True, per_vertex=True)
                assert np.array_equal(out["per_edge"], expect), (n, p, kernel)
                assert int(out["per_edge"].sum()) == 3 * out["total"]
        # the same edges seen from the original ids
        with bb.Graph(n, rp, ci) as g:
            u, v, s = g.edge_support(p=p)
        assert np.array_equal(u, pr["perm"][np.repeat(np.arange(n), np.diff(pr["rowptr"]))])
        assert np.array_equal(s, expect)


def test_per_edge_support_large_sampled():
    # scale 18: edges whose support the oracle recomputes one by one
    n, rp, ci = graphgen.rmat(18, 16, 7)
    with bb.Graph(n, rp, ci, symmetric=True) as g:
        total = g.count(p=4)
        u, v, s = g.edge_support(p=4)
    assert int(s.sum()) == 3 * total
    rng = np.random.default_rng(2)
    for e in rng.choice(len(s), 200, replace=False):
        a, b = int(u[e]), int(v[e])
        na = set(ci[rp[a]:rp[a + 1]].tolist()) - {a}
        nb = set(ci[rp[b]:rp[b + 1]].tolist()) - {b}
        assert s[e] == len(na & nb), (a, b)


def check_probe_partition(g, ps):
    """Probe-based partition: cuts, block sizes, per-task and total counts equal the
    oracle's (bbtc_graph_plan with the partition, then the plan read back)."""
    n, rp, ci = g
    ref = oracle.prepare(n, rp, ci)
    with bb.Graph(n, rp, ci) as dev:
        for p in ps:
            r = oracle.bbtc(n, rp, ci, p=p, prep=ref, partition="probe")
            plan = dev.plan(p, partition="probe")
            assert np.array_equal(plan["cuts"], r["cuts"]), (p, plan["cuts"], r["cuts"])
            assert np.array_equal(plan["block_nnz"], r["block_nnz"])
            assert np.array_equal(plan["exec_time"], r["exec_time"])
            assert np.array_equal(plan["order"], r["order"])
            for kern in KERNELS:
                out = dev.count(p=p, kernel=kern, per_task=True, partition="probe")
                assert out["total"] == r["total"]
                assert np.array_equal(out["per_task"], r["per_task"])
            # and back to the edge-balanced partition on the same handle
            assert np.array_equal(dev.plan(p, partition="edges")["cuts"],
                                  oracle.cuts(n, ref["rowptr"], p))


def test_probe_partition_config1():
    check_probe_partition(graphgen.rmat_s14(), (1, 2, 3, 4, 8, 16))


@pytest.mark.parametrize("seed", range(4))
def test_probe_partition_random(seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(1, 500))
    g = pins.with_noise(*G.gnp(n, float(rng.uniform(0.0, 0.4)), rng), rng, dup=0.2, loops=3)
    check_probe_partition(g, (1, 2, 5, 7))


def test_probe_partition_edge_cases():
    check_probe_partition(G.csr_from_edges(10, []), (1, 3))        # no edges
    check_probe_partition(G.complete(3), (1, 2, 4))                # more parts than vertices
    two_k64 = G.csr_from_edges(128, [(a + o, b + o) for o in (0, 64)
                                      for a in range(64) for b in range(a + 1, 64)])
    check_probe_partition(two_k64, (2, 3))
    # p = 64 (2048 grains) on an R-MAT graph of scale 12
    check_probe_partition(graphgen.rmat(12, 16, 9), (64,))


def test_wide_lists_hash_and_sorted_staging():
    """G(n,m) with n = 200,000 and 6 M pairs: degrees are near uniform, so the
    degree order spreads each out-list over most positions above it. About 62%
    of the probes go to lists whose value range is wider than the 65,536-bit
    bitmap and which are longer than 16: AUTO and HASHMAP stage those as hash
    tables; AUTO with a high threshold and INTERSECT stage them sorted. Every
    staged form must give the oracle's per-task counts."""
    n, rp, ci = graphgen.gnm(200000, 6000000, 78)
    ref = oracle.prepare(n, rp, ci)
    with bb.Graph(n, rp, ci, symmetric=True) as dev:
        for p in (1, 4):
            r = oracle.bbtc(n, rp, ci, p=p, prep=ref)
            for kern, thr in (("auto", 0), ("hashmap", 0), ("auto", 1 << 20), ("intersect", 0)):
                out = dev.count(p=p, kernel=kern, hash_threshold=thr, per_task=True)
                assert out["total"] == r["total"] == 36183, (p, kern, thr)
                assert np.array_equal(out["per_task"], r["per_task"]), (p, kern, thr)
        # per-vertex counts take the single-probe loop through the same staged forms
        pv_ref = oracle.per_vertex(n, ref["rowptr"], ref["colidx"], ref["perm"])
        for kern in ("auto", "hashmap"):
            out = dev.count(p=2, kernel=kern, per_vertex=True)
            assert np.array_equal(out["per_vertex"], pv_ref), kern
