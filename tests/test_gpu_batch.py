"""Batched counting: each graph's count is the same alone and in a batch (GPU)."""
import ctypes

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


def small_batch(seed=0, k=24):
    rng = np.random.default_rng(seed)
    graphs = []
    for i in range(k):
        kind = i % 4
        if kind == 0:
            graphs.append(graphgen.rmat(int(rng.integers(5, 11)), int(rng.integers(4, 17)),
                                        int(rng.integers(0, 1000))))
        elif kind == 1:
            n = int(rng.integers(2, 300))
            graphs.append(graphgen.gnm(n, int(rng.integers(0, 4 * n)), int(rng.integers(0, 1000))))
        elif kind == 2:
            graphs.append(pins.with_noise(*G.gnp(int(rng.integers(3, 60)), 0.3, rng), rng))
        else:
            graphs.append(G.complete(int(rng.integers(3, 12))))
    graphs.append((0, np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32)))  # empty graph
    graphs.append((5, np.zeros(6, dtype=np.int64), np.zeros(0, dtype=np.int32)))  # no edges
    return graphs


def oracle_totals(graphs):
    out = []
    for n, rp, ci in graphs:
        pr = oracle.prepare(n, rp, ci)
        out.append(oracle.tc_hmap(n, pr["rowptr"], pr["colidx"]))
    return np.array(out, dtype=np.uint64)


@pytest.mark.parametrize("p", [1, 3, 8])
def test_create_batch_per_graph_counts(p):
    graphs = small_batch(p)
    expect = oracle_totals(graphs)
    with bb.BatchGraph(graphs) as batch:
        assert batch.info()["num_graphs"] == len(graphs)
        for kernel in ("intersect", "hashmap"):
            out = batch.count(p=p, kernel=kernel, per_graph=True, per_task=True)
            assert np.array_equal(out["per_graph"], expect)
            assert out["total"] == int(expect.sum()) == int(out["per_task"].sum())


def test_batch_is_the_same_as_alone():
    graphs = small_batch(11)
    alone = []
    for g in graphs:
        with bb.Graph(*g) as h:
            alone.append(h.count(p=2))
    with bb.BatchGraph(graphs) as batch:
        assert np.array_equal(batch.count(p=2, per_graph=True)["per_graph"],
                              np.array(alone, dtype=np.uint64))


def test_batch_rejects_entries_outside_their_graph():
    voff = np.array([0, 3, 6], dtype=np.int64)
    rowptr = np.array([0, 1, 2, 3, 4, 5, 6], dtype=np.int64)
    colidx = np.array([1, 2, 0, 1, 2, 3], dtype=np.int32)  # 3 is outside graph 1 (n = 3)
    with pytest.raises(bb.BbtcError) as e:
        bb.bbtc_graph_create_batch(voff, rowptr, colidx)
    assert e.value.status == 1
    with pytest.raises(bb.BbtcError):
        bb.bbtc_graph_create_batch(np.array([0, 3, 2], dtype=np.int64), rowptr, colidx)


def test_count_batch_of_handles():
    graphs = small_batch(5, k=40)
    expect = oracle_totals(graphs)
    handles = [bb.bbtc_graph_create(*g) for g in graphs]
    try:
        counts, stats = bb.bbtc_count_batch(handles, bb.make_opts(p=4))
        assert not stats.any()
        assert np.array_equal(counts, expect)
        # a NULL handle is reported for itself; the others are still counted
        with_null = handles[:3] + [0] + handles[3:6]
        counts, stats = bb.bbtc_count_batch(with_null, bb.make_opts(p=2))
        assert stats.tolist() == [0, 0, 0, 1, 0, 0, 0]
        assert np.array_equal(np.delete(counts, 3), expect[:6])
    finally:
        for h in handles:
            bb.bbtc_graph_destroy(h)


def test_count_async_and_cuda_graph_replay():
    n, rp, ci = graphgen.rmat(12, 16, 21)
    with bb.Graph(n, rp, ci) as g:
        expect = g.count(p=4, per_task=True)   # builds the plan
        nt = bb.bbtc_num_tasks(4)
        total = torch.zeros(1, dtype=torch.int64, device="cuda")
        per_task = torch.zeros(nt, dtype=torch.int64, device="cuda")
        stream = torch.cuda.Stream()
        opts = bb.make_opts(p=4, per_task_out=per_task, stream=stream)
        with torch.cuda.stream(stream):
            bb.bbtc_count_async(g.handle, opts, total)
        stream.synchronize()
        assert int(total.item()) == expect["total"]
        # capture the enqueue-only count and replay it
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg, stream=stream):
            bb.bbtc_count_async(g.handle, opts, total)
        for _ in range(3):
            total.zero_()
            per_task.zero_()
            cg.replay()
            torch.cuda.synchronize()
            assert int(total.item()) == expect["total"]
            assert np.array_equal(per_task.cpu().numpy().astype(np.uint64), expect["per_task"])
        # async without a matching plan is refused instead of building one
        with pytest.raises(bb.BbtcError):
            bb.bbtc_count_async(g.handle, bb.make_opts(p=5), total)


def test_batch_async_capture_per_graph():
    graphs = small_batch(9)
    expect = oracle_totals(graphs)
    with bb.BatchGraph(graphs) as batch:
        batch.count(p=2, per_graph=True)
        pg = torch.zeros(len(graphs), dtype=torch.int64, device="cuda")
        total = torch.zeros(1, dtype=torch.int64, device="cuda")
        stream = torch.cuda.Stream()
        opts = bb.make_opts(p=2, per_graph_out=pg, stream=stream)
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg, stream=stream):
            bb.bbtc_count_async(batch.handle, opts, total)
        cg.replay()
        torch.cuda.synchronize()
        assert np.array_equal(pg.cpu().numpy().astype(np.uint64), expect)


def test_chunk_sizes_give_identical_counts():
    n, rp, ci = graphgen.rmat(13, 16, 6)
    with bb.Graph(n, rp, ci) as g:
        ref = g.count(p=3, per_task=True)
        for chunk in (1, 7, 64, 100000):
            out = g.count(p=3, per_task=True, chunk=chunk)
            assert out["total"] == ref["total"]
            assert np.array_equal(out["per_task"], ref["per_task"])


def test_timeout_is_reported_and_the_handle_stays_usable():
    # the counting kernel stops taking work once its time limit has passed; a
    # 1 ms limit on a graph whose count takes far longer must end in ETIMEOUT
    n, rp, ci = graphgen.rmat(21, 16, 2)
    with bb.Graph(n, rp, ci, symmetric=True) as g:
        full = g.count(p=1)
        with pytest.raises(bb.BbtcError) as e:
            g.count(p=1, timeout_ms=1, chunk=64)
        assert e.value.status == 4
        assert g.count(p=1) == full


def test_per_task_cycles_and_estimator_study():
    from paper_2009_12457_gb300 import workload
    n, rp, ci = graphgen.rmat(14, 16, 1)
    with bb.Graph(n, rp, ci) as g:
        ref = g.count(p=4, per_task=True)
        out = g.count(p=4, per_task=True, per_task_cycles=True)
        assert np.array_equal(out["per_task"], ref["per_task"])  # measuring changes no count
        cyc = out["per_task_cycles"]
        plan = g.plan(4)
        nnz = plan["block_nnz"]
        tl = plan["tasks"]
        has_work = np.array([nnz[i, j] > 0 and nnz[i, k] > 0 and nnz[j, k] > 0 for i, j, k in tl])
        assert np.all(cyc[has_work] > 0) and np.all(cyc[~has_work] == 0)
        s = workload.study(g, p=4, repeats=1)
        assert set(s["coverage"]) == {"nnz", "density", "degree", "bbtc"}
        assert all(0 < v <= 1.0 for c in s["coverage"].values() for v in c.values())


def test_count_batch_each_handle_keeps_its_plan():
    # resident batches count every handle through its own plan in one launch:
    # automatic p per handle, repeated handles, mixed kernels, plans built
    # earlier with other options, and the union path under a device budget
    graphs = small_batch(17, k=20) + [graphgen.rmat(14, 16, 3), graphgen.rmat(13, 8, 4)]
    expect = oracle_totals(graphs)
    handles = [bb.bbtc_graph_create(*g) for g in graphs]
    try:
        bb.bbtc_graph_plan(handles[-1], bb.make_opts(p=7, kernel="hashmap"))
        bb.bbtc_count(handles[-2], bb.make_opts(p=3))
        for opts in (bb.make_opts(), bb.make_opts(p=5, kernel="intersect"),
                     bb.make_opts(p=2, kernel="hashmap", chunk=16),
                     bb.make_opts(p=3, device_budget_bytes=1 << 30)):
            counts, stats = bb.bbtc_count_batch(handles, opts)
            assert not stats.any()
            assert np.array_equal(counts, expect)
        twice = handles[-3:] + handles[-3:]
        counts, _ = bb.bbtc_count_batch(twice, bb.make_opts(p=4))
        assert np.array_equal(counts, np.concatenate([expect[-3:], expect[-3:]]))
    finally:
        for h in handles:
            bb.bbtc_graph_destroy(h)


def test_plan_then_async_without_a_count():
    n, rp, ci = graphgen.rmat(12, 16, 8)
    with bb.Graph(n, rp, ci) as g:
        opts = bb.make_opts(p=3)
        bb.bbtc_graph_plan(g.handle, opts)
        total = torch.zeros(1, dtype=torch.int64, device="cuda")
        bb.bbtc_count_async(g.handle, opts, total)
        torch.cuda.synchronize()
        assert int(total.item()) == oracle_totals([(n, rp, ci)])[0]


def test_symmetric_batch_fast_path_matches_oracle():
    # symmetric batches with sorted rows take the per-row preparation path;
    # each graph keeps its own order and orientation inside the union
    graphs = [graphgen.rmat(s, 8 + 2 * s, 40 + s) for s in range(5, 12)]
    graphs += [graphgen.gnm(n, 6 * n, n) for n in (10, 200, 3000)]
    graphs.append((4, np.zeros(5, dtype=np.int64), np.zeros(0, dtype=np.int32)))
    graphs.append(G.complete(40))
    expect = oracle_totals(graphs)
    with bb.BatchGraph(graphs, symmetric=True) as batch:
        for p in (1, 3):
            out = batch.count(p=p, per_graph=True, per_vertex=True)
            assert np.array_equal(out["per_graph"], expect)
        o = batch.oriented()
        with bb.BatchGraph(graphs) as general:
            og = general.oriented()
        assert np.array_equal(o["rowptr"], og["rowptr"])
        assert np.array_equal(o["colidx"], og["colidx"])
        assert np.array_equal(o["perm"], og["perm"])
    # an entry outside its own graph is rejected on this path too
    voff = np.array([0, 3, 6], dtype=np.int64)
    rowptr = np.array([0, 1, 2, 3, 4, 5, 6], dtype=np.int64)
    colidx = np.array([1, 2, 0, 1, 2, 3], dtype=np.int32)
    with pytest.raises(bb.BbtcError) as e:
        bb.bbtc_graph_create_batch(voff, rowptr, colidx, bb.INPUT_SYMMETRIC)
    assert e.value.status == 1
