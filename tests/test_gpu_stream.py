"""Counting under a device budget (blocks streamed from pinned host memory) (GPU)."""
import numpy as np
import pytest

import graphgen
import oracle
import paper_2009_12457_gb300 as bb

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def block_bytes(g, p):
    """Bytes of the streamed block arrays for p (columns, in-edges, row pointers)."""
    info = g.info()
    return 16 * info["m"] + 4 * info["n"] * (p + 1)


@pytest.mark.parametrize("p", [1, 3, 6])
def test_streamed_equals_resident(p):
    n, rp, ci = graphgen.rmat(14, 16, 1)
    ref = oracle.bbtc(n, rp, ci, p=p, want_per_vertex=True)
    with bb.Graph(n, rp, ci) as g:
        total_blocks = block_bytes(g, p)
        for frac in (4.0, 1.0, 0.3):
            budget = int(total_blocks * frac)
            try:
                out = g.count(p=p, per_task=True, per_vertex=True,
                              device_budget_bytes=budget)
            except bb.BbtcError as e:
                # a single task's blocks may not fit in half of a small budget
                assert e.status == 2
                continue
            assert out["total"] == ref["total"]
            assert np.array_equal(out["per_task"], ref["per_task"])
            assert np.array_equal(out["per_vertex"], ref["per_vertex"])
            tim = g.timings()
            assert tim["stream_rounds"] >= 1 and tim["stream_h2d_bytes"] > 0
        # back to resident counting on the same handle
        assert g.count(p=p) == ref["total"]


def test_many_rounds_and_too_small_budget():
    n, rp, ci = graphgen.rmat(15, 16, 4)
    with bb.Graph(n, rp, ci) as g:
        ref = g.count(p=8, per_task=True)
        # the largest task (three blocks) must fit in half the budget
        out = g.count(p=8, per_task=True, device_budget_bytes=block_bytes(g, 8) // 2)
        assert out["total"] == ref["total"]
        assert np.array_equal(out["per_task"], ref["per_task"])
        assert g.timings()["stream_rounds"] > 1
        with pytest.raises(bb.BbtcError) as e:
            g.count(p=8, device_budget_bytes=4096)
        assert e.value.status == 2
        assert g.count(p=8) == ref["total"]


def test_streamed_batch_per_graph():
    graphs = [graphgen.rmat(s, 8, 10 + s) for s in range(6, 13)]
    alone = []
    for gr in graphs:
        with bb.Graph(*gr) as h:
            alone.append(h.count(p=2))
    with bb.BatchGraph(graphs) as batch:
        out = batch.count(p=4, per_graph=True, device_budget_bytes=block_bytes(batch, 4))
        assert np.array_equal(out["per_graph"], np.array(alone, dtype=np.uint64))


def test_async_refuses_a_streamed_plan():
    n, rp, ci = graphgen.rmat(12, 8, 2)
    with bb.Graph(n, rp, ci) as g:
        g.count(p=2, device_budget_bytes=1 << 30)
        total = torch.zeros(1, dtype=torch.int64, device="cuda")
        with pytest.raises(bb.BbtcError):
            bb.bbtc_count_async(g.handle, bb.make_opts(p=2), total)
