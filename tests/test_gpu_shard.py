"""Counting a share of the task list (opts.task_mask) on the GPU: the count of a
share is the sum of its tasks' exact counts, and disjoint shares that cover the
task list add up to the graph's count (Sec. 4.2: the tasks are independent)."""
import numpy as np
import pytest

import graphgen
import oracle
import paper_2009_12457_gb300 as bb
from paper_2009_12457_gb300 import shard

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def test_shares_add_up_resident_and_streamed():
    n, rp, ci = graphgen.rmat(14, 16, 1)
    p = 5
    ref = oracle.bbtc(n, rp, ci, p=p)
    with bb.Graph(n, rp, ci) as g:
        est = g.plan(p)["exec_time"]
        assert np.array_equal(est, ref["exec_time"])
        for world in (2, 3):
            masks = shard.lpt_masks(est, world)
            parts = []
            for m in masks:
                pt = np.zeros(bb.bbtc_num_tasks(p), dtype=np.uint64)
                total = bb.bbtc_count(g.handle, bb.make_opts(p=p, task_mask=m, per_task_out=pt))
                keep = m.astype(bool)
                assert total == int(ref["per_task"][keep].sum())
                assert np.array_equal(pt[keep], ref["per_task"][keep])
                assert not np.any(pt[~keep])
                parts.append(total)
            assert sum(parts) == ref["total"]
        # the same shares with the blocks streamed through a small device pool
        m0, m1 = shard.lpt_masks(est, 2)
        budget = 3 << 20
        a = bb.bbtc_count(g.handle, bb.make_opts(p=p, task_mask=m0, device_budget_bytes=budget))
        b = bb.bbtc_count(g.handle, bb.make_opts(p=p, task_mask=m1, device_budget_bytes=budget))
        assert a + b == ref["total"]
        assert a == int(ref["per_task"][m0.astype(bool)].sum())
        # one rank alone counts everything
        assert shard.shard_count(g.handle, p, 0, 1) == ref["total"]
        # an all-zero mask counts nothing
        assert bb.bbtc_count(g.handle, bb.make_opts(
            p=p, task_mask=np.zeros(bb.bbtc_num_tasks(p), dtype=np.uint8))) == 0


def test_async_refuses_a_task_mask():
    n, rp, ci = graphgen.rmat(10, 8, 2)
    with bb.Graph(n, rp, ci) as g:
        g.count(p=2)
        total = torch.zeros(1, dtype=torch.int64, device="cuda")
        with pytest.raises(bb.BbtcError):
            bb.bbtc_count_async(g.handle, bb.make_opts(p=2, task_mask=np.ones(4, np.uint8)),
                                total)
