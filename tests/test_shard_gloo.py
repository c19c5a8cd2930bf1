"""One graph's task list shared over CPU ranks (gloo): the multi-GPU form of
Alg. 7 / Alg. 9, checked with the oracle's per-task counts (no GPU needed).

Each rank takes its longest-processing-time-first share of the tasks by the
Sec. 5 estimate, sums the oracle's counts of those tasks, and the ranks' sums
are added with one all-reduce: the result must be the graph's count."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import graphgen
import oracle
from paper_2009_12457_gb300 import shard

P_LIST = (1, 3, 5, 8)


def _reference():
    n, rp, ci = graphgen.rmat(11, 8, 7)
    pr = oracle.prepare(n, rp, ci)
    out = {"total": oracle.tc_intersect(n, pr["rowptr"], pr["colidx"])}
    for p in P_LIST:
        c = oracle.cuts(n, pr["rowptr"], p)
        nnz = oracle.block_nnz(n, pr["rowptr"], pr["colidx"], p, c)
        out[p] = (oracle.exec_time(p, c, nnz),
                  oracle.classify_triangles(n, pr["rowptr"], pr["colidx"], p, c))
    return out


def _rank_main(rank, world, port, ref, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = {}
        for p in P_LIST:
            est, per_task = ref[p]
            mask = shard.lpt_masks(est, world)[rank].astype(bool)
            t = torch.tensor([int(per_task[mask].sum())], dtype=torch.int64)
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
            res[p] = int(t.item())
        out[rank] = res
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_shares_of_the_task_list_add_up_to_the_count(world):
    ref = _reference()
    port = 29600 + (os.getpid() % 2000) + world
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, port, ref, out), nprocs=world, join=True)
    for r in range(world):
        assert out[r] == {p: ref["total"] for p in P_LIST}


def test_lpt_masks_partition_and_balance():
    rng = np.random.default_rng(3)
    for world in (1, 2, 3, 8):
        for nt in (1, 4, 20, 120, 816):
            est = rng.exponential(1.0, nt) * (rng.random(nt) < 0.8)
            masks = shard.lpt_masks(est, world)
            cover = np.sum(np.stack(masks), axis=0)
            assert np.all(cover == 1)  # every task in exactly one share
            loads = shard.mask_loads(est, masks)
            # Graham's bound for greedy LPT: no share exceeds the mean by more
            # than one task
            assert max(loads) <= est.sum() / world + est.max() + 1e-9
    # by hand, estimates 5, 4, 3, 3, 2 over two ranks: 5 -> rank 0; 4 -> rank 1; the
    # first 3 -> rank 1 (load 4 < 5); the second 3 -> rank 0 (5 < 7); 2 -> rank 1 (7 < 8)
    masks = shard.lpt_masks([5, 4, 3, 3, 2], 2)
    assert masks[0].tolist() == [1, 0, 0, 1, 0] and masks[1].tolist() == [0, 1, 1, 0, 1]


def _rank_shard_count(rank, world, port, ref, out):
    """shard.shard_count's own steps (plan, estimate, share, count, one sum) on a
    gloo rank, with the library's calls answered from the oracle's values."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_2009_12457_gb300 as bb
        planned = []
        bb.bbtc_graph_plan = lambda h, o: planned.append(o["p"])
        bb.bbtc_graph_get_plan = lambda h, p: {"exec_time": ref[p][0]}
        bb.make_opts = lambda **kw: kw
        bb.bbtc_count = lambda h, o: int(ref[o["p"]][1][np.asarray(o["task_mask"]).astype(bool)].sum())
        res = {p: shard.shard_count(0, p, rank, world, dist) for p in P_LIST}
        out[rank] = (res, planned)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_shard_count_over_gloo_ranks(world):
    ref = _reference()
    port = 31700 + (os.getpid() % 2000) + world
    out = mp.Manager().dict()
    mp.spawn(_rank_shard_count, args=(world, port, ref, out), nprocs=world, join=True)
    for r in range(world):
        res, planned = out[r]
        assert res == {p: ref["total"] for p in P_LIST}
        assert planned == list(P_LIST)  # the plan is built before its estimate is read
