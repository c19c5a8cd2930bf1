"""One graph's task list shared over ranks (the multi-GPU form of Alg. 7 / Alg. 9).

The tasks (i, j, k) are independent (Sec. 4.2): a rank that counts a subset of
them gets their exact per-task counts, and the ranks' totals add up to the
graph's count. The tasks are dealt longest-processing-time first: in the
order of the Sec. 5 estimate (non-increasing, ties in Alg. 4 order), each task
goes to the rank with the least estimated work so far (ties to the lower
rank). The final sum of one uint64 per rank is the only exchange.
"""
from __future__ import annotations

import heapq

import numpy as np


def lpt_masks(estimates, world: int) -> list[np.ndarray]:
    """One uint8 mask per rank over the tasks (Alg. 4 order): 1 where the rank
    counts the task. Every task is in exactly one mask."""
    est = np.asarray(estimates, dtype=np.float64)
    if world < 1:
        raise ValueError("world must be >= 1")
    masks = [np.zeros(est.shape[0], dtype=np.uint8) for _ in range(world)]
    order = np.argsort(-est, kind="stable")  # non-increasing, ties by task index
    heap = [(0.0, r) for r in range(world)]
    for t in order:
        load, r = heapq.heappop(heap)
        masks[r][t] = 1
        heapq.heappush(heap, (load + float(est[t]), r))
    return masks


def mask_loads(estimates, masks) -> list[float]:
    """Estimated work of each rank's share."""
    est = np.asarray(estimates, dtype=np.float64)
    return [float(est[m.astype(bool)].sum()) for m in masks]


def shard_count(handle: int, p: int, rank: int, world: int, dist=None, device=None,
                **count_opts) -> int:
    """Counts this rank's share of the handle's tasks for p and sums the shares of
    all ranks with `dist` (torch.distributed, any backend; None for one rank).
    Returns the whole graph's count on every rank."""
    import torch

    from . import bbtc_count, bbtc_graph_get_plan, bbtc_graph_plan, make_opts

    bbtc_graph_plan(handle, make_opts(p=p, **count_opts))  # the plan the count will use
    est = bbtc_graph_get_plan(handle, p)["exec_time"]
    mask = lpt_masks(est, world)[rank]
    local = bbtc_count(handle, make_opts(p=p, task_mask=mask, **count_opts))
    if dist is None or world == 1:
        return local
    t = torch.tensor([local], dtype=torch.int64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return int(t.item())
