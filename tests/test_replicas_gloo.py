"""Multi-GPU form is replicas only: the bench's cross-rank steps on CPU ranks (gloo)."""
import os

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r "took" 10 + r ms; the job time is the slowest rank's
        ms = bench.reduce_max_ms(10.0 + rank, dist, "cpu")
        dist.barrier()
        out[rank] = ms
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_max_over_ranks_and_whole_job_rate(world):
    port = 29500 + (os.getpid() % 2000)
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    assert [out[r] for r in range(world)] == [10.0 + world - 1] * world
    # each replica counts the whole graph: the job processes world x m edges
    assert bench.replica_throughput(1000, world, 11.0) == pytest.approx(world * 1000 / 0.011)


def test_single_rank_needs_no_collective():
    assert bench.reduce_max_ms(7.5, None, "cpu") == 7.5
