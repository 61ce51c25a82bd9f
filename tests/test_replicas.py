"""The multi-GPU path of the bench is replicas (one graph per rank, no collective on the data
path): the job's time is the slowest rank's and its work the sum of the ranks'. Checked with
two gloo ranks on the CPU."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed, edges = bench.reduce_over_ranks(10.0 + 5.0 * rank, 100 * (rank + 1), world)
    out[rank] = (elapsed, edges)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_replicas_take_the_slowest_rank_and_the_sum_of_the_work():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(90)
            assert p.exitcode == 0
        for r in range(world):
            assert out[r] == (15.0, 300)


def test_single_rank_is_unchanged():
    import bench
    assert bench.reduce_over_ranks(12.5, 77, 1) == (12.5, 77)
