"""The N>1 path of the benchmark is replicas: every rank renders its own frame, and the
whole-job throughput is all ranks' units over the slowest rank's time (max over ranks,
no data-path collective).  Checked here with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    r, w, _ = bench.dist_env()
    assert (r, w) == (rank, world)
    bench.barrier(world)
    seconds = 1.0 + rank  # rank 1 is the slow one
    value, t = bench.aggregate(10.0, seconds, world, device="cpu")
    out[rank] = (value, t)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        value, t = out[r]
        assert t == pytest.approx(2.0)
        assert value == pytest.approx(10.0 * world / 2.0)


def test_single_rank_aggregate_is_identity():
    import bench
    value, t = bench.aggregate(6.0, 3.0, 1)
    assert (value, t) == (2.0, 3.0)
