"""The benchmark's N-replica aggregation on CPU ranks (gloo, world size 2):
barrier, maximum over ranks of the timed region, whole-job throughput."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    ms = [10.0, 14.5][rank]
    worst = bench.max_over_ranks(ms, dist, "cpu")
    out[rank] = (worst, bench.job_mlups(1000, 50, world, worst))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 14.5
    # 2 ranks x 1000 cells x 50 steps in 14.5 ms
    assert abs(out[0][1] - 2 * 1000 * 50 / (14.5 * 1e3)) < 1e-12


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.job_mlups(10, 10, 1, 1.0) == 0.1
