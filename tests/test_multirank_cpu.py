"""The multi-GPU path is replicas only: each rank advances its own lattice and
the ranks meet only around the timed region (a barrier and the maximum of
their times).  This checks that host logic with two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
    dist.barrier()
    got = bench.max_over_ranks(ms, dist, "cpu")
    out[rank] = got
    dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    assert out[0] == out[1] == 15.0


def test_job_rate_counts_every_replica():
    import bench
    # two replicas of 1024 x 2048 nodes, 100 steps in 10 ms -> 4.19e4 MLUPS
    assert bench.job_mlups(2, 1024 * 2048, 100, 10.0) == pytest.approx(2 * 1024 * 2048 * 100 / 1e4)
    assert bench.max_over_ranks(3.5) == 3.5
