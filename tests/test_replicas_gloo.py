"""Multi-GPU runs are independent replicas: each rank solves its own instances and rank 0 reports all
ranks' solves over the slowest rank's time.  The host logic is checked with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [0.5, 1.25][rank]          # rank 1 is the slow one
    t_max = bench.max_over_ranks(local, dist, torch.device("cpu"))
    out[rank] = (t_max, bench.replica_value(10, world, t_max))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        assert out[0][0] == out[1][0] == 1.25
        assert out[0][1] == pytest.approx(20 / 1.25)


def test_single_process_needs_no_collective():
    import bench
    assert bench.max_over_ranks(0.7) == 0.7 and bench.replica_value(5, 1, 0.5) == 10.0
