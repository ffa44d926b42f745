"""World-size-2 check of the benchmark's multi-rank path on CPU (gloo): each
rank is an independent replica; the job takes the slowest rank's time and
reports the aggregate rate.  The reference arm runs on rank 0 only."""
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
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, lr = bench.dist_setup()
    assert (w, r, lr) == (world, rank, rank)
    dist.barrier()
    local_ms = 10.0 * (rank + 1)                 # rank 1 is the slow one
    ms = bench.max_over_ranks(local_ms, dist, torch.device("cpu"))
    value = bench.aggregate_rate(200, w, ms)     # 100 steps x 2 solves per rank
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_aggregate():
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1]
    ms, value = out[0]
    assert ms == 20.0
    assert value == pytest.approx(200 * world / 0.020)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import bench

    class Args:
        gpus, steps, warmup = 2, 1, 3
    assert bench.run_reference(Args, world=2, rank=1) is None
    assert capsys.readouterr().out == ""
