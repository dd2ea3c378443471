"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): walkers are
sharded with no data-path collective, the step time is the maximum over
ranks and the value is the whole-job rate."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import qmc_inputs as qi

    per_rank_ms = 10.0 + 5.0 * rank  # the slower rank sets the step time
    mx = bench.reduce_max(per_rank_ms, dist)
    r = qi.walkers(qi.make_h2(), 8, seed=bench.rank_walker_seed(rank))
    out[rank] = (mx, bench.whole_job_rate(world, 1000, 4, mx), float(r.sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_whole_job_rate():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    assert out[0][0] == out[1][0] == 15.0
    assert out[0][1] == pytest.approx(2 * 1000 * 4 / 0.015)
    assert out[0][2] != out[1][2]  # each rank draws its own walkers


def test_single_process_reduce_is_identity():
    import bench

    assert bench.reduce_max(3.5, None) == 3.5
    assert bench.whole_job_rate(1, 262144, 20, 1000.0) == 262144 * 20
