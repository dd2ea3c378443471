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


def _grad_worker(rank, world, port, out):
    """One rank of a sharded sample: the oracle's per-batch sums of the
    energy-gradient estimators on this rank's walkers, one all-reduce (sum),
    then the estimator assembled by the oracle and by the C library."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import qmc_inputs as qi
    from oracle import qmc_oracle as O

    mol = qi.make_lih()
    r = qi.walkers(mol, 40, seed=51)
    lo, hi = (0, 17) if rank == 0 else (17, 40)  # uneven shards
    wf = O.Wavefunction(mol, requires_grad=True)
    sums = O.energy_grad_sums(wf, torch.tensor(r[lo:hi]))
    dist.all_reduce(sums, op=dist.ReduceOp.SUM)
    if rank == 0:
        n_param = sum(p.numel() for p in wf.params().values())
        out["sums"] = sums.numpy().copy()
        out["n_param"] = n_param
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_energy_gradient_assembles_to_the_whole_batch():
    """Eq. nabla_loss and Eq. force assembled from two ranks' sums after one
    all-reduce equal the single-rank estimator on the whole batch (1e-12),
    whether the oracle or the library's host assembly does the arithmetic."""
    import qmc_inputs as qi
    from oracle import qmc_oracle as O
    from paper_2506_09743_gb300 import _lib, build_ext

    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    mp.start_processes(_grad_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    mol = qi.make_lih()
    wf = O.Wavefunction(mol, requires_grad=True)
    Ev, var, grad, F = O.energy_grad(wf, torch.tensor(qi.walkers(mol, 40, seed=51)))
    sums, n_param = torch.tensor(out["sums"]), out["n_param"]
    build_ext.build()
    for ev2, var2, g2, f2 in (O.assemble_energy_grad(sums, n_param, mol.n_atom),
                              _lib.assemble_energy_grad(out["sums"], n_param, mol.n_atom)):
        assert abs(float(ev2) - float(Ev)) <= 1e-12 * abs(float(Ev))
        assert abs(float(var2) - float(var)) <= 1e-10 * float(var)
        g2, f2 = np.asarray(g2), np.asarray(f2)
        assert np.abs(g2 - grad.numpy()).max() <= 1e-12 * np.abs(grad.numpy()).max()
        assert np.abs(f2 - F.numpy()).max() <= 1e-12 * max(1.0, np.abs(F.numpy()).max())
