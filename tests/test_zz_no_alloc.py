"""The allocation-free local-energy entry point (qmc_local_energy_noalloc).

It exists for callers that must not allocate device memory inside a call (a
serving loop running concurrent requests under a fixed memory budget, a
process whose device memory belongs to another allocator, latency-bound
callers).  It uses the library's static device scratch array instead of a
workspace, so it must return what qmc_local_energy returns, call after call,
even though the array keeps the previous call's contents.

This file is collected last on purpose, so that a run that stops at the first
failure has already run every other test; it also passes on its own in a
fresh process.
"""
import numpy as np
import pytest
import torch

import qmc_inputs as qi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2506_09743_gb300 as p

    return p


@pytest.mark.parametrize("precision", ["fp64", "mixed_tf32", "fp32x2"])
def test_noalloc_matches_workspace_entry_point_on_two_calls(pkg, precision):
    """A fresh wavefunction that has only ever used the static scratch gives,
    bit for bit, what another wavefunction gives through its own workspace
    (same kernels, same inputs), on two different batches in a row (the
    second call sees the first call's leftovers in the shared array), and
    allocates no device memory from its first call on."""
    mol = qi.make_co()
    wf_na = pkg.Wavefunction(mol, precision=precision)
    wf_ws = pkg.Wavefunction(mol, precision=precision)
    batches = []
    for seed, W in ((31, 5000), (32, 3001)):
        x = torch.tensor(qi.to_soa(qi.walkers(mol, W, seed=seed)), device="cuda")
        e = torch.empty(W, dtype=torch.float64, device="cuda")
        lp = torch.empty(W, dtype=torch.float64, device="cuda")
        batches.append((x, e, lp))
    refs = []
    for x, _, _ in batches:
        e_ref, lp_ref = wf_ws.local_energy(x)
        refs.append((e_ref.cpu().numpy(), lp_ref.cpu().numpy()))
    # first call on this device: looks the static array's address up once
    x0, e0, lp0 = batches[0]
    wf_na.local_energy_noalloc(x0, e_loc=e0, log_psi=lp0)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for (x, e, lp), (e_ref, lp_ref) in zip(batches, refs):
        wf_na.local_energy_noalloc(x, e_loc=e, log_psi=lp)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before
        assert np.array_equal(e.cpu().numpy(), e_ref)
        assert np.array_equal(lp.cpu().numpy(), lp_ref)
    wf_na.check_status()
    wf_na.close()
    wf_ws.close()


def test_noalloc_limit_is_the_one_in_the_message(pkg):
    """The largest batch the error message names is accepted; one walker more
    is refused."""
    import re

    from paper_2506_09743_gb300 import QmcError
    from paper_2506_09743_gb300 import _lib

    mol = qi.make_co()
    wf = pkg.Wavefunction(mol, precision="mixed_tf32")
    with pytest.raises(QmcError) as ei:
        wf.local_energy_noalloc(torch.zeros(3 * mol.n_elec, 100000, dtype=torch.float64, device="cuda"))
    n_max = int(re.search(r"at most (\d+) walkers", str(ei.value)).group(1))
    assert wf.workspace_size(n_max) <= _lib.NOALLOC_SCRATCH_BYTES < wf.workspace_size(n_max + 1)
    x = torch.tensor(qi.to_soa(qi.walkers(mol, n_max + 1, seed=33)), device="cuda")
    e, _ = wf.local_energy_noalloc(x, n_walkers=n_max)
    torch.cuda.synchronize()
    assert torch.isfinite(e).float().mean() > 0.99
    with pytest.raises(QmcError) as ei:
        wf.local_energy_noalloc(x, n_walkers=n_max + 1)
    assert ei.value.status == _lib.QMC_ERR_ARG
    wf.close()


def test_noalloc_rejects_batches_beyond_the_static_scratch(pkg):
    from paper_2506_09743_gb300 import QmcError
    from paper_2506_09743_gb300 import _lib

    mol = qi.make_co()
    wf = pkg.Wavefunction(mol, precision="mixed_tf32")
    W = 200000  # needs far more than the 64 MiB static scratch
    x = torch.zeros(3 * mol.n_elec, W, dtype=torch.float64, device="cuda")
    with pytest.raises(QmcError) as ei:
        wf.local_energy_noalloc(x)
    assert ei.value.status == _lib.QMC_ERR_ARG
    assert "static scratch" in str(ei.value) and "at most" in str(ei.value)
    wf.close()
