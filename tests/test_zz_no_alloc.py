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


@pytest.mark.parametrize("precision,rel,abs_tol", [("fp64", 1e-10, 0.0), ("mixed_tf32", 0.0, 2e-4)])
def test_noalloc_matches_workspace_entry_point_on_two_calls(pkg, precision, rel, abs_tol):
    mol = qi.make_co()
    wf = pkg.Wavefunction(mol, precision=precision)
    # two different batches in a row: the second call sees the first call's
    # leftovers in the shared static scratch
    for seed, W in ((31, 5000), (32, 3001)):
        x = torch.tensor(qi.to_soa(qi.walkers(mol, W, seed=seed)), device="cuda")
        e_ref, lp_ref = wf.local_energy(x)
        e_na, lp_na = wf.local_energy_noalloc(x)
        torch.cuda.synchronize()
        e_ref, e_na = e_ref.cpu().numpy(), e_na.cpu().numpy()
        lp_ref, lp_na = lp_ref.cpu().numpy(), lp_na.cpu().numpy()
        tol = rel * np.maximum(1.0, np.abs(e_ref)) + abs_tol
        assert np.all(np.abs(e_na - e_ref) <= tol)
        assert np.all(np.abs(lp_na - lp_ref) <= rel * np.maximum(1.0, np.abs(lp_ref)) + abs_tol)
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
