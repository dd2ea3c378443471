"""GPU optimisation loop (qmc_optimize, App. B) and batched symmetrised
forces (qmc_force_batches, Sec. 3.3) against the oracle of the same loop."""
import numpy as np
import pytest
import torch

import qmc_inputs as qi
from oracle import optim as OP
from oracle import qmc_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2506_09743_gb300 as p

    return p


def _mask(mol, frozen=("det_weight", "backflow_w")):
    wf = O.Wavefunction(mol)
    return np.concatenate([np.full(p.numel(), 0 if k in frozen else 1, dtype=np.uint8)
                           for k, p in wf.params().items()])


@pytest.mark.parametrize("name", ["h2", "lih"])
def test_optimize_matches_the_oracle_loop(pkg, name):
    mol = qi.make_molecule(name)
    W = 96
    r0 = qi.walkers(mol, W, seed=31)
    mask = _mask(mol)
    kw = dict(n_iter=3, n_equil=20, n_resample=10, step=0.2, seed=77, lr=1e-2)
    h_ref, th_ref, r_ref = OP.optimize(mol, r0, mask=mask, **kw)
    wf = pkg.Wavefunction(mol, precision="fp64")
    x = torch.tensor(qi.to_soa(r0), device="cuda")
    hist = wf.optimize(x, mask=mask, **kw)
    n, _ = wf.param_layout()
    assert hist.shape == (3, 3)
    assert np.allclose(hist[:, 0], h_ref[:, 0], rtol=1e-10, atol=0)
    assert np.allclose(hist[:, 1], h_ref[:, 1], rtol=1e-8, atol=0)
    assert np.array_equal(hist[:, 2], h_ref[:, 2])
    r = qi.from_soa(x.cpu().numpy(), W, mol.n_elec)
    assert np.allclose(r, r_ref.numpy(), rtol=0, atol=1e-12)
    # the wavefunction keeps the final parameters: same energies as a fresh one built from them
    fresh = pkg.Wavefunction(OP.molecule_with_params(mol, th_ref), precision="fp64")
    e1, _ = wf.local_energy(x)
    e2, _ = fresh.local_energy(x)
    assert torch.allclose(e1, e2, rtol=1e-9, atol=1e-9)
    wf.close()
    fresh.close()


def test_optimize_lowers_the_h2_energy(pkg):
    mol = qi.make_h2()
    th = OP.params_vector(O.Wavefunction(mol))
    th[:2] = 0.7
    mol = OP.molecule_with_params(mol, th)
    wf = pkg.Wavefunction(mol, precision="fp64")
    x = torch.tensor(qi.to_soa(qi.walkers(mol, 8192, seed=32)), device="cuda")
    hist = wf.optimize(x, n_iter=40, n_equil=200, n_resample=20, step=0.3, seed=5, lr=0.05, mask=_mask(mol))
    sig = np.sqrt(hist[:, 1] / 8192)
    assert hist[-5:, 0].mean() < hist[:3, 0].mean() - 10 * sig.max()
    wf.close()


@pytest.mark.parametrize("symmetrize", [False, True])
def test_force_batches_match_the_oracle(pkg, symmetrize):
    mol = qi.make_h2()
    r = qi.walkers(mol, 200, seed=33)
    e_ref, f_ref = OP.force_batches(mol, r, 4, symmetrize)
    wf = pkg.Wavefunction(mol, precision="fp64")
    x = torch.tensor(qi.to_soa(r), device="cuda")
    e, f = wf.force_batches(x, 4, symmetrize=symmetrize)
    assert np.allclose(e, e_ref, rtol=1e-11, atol=0)
    assert np.allclose(f, f_ref, rtol=1e-9, atol=1e-11)
    if symmetrize:
        assert np.abs(f[:, :, :2]).max() < 1e-11
    wf.close()


def test_optimize_rejects_bad_configuration(pkg):
    from paper_2506_09743_gb300 import QmcError

    mol = qi.make_h2()
    wf = pkg.Wavefunction(mol, precision="fp64")
    x = torch.tensor(qi.to_soa(qi.walkers(mol, 8, seed=1)), device="cuda")
    with pytest.raises(QmcError):
        wf.optimize(x, n_iter=1, n_equil=0, n_resample=1, step=0.1, seed=1, beta1=1.0)
    with pytest.raises(QmcError):
        wf.optimize(x, n_iter=1, n_equil=0, n_resample=1, step=-0.1, seed=1)
    wf.close()
