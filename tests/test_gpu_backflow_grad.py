"""GPU parity of the backflow local energy (Eq. nabla_d), the energy-gradient
estimator (Eq. nabla_loss) and the force estimator (Eq. force) against the
oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import qmc_inputs as qi
from oracle import qmc_oracle as O

from gpu_common import fp64_check, gated_check, oracle_reference

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2506_09743_gb300 as p

    return p


def _x(r):
    return torch.tensor(qi.to_soa(r), device="cuda")


def test_li2_backflow_local_energy_parity(pkg):
    mol = qi.make_li2()
    r = qi.walkers(mol, 700, seed=41)  # several 128-walker blocks and a ragged tail
    E_ref, lp_ref, sens = oracle_reference(mol, r)
    wf = pkg.Wavefunction(mol, precision="fp64")
    e, lp = wf.local_energy(_x(r))
    torch.cuda.synchronize()
    st = fp64_check(e.cpu().numpy(), E_ref, sens)
    assert np.all(np.abs(lp.cpu().numpy() - lp_ref) <= 1e-10 * np.maximum(1.0, np.abs(lp_ref)))
    print("li2 backflow fp64", st)


@pytest.mark.parametrize("n_det,W", [(1, 700), (20, 300)])
def test_backflow_fp32x2_local_energy_parity(pkg, n_det, W):
    """Backflow in the FP32X2 form (orbitals in pairs of FP32, everything
    else FP64): |dE| <= 2e-4 Ha on every walker inside the conditioning cut,
    log|Psi| within the pairs' rounding of the FP64 value."""
    mol = qi.make_li2() if n_det == 1 else qi.make_li2(n_mo=6, n_det=n_det)
    r = qi.walkers(mol, W, seed=41 + n_det)
    E_ref, lp_ref, sens = oracle_reference(mol, r)
    wf = pkg.Wavefunction(mol, precision="fp32x2")
    e, lp = wf.local_energy(_x(r))
    torch.cuda.synchronize()
    st = gated_check(e.cpu().numpy(), E_ref, sens)
    assert np.all(np.abs(lp.cpu().numpy() - lp_ref) <= 1e-9 * np.maximum(1.0, np.abs(lp_ref)) * np.maximum(1.0, sens))
    print(f"li2 backflow {n_det} det fp32x2", st)
    wf.close()


@pytest.mark.parametrize("n_det", [5, 20, 118])
def test_multidet_backflow_local_energy_parity(pkg, n_det):
    """Several determinants with backflow: excited determinants from tables of
    the reference inverse per coordinate (Eqs. table, table_squared), against
    the oracle's explicit per-determinant Eq. nabla_d."""
    mol = qi.make_li2(n_mo=6, n_det=n_det)
    r = qi.walkers(mol, 300, seed=42)
    E_ref, lp_ref, sens = oracle_reference(mol, r)
    wf = pkg.Wavefunction(mol, precision="fp64")
    e, lp = wf.local_energy(_x(r))
    torch.cuda.synchronize()
    st = fp64_check(e.cpu().numpy(), E_ref, sens, min_within=0.98)
    scale = np.maximum(1.0, np.abs(lp_ref))
    assert np.all(np.abs(lp.cpu().numpy() - lp_ref) <= 128 * 2.0 ** -53 * sens * scale)
    print(f"li2 backflow {n_det} dets fp64", st)


def test_multidet_backflow_chain_matches_oracle(pkg):
    mol = qi.make_li2(n_mo=6, n_det=20)
    r0 = qi.walkers(mol, 64, seed=48)
    r_ref, _, acc_ref = O.metropolis(O.Wavefunction(mol), torch.tensor(r0), 10, 0.1, seed=6)
    wf = pkg.Wavefunction(mol)
    x = _x(r0)
    acc = torch.zeros(64, dtype=torch.int64, device="cuda")
    wf.sample(x, n_steps=10, step=0.1, seed=6, n_accept=acc)
    torch.cuda.synchronize()
    same = acc.cpu().numpy() == acc_ref.numpy()
    assert same.mean() >= 0.98
    r_gpu = qi.from_soa(x.cpu().numpy(), 64, mol.n_elec)
    assert np.abs(r_gpu - r_ref.numpy()).max(axis=(1, 2))[same].max() < 1e-9


def test_backflow_rejected_outside_its_scope(pkg):
    from paper_2506_09743_gb300 import QmcError

    with pytest.raises(QmcError):
        pkg.Wavefunction(qi.make_li2(), precision="mixed_tf32")
    # the FP32X2 form has backflow, but gradients stay FP64
    wf = pkg.Wavefunction(qi.make_li2(), precision="fp32x2")
    with pytest.raises(QmcError):
        wf.energy_grad(_x(qi.walkers(qi.make_li2(), 16, seed=1)))
    wf.close()
    mol = qi.make_co(n_det=3)
    mol.backflow_w = 0.1
    with pytest.raises(QmcError):
        pkg.Wavefunction(mol, precision="fp64")
    # with backflow, gradients and forces are single-determinant only
    wf = pkg.Wavefunction(qi.make_li2(n_mo=6, n_det=5), precision="fp64")
    with pytest.raises(QmcError):
        wf.energy_grad(_x(qi.walkers(qi.make_li2(), 16, seed=1)))
    wf.close()


def _oracle_energy_grad(mol, r):
    wf = O.Wavefunction(mol, requires_grad=True)
    Ev, var, grad, F = O.energy_grad(wf, torch.tensor(r))
    return Ev.item(), var.item(), grad.numpy(), F.numpy()


@pytest.mark.parametrize("name,W", [("li2", 256), ("lih", 300), ("h2", 200)])
def test_energy_gradient_and_forces_match_oracle(pkg, name, W):
    mol = qi.make_molecule(name)
    r = qi.walkers(mol, W, seed=43)
    Ev, var, g_ref, F_ref = _oracle_energy_grad(mol, r)
    wf = pkg.Wavefunction(mol, precision="fp64")
    e_mean, e_var, grad, forces = wf.energy_grad(_x(r))
    g, F = grad.cpu().numpy(), forces.cpu().numpy()
    assert abs(e_mean - Ev) <= 1e-10 * max(1.0, abs(Ev))
    assert abs(e_var - var) <= 1e-8 * max(1.0, abs(var))
    n, off = wf.param_layout()
    assert g.shape == g_ref.shape == (n,)
    scale = np.abs(g_ref).max()
    assert np.abs(g - g_ref).max() <= 1e-8 * scale, (np.abs(g - g_ref).max(), scale)
    fscale = max(1.0, np.abs(F_ref).max())
    assert np.abs(F - F_ref).max() <= 1e-8 * fscale, (F, F_ref)


def test_gradient_is_bitwise_reproducible(pkg):
    mol = qi.make_li2()
    x = _x(qi.walkers(mol, 500, seed=44))
    wf = pkg.Wavefunction(mol)
    a = wf.energy_grad(x)
    b = wf.energy_grad(x)
    assert a[0] == b[0] and torch.equal(a[2], b[2]) and torch.equal(a[3], b[3])


def test_set_params_matches_fresh_wavefunction(pkg):
    mol = qi.make_li2()
    r = qi.walkers(mol, 300, seed=45)
    wf = pkg.Wavefunction(mol)
    n, off = wf.param_layout()
    p = np.concatenate([mol.prim_exp, mol.mo_coeff.reshape(-1), mol.det_weight, [mol.jastrow_b, mol.backflow_w]])
    assert p.shape[0] == n
    p2 = p.copy()
    p2[off[0]:off[1]] *= 1.05
    p2[off[3]] = 0.8
    p2[off[4]] = 0.15
    wf.set_params(p2)
    e1, _ = wf.local_energy(_x(r))
    mol2 = qi.make_li2(backflow_w=0.15)
    mol2.prim_exp = p2[off[0]:off[1]].copy()
    mol2.jastrow_b = 0.8
    e2, _ = pkg.Wavefunction(mol2).local_energy(_x(r))
    torch.cuda.synchronize()
    assert torch.equal(e1, e2)


def test_variational_energy_autograd_function(pkg):
    from paper_2506_09743_gb300 import variational_energy

    mol = qi.make_lih()
    x = _x(qi.walkers(mol, 256, seed=46))
    wf = pkg.Wavefunction(mol)
    p = torch.tensor(np.concatenate([mol.prim_exp, mol.mo_coeff.reshape(-1), mol.det_weight,
                                     [mol.jastrow_b, mol.backflow_w]]), requires_grad=True)
    R = torch.tensor(mol.atom_xyz, requires_grad=True)
    E = variational_energy(p, R, wf, x)
    E.backward()
    e_mean, _, grad, forces = wf.energy_grad(x)
    assert abs(E.item() - e_mean) == 0.0
    assert torch.equal(p.grad, grad.cpu()) and torch.equal(R.grad, -forces.cpu())


def test_backflow_metropolis_chain_matches_oracle(pkg):
    mol = qi.make_li2()
    r0 = qi.walkers(mol, 96, seed=47)
    r_ref, lp_ref, acc_ref = O.metropolis(O.Wavefunction(mol), torch.tensor(r0), 20, 0.1, seed=5)
    wf = pkg.Wavefunction(mol)
    x = _x(r0)
    acc = torch.zeros(96, dtype=torch.int64, device="cuda")
    lp = torch.empty(96, dtype=torch.float64, device="cuda")
    wf.sample(x, n_steps=20, step=0.1, seed=5, n_accept=acc, log_psi=lp)
    torch.cuda.synchronize()
    same = acc.cpu().numpy() == acc_ref.numpy()
    assert same.mean() >= 0.98
    r_gpu = qi.from_soa(x.cpu().numpy(), 96, mol.n_elec)
    assert np.abs(r_gpu - r_ref.numpy()).max(axis=(1, 2))[same].max() < 1e-9


def test_full_size_li2_energy_gradient_runs(pkg):
    mol = qi.make_li2()
    W = qi.WORKLOAD_WALKERS["li2"]
    r = qi.walkers(mol, W, seed=qi.SEED_WALKERS)
    wf = pkg.Wavefunction(mol)
    e_mean, e_var, grad, forces = wf.energy_grad(_x(r))
    assert np.isfinite(e_mean) and np.isfinite(e_var)
    assert torch.isfinite(grad).all() and torch.isfinite(forces).all()
    idx = np.random.default_rng(1).choice(W, size=128, replace=False)
    E_ref, _, sens = oracle_reference(mol, r[idx])
    e, _ = wf.local_energy(_x(r))
    torch.cuda.synchronize()
    fp64_check(e.cpu().numpy()[idx], E_ref, sens)


@pytest.mark.parametrize("name", ["li2", "lih"])
def test_sharded_sums_reproduce_the_whole_batch(pkg, name):
    """Per-batch sums of two uneven halves, added (the all-reduce of a
    sharded sample) and assembled, give qmc_energy_grad on the whole batch
    (Eq. nabla_loss, Eq. force) to 1e-10."""
    from paper_2506_09743_gb300 import _lib

    mol = qi.make_molecule(name)
    W, cut = 1000, 417
    r = qi.walkers(mol, W, seed=53)
    wf = pkg.Wavefunction(mol, precision="fp64")
    e_mean, e_var, grad, forces = wf.energy_grad(_x(r))
    s = wf.energy_grad_sums(_x(r[:cut])) + wf.energy_grad_sums(_x(r[cut:]))
    n, _ = wf.param_layout()
    ev, var, g, f = _lib.assemble_energy_grad(s.cpu().numpy(), n, mol.n_atom)
    g_ref, f_ref = grad.cpu().numpy(), forces.cpu().numpy()
    assert abs(ev - e_mean) <= 1e-10 * abs(e_mean)
    assert abs(var - e_var) <= 1e-8 * e_var
    assert np.abs(g - g_ref).max() <= 1e-10 * np.abs(g_ref).max()
    assert np.abs(f - f_ref).max() <= 1e-10 * max(1.0, np.abs(f_ref).max())
    s1 = wf.energy_grad_sums(_x(r))
    s2 = wf.energy_grad_sums(_x(r))
    assert torch.equal(s1, s2)  # fixed summation order
    wf.close()
