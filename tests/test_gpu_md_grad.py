"""GPU parity of the energy-gradient estimator (Eq. nabla_loss) for
multi-determinant expansions without backflow (Eq. psimol with the CI sum):
the parameter gradient of log|Psi| through tables of the reference inverse,
against the oracle's autograd gradient, through the C ABI."""
import numpy as np
import pytest
import torch

import qmc_inputs as qi
from oracle import qmc_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2506_09743_gb300 as p

    return p


def _x(r):
    return torch.tensor(qi.to_soa(r), device="cuda")


def _oracle(mol, r):
    wf = O.Wavefunction(mol, requires_grad=True)
    Ev, var, grad, _ = O.energy_grad(wf, torch.tensor(r))
    return Ev.item(), var.item(), grad.numpy()


@pytest.mark.parametrize("n_det,W", [(20, 96), (100, 70), (1, 45), (5, 37)])
def test_multidet_energy_gradient_matches_oracle(pkg, n_det, W):
    """CO (14 electrons, 58 GTOs, 14 MOs): CI weights, MO coefficients,
    exponents, Jastrow b and the backflow weight at w = 0, at 1e-8 of the
    largest component; W spans several warps with ragged tails."""
    mol = qi.make_co(n_det=n_det)
    r = qi.walkers(mol, W, seed=61 + n_det)
    Ev, var, g_ref = _oracle(mol, r)
    wf = pkg.Wavefunction(mol, precision="fp64")
    e_mean, e_var, grad, forces = wf.energy_grad(_x(r), want_forces=False)
    assert forces is None
    g = grad.cpu().numpy()
    assert abs(e_mean - Ev) <= 1e-10 * max(1.0, abs(Ev))
    assert abs(e_var - var) <= 1e-8 * max(1.0, abs(var))
    n, off = wf.param_layout()
    assert g.shape == g_ref.shape == (n,)
    scale = np.abs(g_ref).max()
    err = np.abs(g - g_ref)
    assert err.max() <= 1e-8 * scale, (err.max(), scale, int(err.argmax()))
    # every block on its own scale too (the CI weights' gradient is far smaller
    # than the exponents'); a block that vanishes in exact arithmetic (one
    # determinant: the CI weight's gradient is 2 sum (E_L - E_v) / (M d_0) = 0)
    # is rounding noise on both sides and is held to the overall scale
    for k in range(5):
        lo, hi = off[k], off[k + 1]
        if hi > lo:
            s = max(np.abs(g_ref[lo:hi]).max(), 1e-6 * scale)
            assert err[lo:hi].max() <= 1e-7 * s, (k, err[lo:hi].max(), s)
    wf.close()


def test_multidet_gradient_is_bitwise_reproducible(pkg):
    mol = qi.make_co(n_det=20)
    x = _x(qi.walkers(mol, 300, seed=66))
    wf = pkg.Wavefunction(mol)
    a = wf.energy_grad(x, want_forces=False)
    b = wf.energy_grad(x, want_forces=False)
    assert a[0] == b[0] and torch.equal(a[2], b[2])
    wf.close()


def test_multidet_forces_refused(pkg):
    from paper_2506_09743_gb300 import QmcError

    mol = qi.make_co(n_det=20)
    wf = pkg.Wavefunction(mol)
    x = _x(qi.walkers(mol, 16, seed=67))
    with pytest.raises(QmcError):
        wf.energy_grad(x, want_forces=True)
    wf.close()


def test_full_size_co_multidet_gradient_runs(pkg):
    """131,072 CO walkers, 100 determinants: the gradient is finite and its
    CI-weight block sums to 2 (E[E_L R/S] - E_v E[R/S]) computed from the
    same walkers' energies (a property that holds at any size)."""
    mol = qi.make_co()
    W = 131072
    x = _x(qi.walkers(mol, W, seed=68))
    wf = pkg.Wavefunction(mol)
    e_mean, e_var, grad, _ = wf.energy_grad(x, want_forces=False)
    g = grad.cpu().numpy()
    assert np.isfinite(e_mean) and np.isfinite(g).all()
    n, off = wf.param_layout()
    # sum_n d_n dlogPsi/dd_n = 1 for every walker, so sum_n d_n grad_n = 2 (E_v - E_v) = 0
    d = np.asarray(mol.det_weight)
    ci = g[off[2]:off[3]]
    assert abs(float(np.dot(d, ci))) <= 1e-9 * max(1.0, float(np.abs(d * ci).sum())), float(np.dot(d, ci))
    wf.close()


@pytest.mark.parametrize("name,n_det,W", [("co", 20, 40), ("lih", 1, 100)])
def test_manybody_jastrow_gradient_matches_oracle(pkg, name, n_det, W):
    """The many-body Jastrow's parameters (App. D: K_en and five K_een terms)
    join the gradient after the backflow weight; the whole gradient matches
    the oracle's autograd gradient at 1e-8 of its largest component, the
    many-body block at 1e-7 of its own."""
    base = qi.make_co(n_det=n_det) if name == "co" else qi.make_lih()
    mol = qi.with_manybody_jastrow(base)
    r = qi.walkers(mol, W, seed=69)
    Ev, var, g_ref = _oracle(mol, r)
    wf = pkg.Wavefunction(mol, precision="fp64")
    n, off = wf.param_layout()
    assert n == off[4] + 1 + 3 + 7 * 5 == g_ref.shape[0]
    e_mean, _, grad, _ = wf.energy_grad(_x(r), want_forces=False)
    g = grad.cpu().numpy()
    assert abs(e_mean - Ev) <= 1e-10 * max(1.0, abs(Ev))
    err = np.abs(g - g_ref)
    assert err.max() <= 1e-8 * np.abs(g_ref).max(), (err.max(), int(err.argmax()))
    mb = slice(off[4] + 1, n)
    assert err[mb].max() <= 1e-7 * np.abs(g_ref[mb]).max(), (err[mb], g_ref[mb])
    with pytest.raises(Exception):
        wf.energy_grad(_x(r), want_forces=True)
    wf.close()


def test_set_params_covers_the_manybody_jastrow(pkg):
    """qmc_set_params with changed many-body parameters gives the energies of
    a wavefunction built with them (bitwise)."""
    mol = qi.with_manybody_jastrow(qi.make_co(n_det=20))
    r = qi.walkers(mol, 256, seed=70)
    wf = pkg.Wavefunction(mol, precision="fp64")
    n, off = wf.param_layout()
    en, een = np.asarray(mol.jastrow_en), np.asarray(mol.jastrow_een)
    p = np.concatenate([mol.prim_exp, mol.mo_coeff.reshape(-1), mol.det_weight, [mol.jastrow_b, mol.backflow_w],
                        en, een.reshape(-1)])
    assert p.shape[0] == n
    en2, een2 = en * 1.1, een.copy()
    een2[:, 0] *= -0.7
    p[off[4] + 1:] = np.concatenate([en2, een2.reshape(-1)])
    wf.set_params(p)
    e1, _ = wf.local_energy(_x(r))
    mol2 = qi.with_manybody_jastrow(qi.make_co(n_det=20))
    mol2.jastrow_en, mol2.jastrow_een = en2, een2
    e2, _ = pkg.Wavefunction(mol2, precision="fp64").local_energy(_x(r))
    torch.cuda.synchronize()
    assert torch.equal(e1, e2)
    wf.close()


def test_multidet_gradient_sums_of_halves_match_the_whole(pkg):
    """Per-batch sums (qmc_energy_grad_sums) of two halves of a CO-20 batch,
    added and assembled, reproduce qmc_energy_grad on the whole batch; the
    force blocks are NaN on this path."""
    from paper_2506_09743_gb300 import _lib

    mol = qi.make_co(n_det=20)
    W = 300
    r = qi.walkers(mol, W, seed=72)
    wf = pkg.Wavefunction(mol, precision="fp64")
    n, _ = wf.param_layout()
    e_mean, e_var, grad, _ = wf.energy_grad(_x(r), want_forces=False)
    s1 = wf.energy_grad_sums(_x(r[:131])).cpu().numpy()
    s2 = wf.energy_grad_sums(_x(r[131:])).cpu().numpy()
    assert np.isnan(s1[3 + 2 * n:]).all() and np.isnan(s2[3 + 2 * n:]).all()
    tot = s1 + s2
    tot[3 + 2 * n:] = 0.0
    ev, var, g, _ = _lib.assemble_energy_grad(tot, n, mol.n_atom)
    g_ref = grad.cpu().numpy()
    assert abs(ev - e_mean) <= 1e-12 * abs(e_mean)
    assert abs(var - e_var) <= 1e-10 * e_var
    assert np.abs(np.asarray(g) - g_ref).max() <= 1e-10 * np.abs(g_ref).max()
    wf.close()
