"""Pins of the optimisation-loop oracle (oracle/optim.py) against what the
ADAM definition (Kingma and Ba 2015, Algorithm 1), the sampler's counter
design and the molecule's symmetry fix, with no GPU."""
import numpy as np
import torch

import qmc_inputs as qi
from oracle import optim as OP
from oracle import qmc_oracle as O

LR, B1, B2, EPS = 1e-2, 0.9, 0.999, 1e-8


def _first_step_ok(adam):
    """First ADAM step: mhat = g and vhat = g^2 exactly in exact arithmetic,
    so every coordinate moves by lr g / (|g| + eps)."""
    rng = np.random.default_rng(0)
    th = rng.standard_normal(50)
    g = rng.standard_normal(50) * np.exp(rng.uniform(-5, 5, 50))
    new, _, _ = adam(th, np.zeros(50), np.zeros(50), g, 1, LR, B1, B2, EPS)
    want = th - LR * g / (np.abs(g) + EPS)
    return np.allclose(new, want, rtol=0, atol=1e-14)


def test_adam_first_step_closed_form():
    assert _first_step_ok(OP.adam_step)


def test_adam_constant_gradient_moves_linearly():
    """With a constant gradient mhat = g and vhat = g^2 at every step, so T
    steps move each coordinate by T lr g / (|g| + eps)."""
    th0 = np.array([0.3, -1.0, 2.0])
    g = np.array([4.0, -0.5, 1e-3])
    th, m, v = th0.copy(), np.zeros(3), np.zeros(3)
    for t in range(1, 201):
        th, m, v = OP.adam_step(th, m, v, g, t, LR, B1, B2, EPS)
    assert np.allclose(th, th0 - 200 * LR * g / (np.abs(g) + EPS), rtol=0, atol=1e-12)


def test_adam_gradient_scale_invariance():
    rng = np.random.default_rng(1)
    th = rng.standard_normal(8)
    a, b = (th.copy(), np.zeros(8), np.zeros(8)), (th.copy(), np.zeros(8), np.zeros(8))
    for t in range(1, 30):
        g = rng.standard_normal(8)
        a = OP.adam_step(*a, g, t, LR, B1, B2, EPS)
        b = OP.adam_step(*b, 1000.0 * g, t, LR, B1, B2, EPS)
    assert np.allclose(a[0], b[0], rtol=0, atol=1e-7)


def test_adam_minimises_a_quadratic():
    a = np.array([1.0, 10.0, 0.1])
    th, m, v = np.array([1.0, -1.0, 0.5]), np.zeros(3), np.zeros(3)
    for t in range(1, 3001):
        th, m, v = OP.adam_step(th, m, v, a * th, t, LR, B1, B2, EPS)
    assert np.abs(th).max() < 0.05


def test_planted_mistake_missing_bias_correction_is_caught():
    def broken(th, m, v, g, t, lr, b1, b2, eps):
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        return th - lr * m / (np.sqrt(v) + eps), m, v

    assert not _first_step_ok(broken)


def test_planted_mistake_swapped_betas_is_caught():
    def broken(th, m, v, g, t, lr, b1, b2, eps):
        return OP.adam_step(th, m, v, g, t, lr, b2, b1, eps)

    th0 = np.array([0.5, -0.25])
    g = np.array([1.0, -2.0])
    ok = []
    for fn in (OP.adam_step, broken):
        th, m, v = th0.copy(), np.zeros(2), np.zeros(2)
        for t, sgn in zip(range(1, 4), (1.0, -1.0, 1.0)):
            th, m, v = fn(th, m, v, sgn * g, t, LR, B1, B2, EPS)
        # first moment after gradients g, -g, g: the beta1 = 0.9 recursion written out
        m1 = 0.1 * g
        m2 = 0.9 * m1 - 0.1 * g
        m3 = 0.9 * m2 + 0.1 * g
        ok.append(np.allclose(m, m3, rtol=1e-15, atol=0))
    assert ok == [True, False]


def test_loop_with_everything_frozen_is_one_metropolis_chain():
    """With every parameter frozen the parameters never change and the
    walkers follow one Metropolis chain of n_equil + n_iter n_resample steps
    (the global step numbering of the sampler)."""
    mol = qi.make_h2()
    r0 = qi.walkers(mol, 16, seed=3)
    n_param = O.Wavefunction(mol).params()
    n = sum(int(p.numel()) for p in n_param.values())
    hist, theta, r = OP.optimize(mol, r0, n_iter=3, n_equil=5, n_resample=4, step=0.2, seed=11,
                                 mask=np.zeros(n))
    assert np.array_equal(theta, OP.params_vector(O.Wavefunction(mol)))
    r_chain, _, _ = O.metropolis(O.Wavefunction(mol), torch.tensor(r0), 17, 0.2, 11)
    assert torch.equal(r, r_chain)
    assert hist.shape == (3, 3) and np.all(hist[:, 2] > 0)


def test_loop_lowers_the_h2_energy():
    """A poor starting exponent (zeta = 0.7 instead of 1.24) is improved: the
    energy after a few ADAM steps is lower than at the start."""
    mol = qi.make_h2()
    mol = OP.molecule_with_params(mol, np.concatenate([[0.7, 0.7], OP.params_vector(O.Wavefunction(mol))[2:]]))
    r0 = qi.walkers(mol, 400, seed=4)
    n = OP.params_vector(O.Wavefunction(mol)).shape[0]
    mask = np.zeros(n)
    mask[:2] = 1  # exponents only
    hist, theta, _ = OP.optimize(mol, r0, n_iter=25, n_equil=60, n_resample=5, step=0.3, seed=5, lr=0.05,
                                 mask=mask)
    assert theta[0] > 0.75 and theta[1] > 0.75
    assert hist[-5:, 0].mean() < hist[:3, 0].mean() - 0.05


def test_axis_images_preserve_a_symmetric_wavefunction():
    """H2 on the z axis with 1s orbitals is symmetric under x -> -x and
    y -> -y: the images have the same local energy, and the symmetrised
    force has no x or y component."""
    mol = qi.make_h2()
    r = qi.walkers(mol, 32, seed=6)
    img = OP.axis_images(r)
    wf = O.Wavefunction(mol)
    E = O.local_energy(wf, img).reshape(4, 32)
    assert torch.allclose(E, E[0:1].expand(4, 32), rtol=1e-12, atol=1e-12)
    _, F = OP.force_batches(mol, r, 2, symmetrize=True)
    assert np.abs(F[:, :, :2]).max() < 1e-12
    assert np.abs(F[:, :, 2]).max() > 1e-6


def test_force_batches_single_batch_equals_the_estimator():
    mol = qi.make_h2()
    r = qi.walkers(mol, 24, seed=7)
    e, F = OP.force_batches(mol, r, 1, symmetrize=False)
    Ev, _, _, F0 = O.energy_grad(O.Wavefunction(mol, requires_grad=True), torch.tensor(r))
    assert e[0] == float(Ev) and np.array_equal(F[0], F0.numpy())
