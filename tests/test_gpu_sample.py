"""GPU Metropolis sampler (qmc_sample) against the oracle chain and physics."""
import math

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


def test_h2_chain_matches_oracle(pkg):
    """The H2 workload: 1024 walkers, 200 steps of 0.2 bohr.  Same Philox
    counters on both sides: identical accept decisions, positions equal to
    rounding of the Box-Muller transcendental functions."""
    mol = qi.make_h2()
    r0 = qi.walkers(mol, 1024, seed=qi.SEED_WALKERS)
    r_ref, lp_ref, acc_ref = O.metropolis(O.Wavefunction(mol), torch.tensor(r0), 200, 0.2, seed=0x5EED)
    wf = pkg.Wavefunction(mol)
    x = torch.tensor(qi.to_soa(r0), device="cuda")
    lp = torch.empty(1024, dtype=torch.float64, device="cuda")
    acc = torch.zeros(1024, dtype=torch.int64, device="cuda")
    wf.sample(x, n_steps=200, step=0.2, seed=0x5EED, log_psi=lp, n_accept=acc)
    torch.cuda.synchronize()
    r_gpu = qi.from_soa(x.cpu().numpy(), 1024, 2)
    same = acc.cpu().numpy() == acc_ref.numpy()
    assert same.mean() >= 0.999, same.mean()
    d = np.abs(r_gpu - r_ref.numpy()).max(axis=(1, 2))
    assert np.all(d[same] < 1e-10), d[same].max()
    assert np.abs(lp.cpu().numpy() - lp_ref.numpy())[same].max() < 1e-10


def test_chain_resume_and_batching_on_gpu(pkg):
    mol = qi.make_lih()
    r0 = torch.tensor(qi.to_soa(qi.walkers(mol, 300, seed=3)), device="cuda")
    wf = pkg.Wavefunction(mol)
    a = r0.clone()
    wf.sample(a, n_steps=10, step=0.3, seed=42)
    b = r0.clone()
    wf.sample(b, n_steps=4, step=0.3, seed=42)
    wf.sample(b, n_steps=6, step=0.3, seed=42, step_offset=4)
    c = r0.clone()
    wf.sample(c[:, :100], n_steps=10, step=0.3, seed=42, n_walkers=100)
    tail = r0[:, 100:].contiguous()
    wf.sample(tail, n_steps=10, step=0.3, seed=42, first_walker=100)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert torch.equal(a[:, :100], c[:, :100]) and torch.equal(a[:, 100:], tail)


def test_helium_mean_energy_within_3_sigma_gpu(pkg):
    """He with the optimal 1s(27/16) product: <E> = -(27/16)^2 exactly."""
    he = qi.make_helium(1.6875)
    W = 16384
    wf = pkg.Wavefunction(he)
    x = torch.tensor(qi.to_soa(qi.walkers(he, W, seed=13)), device="cuda")
    wf.sample(x, n_steps=300, step=0.5, seed=77)
    acc = torch.zeros(W, dtype=torch.float64, device="cuda")
    n_blk = 8
    for k in range(n_blk):
        wf.sample(x, n_steps=20, step=0.5, seed=77, step_offset=300 + 20 * k)
        e, _ = wf.local_energy(x)
        acc += e
    torch.cuda.synchronize()
    per_walker = (acc / n_blk).cpu().numpy()
    mean = per_walker.mean()
    err = per_walker.std() / math.sqrt(W)
    assert abs(mean - (-2.84765625)) < 3 * err, (mean, err)


def test_mixed_precision_sampler_runs_and_accepts(pkg):
    mol = qi.make_co(n_det=100)
    W = 4096
    wf = pkg.Wavefunction(mol, precision="mixed_tf32")
    x = torch.tensor(qi.to_soa(qi.walkers(mol, W, seed=2)), device="cuda")
    acc = torch.zeros(W, dtype=torch.int64, device="cuda")
    lp = torch.empty(W, dtype=torch.float64, device="cuda")
    wf.sample(x, n_steps=20, step=0.05, seed=9, n_accept=acc, log_psi=lp)
    torch.cuda.synchronize()
    rate = acc.double().mean().item() / 20
    assert 0.3 < rate < 1.0, rate
    assert torch.isfinite(lp).float().mean().item() > 0.999


def test_backflow_chain_matches_oracle(pkg):
    """Li2 with backflow (the FP64 value-only kernel of the general path):
    256 walkers, 30 steps of 0.2 bohr against the oracle chain with the same
    Philox counters; and the sampler's final log|Psi| against the local-energy
    call's at the same positions."""
    mol = qi.make_li2()
    W = 256
    r0 = qi.walkers(mol, W, seed=21)
    r_ref, lp_ref, acc_ref = O.metropolis(O.Wavefunction(mol), torch.tensor(r0), 30, 0.2, seed=77)
    wf = pkg.Wavefunction(mol, precision="fp64")
    x = torch.tensor(qi.to_soa(r0), device="cuda")
    lp = torch.empty(W, dtype=torch.float64, device="cuda")
    acc = torch.zeros(W, dtype=torch.int64, device="cuda")
    wf.sample(x, n_steps=30, step=0.2, seed=77, log_psi=lp, n_accept=acc)
    torch.cuda.synchronize()
    r_gpu = qi.from_soa(x.cpu().numpy(), W, mol.n_elec)
    same = acc.cpu().numpy() == acc_ref.numpy()
    assert same.mean() >= 0.99, same.mean()
    d = np.abs(r_gpu - r_ref.numpy()).max(axis=(1, 2))
    assert np.all(d[same] < 1e-10), d[same].max()
    assert np.abs(lp.cpu().numpy() - lp_ref.numpy())[same].max() < 1e-10
    _, lp_e = wf.local_energy(x)
    assert torch.allclose(lp, lp_e, rtol=0, atol=1e-12)
    wf.close()


@pytest.mark.parametrize("name,precision", [("lih", "fp64"), ("co", "mixed_tf32"), ("li2", "fp64")])
def test_step_graph_replays_the_plain_loop(pkg, name, precision):
    """n_steps >= 4 run as a replayed CUDA graph of one step; one-step calls
    run the plain launch loop.  Same chain bit for bit: positions, log|Psi|
    and acceptance counts."""
    mol = qi.make_molecule(name)
    W = 777
    r0 = torch.tensor(qi.to_soa(qi.walkers(mol, W, seed=5)), device="cuda")
    wf = pkg.Wavefunction(mol, precision=precision)
    a, b = r0.clone(), r0.clone()
    lpa = torch.empty(W, dtype=torch.float64, device="cuda")
    lpb = torch.empty_like(lpa)
    acca = torch.zeros(W, dtype=torch.int64, device="cuda")
    accb = torch.zeros_like(acca)
    wf.sample(a, n_steps=12, step=0.1, seed=99, step_offset=3, log_psi=lpa, n_accept=acca)
    for t in range(12):
        wf.sample(b, n_steps=1, step=0.1, seed=99, step_offset=3 + t, log_psi=lpb, n_accept=accb)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(lpa, lpb) and torch.equal(acca, accb)
    assert 0 < int(acca.sum()) < 12 * W
    wf.close()


def test_proposal_gaussians_match_library_box_muller(pkg):
    """The proposal kernel's table-driven Box-Muller against the oracle's
    FP64 library Box-Muller on the same Philox words: one step of 1 bohr, so
    an accepted walker moves by its Gaussian vector; agreement to a few ulp
    over 40,000 walkers x 12 coordinates (the far tail included)."""
    from oracle import philox

    mol = qi.make_lih()
    W = 40000
    x0 = torch.tensor(qi.to_soa(qi.walkers(mol, W, seed=8)), device="cuda")
    x = x0.clone()
    wf = pkg.Wavefunction(mol, precision="fp64")
    acc = torch.zeros(W, dtype=torch.int64, device="cuda")
    wf.sample(x, n_steps=1, step=1.0, seed=4242, step_offset=17, n_accept=acc)
    torch.cuda.synchronize()
    z_ref, _ = philox.walker_normals_and_uniform(4242, np.arange(W), 17, 3 * mol.n_elec)
    a = acc.cpu().numpy() == 1
    assert a.sum() > 1000
    x0n, x1n = x0.cpu().numpy().T[a], x.cpu().numpy().T[a]
    z = z_ref[a]
    eps = np.finfo(np.float64).eps
    # the subtraction x1 - x0 rounds at the positions' scale; the Gaussians
    # themselves are compared at a few ulp
    tol = 2 * eps * (np.abs(x0n) + np.abs(x1n)) + 8 * eps * np.maximum(1.0, np.abs(z))
    assert np.all(np.abs((x1n - x0n) - z) <= tol), float((np.abs((x1n - x0n) - z) / tol).max())
    wf.close()


@pytest.mark.parametrize("name,precision", [("lih", "fp32x2"), ("lih", "mixed_tf32"), ("co", "fp32x2"),
                                            ("co", "mixed_tf32"), ("li2", "fp32x2")])
def test_reduced_precision_chain_mean_matches_fp64_chain(pkg, name, precision):
    """The Metropolis chain of a reduced-precision form samples the same
    |Psi|^2 as the FP64 form: from the same walkers and Philox key, its mean
    local energy (10 blocks of 10 steps after 100 steps of equilibration,
    4,096 walkers, per-walker block means) agrees with the FP64 chain's
    within 3 sigma of the two estimates combined."""
    mol = qi.make_molecule(name)
    W = 4096
    r0 = qi.walkers(mol, W, seed=71)
    means = {}
    for prec in ("fp64", precision):
        wf = pkg.Wavefunction(mol, precision=prec)
        x = torch.tensor(qi.to_soa(r0), device="cuda")
        wf.sample(x, n_steps=100, step=0.05, seed=123)
        acc = torch.zeros(W, dtype=torch.float64, device="cuda")
        for blk in range(10):
            wf.sample(x, n_steps=10, step=0.05, seed=123, step_offset=100 + 10 * blk)
            e, _ = wf.local_energy(x)
            acc += e
        torch.cuda.synchronize()
        per_walker = (acc / 10).cpu().numpy()
        assert np.isfinite(per_walker).all()
        means[prec] = (per_walker.mean(), per_walker.std() / math.sqrt(W))
        wf.close()
    (m64, s64), (m, s) = means["fp64"], means[precision]
    assert abs(m - m64) < 3 * math.sqrt(s64 ** 2 + s ** 2), (means, name, precision)
