"""Pins of the CPU oracle against what the paper and mathematics fix.

Every check here is independent of the oracle's own formulas: closed forms,
finite differences, brute-force (autograd) differentiation, explicit
inversion of every excited matrix, numerical quadrature, printed
determinant counts and published generator test vectors.
"""
import math
import os

import numpy as np
import pytest
import torch

import qmc_inputs as qi
from oracle import philox
from oracle import qmc_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b):
    return ((a - b).abs() / b.abs().clamp(min=1.0)).max().item()


def _walkers(mol, n, seed=1):
    return torch.tensor(qi.walkers(mol, n, seed=seed))


# --------------------------------------------------------------------------
# printed values


def test_sd_counts_match_paper():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "sd_counts.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 5
    for ne, no, cnt in rows:
        assert qi.sd_count(int(ne), int(no)) == int(cnt)


def test_co_active_space_candidates():
    # (10e, 12o) above 2 frozen core orbitals per spin: 1 + 70 + 420 + 1225
    assert len(qi.sd_expansion(7, 7, 14, 2)) == 1716
    mol = qi.make_co()
    assert mol.n_det == 100 and mol.det_weight[0] == 0.95
    assert abs(np.sum(mol.det_weight[1:] ** 2) - (1 - 0.95 ** 2)) < 1e-14


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        v = [int(x, 16) for x in row]
        out = philox.philox4x32_10(*v[:6])
        assert [int(o) for o in out] == v[6:]


def test_box_muller_moments():
    z, u = philox.walker_normals_and_uniform(1234, np.arange(20000), 7, 6)
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1.0) < 0.02
    assert 0.0 < u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01


# --------------------------------------------------------------------------
# atomic orbitals


def _ao_test_molecule():
    bb = qi._BasisBuilder()
    specs = [
        (qi.STO, (0, 0, 0, 0), [1.7], [1.0]),
        (qi.STO, (0, 0, 0, 1), [0.9], [1.0]),
        (qi.STO, (1, 0, 0, 0), [1.1], [1.0]),
        (qi.STO, (0, 1, 1, 1), [1.3], [1.0]),
        (qi.GTO, (0, 0, 0, 0), [3.0, 0.7, 0.2], [0.3, 0.5, 0.6]),
        (qi.GTO, (0, 0, 1, 0), [2.0, 0.4, 0.15], [0.4, 0.8, 0.3]),
        (qi.GTO, (2, 0, 0, 0), [1.5, 0.5], [0.7, 0.6]),
        (qi.GTO, (1, 1, 0, 0), [1.2], [1.0]),
    ]
    for kind, pw, e, c in specs:
        bb.add(0, kind, *pw, e, c)
    return qi.Molecule(name="ao", atom_xyz=np.array([[0.1, -0.2, 0.3]]), atom_z=np.array([1.0]), n_up=1, n_down=0,
                       **bb.arrays(), mo_coeff=np.ones((len(specs), 1)), det_weight=np.ones(1),
                       det_exc=np.zeros((1, 2, 5), dtype=np.int32))


def test_ao_normalisation_by_quadrature():
    """Primitive AOs integrate to one: radial quadrature times a product
    Gauss-Legendre x trapezoid rule on the sphere, on the oracle's values."""
    from scipy import integrate

    bb = qi._BasisBuilder()
    cases = [(qi.STO, (0, 0, 0, 0), 1.4), (qi.STO, (0, 0, 0, 1), 0.8), (qi.STO, (0, 0, 1, 0), 1.2),
             (qi.STO, (1, 1, 0, 0), 1.0), (qi.GTO, (0, 0, 0, 0), 0.9), (qi.GTO, (1, 0, 0, 0), 1.3),
             (qi.GTO, (0, 0, 2, 0), 0.6), (qi.GTO, (0, 1, 1, 0), 2.1)]
    for kind, pw, e in cases:
        bb.add(0, kind, *pw, [e], [1.0])
    mol = qi.Molecule(name="n", atom_xyz=np.zeros((1, 3)), atom_z=np.ones(1), n_up=1, n_down=0, **bb.arrays(),
                      mo_coeff=np.ones((len(cases), 1)), det_weight=np.ones(1),
                      det_exc=np.zeros((1, 2, 5), dtype=np.int32))
    wf = O.Wavefunction(mol)
    ct, wt = np.polynomial.legendre.leggauss(24)
    ph = np.arange(48) * 2 * np.pi / 48
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([np.outer(st, np.cos(ph)), np.outer(st, np.sin(ph)), np.outer(ct, np.ones_like(ph))], -1).reshape(-1, 3)
    wang = np.outer(wt, np.full(48, 2 * np.pi / 48)).reshape(-1)

    def shell(rho):
        pts = torch.tensor(rho * dirs)[:, None, :]
        v = O.ao_eval(wf, pts)[:, 0, :].numpy()
        return (wang[:, None] * v * v).sum(0) * rho * rho

    for k in range(len(cases)):
        val = integrate.quad(lambda x: shell(x)[k], 0, 60, limit=200, epsabs=1e-12)[0]
        assert abs(val - 1.0) < 1e-8, (cases[k], val)


def test_ao_derivatives_finite_difference():
    wf = O.Wavefunction(_ao_test_molecule())
    r = torch.tensor(np.random.default_rng(3).normal(size=(16, 1, 3)))
    v, g, lp, H = O.ao_eval(wf, r, order=2)
    h = 1e-5
    for d in range(3):
        e = torch.zeros(3, dtype=torch.float64)
        e[d] = h
        fd = (O.ao_eval(wf, r + e) - O.ao_eval(wf, r - e)) / (2 * h)
        assert _rel(g[..., d], fd) < 1e-7
        gp = O.ao_eval(wf, r + e, order=1)[1]
        gm = O.ao_eval(wf, r - e, order=1)[1]
        assert _rel(H[..., d, :], (gp - gm) / (2 * h)) < 1e-6
    assert _rel(lp, H.diagonal(dim1=-2, dim2=-1).sum(-1)) < 1e-12


def test_hydrogen_atom_exact_1s():
    mol = qi.make_hydrogenic(1.0, 1.0)
    wf = O.Wavefunction(mol)
    r = _walkers(mol, 64)
    E = O.local_energy(wf, r)
    assert torch.allclose(E, torch.full_like(E, -0.5), atol=1e-13, rtol=0)
    assert E.var().item() < 1e-26


def test_hydrogen_with_electron_nucleus_kernel_closed_form():
    """One electron in the exact 1s orbital times exp(K_en(r)): with
    Psi = exp(K(r) - r), lap Psi / Psi = (K' - 1)^2 + K'' + 2 (K' - 1) / r, so
    E_L = -1/2 [(K' - 1)^2 + K'' + 2 (K' - 1)/r] - 1/r, with K' and K'' of
    K(r) = (w0 r + w1 r^2)/(1 + w2 r) differentiated by hand."""
    import dataclasses

    w0, w1, w2 = -0.2, 0.03, 0.8
    mol = dataclasses.replace(qi.make_hydrogenic(1.0, 1.0), jastrow_en=np.array([w0, w1, w2]))
    wf = O.Wavefunction(mol)
    r = _walkers(mol, 64)
    x = torch.sqrt((r[:, 0] ** 2).sum(-1))
    d = 1 + w2 * x
    K1 = (w0 + w1 * x * (2 + w2 * x)) / d ** 2
    K2 = 2 * (w1 - w0 * w2) / d ** 3
    ref = -0.5 * ((K1 - 1) ** 2 + K2 + 2 * (K1 - 1) / x) - 1 / x
    assert _rel(O.local_energy(wf, r), ref) < 1e-12


def test_electron_electron_nucleus_kernel_is_exchange_symmetric():
    """The many-body terms are spin independent and symmetric under the
    exchange of any two electrons (the kernel is summed over ordered pairs),
    although each of its terms is not."""
    mol = qi.with_manybody_jastrow(qi.make_lih(), en=False)
    wf = O.Wavefunction(mol)
    r = _walkers(mol, 8)
    J0 = O.jastrow_manybody(wf, r)[0]
    for i, j in ((0, 1), (0, 2), (1, 3)):
        rs = r.clone()
        rs[:, [i, j]] = r[:, [j, i]]
        assert torch.allclose(O.jastrow_manybody(wf, rs)[0], J0, atol=1e-13, rtol=0)


@pytest.mark.parametrize("zeta,Z", [(1.3, 1.0), (0.7, 2.0), (2.5, 3.0)])
def test_hydrogenic_closed_form(zeta, Z):
    mol = qi.make_hydrogenic(zeta, Z)
    wf = O.Wavefunction(mol)
    r = _walkers(mol, 64)
    rr = r[:, 0].norm(dim=-1)
    assert _rel(O.local_energy(wf, r), -zeta ** 2 / 2 + (zeta - Z) / rr) < 1e-13


def test_helium_product_closed_form():
    mol = qi.make_helium(1.6875)
    wf = O.Wavefunction(mol)
    r = _walkers(mol, 64)
    z = 1.6875
    r1, r2 = r[:, 0].norm(dim=-1), r[:, 1].norm(dim=-1)
    r12 = (r[:, 0] - r[:, 1]).norm(dim=-1)
    assert _rel(O.local_energy(wf, r), -z * z + (z - 2) * (1 / r1 + 1 / r2) + 1 / r12) < 1e-13


def test_nuclear_repulsion_closed_form():
    for name in ("h2", "lih", "li2", "co"):
        mol = qi.make_molecule(name)
        wf = O.Wavefunction(mol)
        R = np.linalg.norm(mol.atom_xyz[0] - mol.atom_xyz[1])
        assert abs(O.nuclear_repulsion(wf).item() - mol.atom_z[0] * mol.atom_z[1] / R) < 1e-13


# --------------------------------------------------------------------------
# kinetic energy: trace formulas against brute-force differentiation


@pytest.mark.parametrize("name", ["h2", "lih", "co_small", "li2", "li2_multidet", "li2_sd20", "lih_mbj", "li2_mbj"])
def test_local_energy_matches_autograd_laplacian(name):
    if name == "co_small":
        mol = qi.make_co(n_det=8)
    elif name == "lih_mbj":
        mol = qi.with_manybody_jastrow(qi.make_lih())
    elif name == "li2_mbj":
        mol = qi.with_manybody_jastrow(qi.make_li2(backflow_w=0.0))
    elif name == "li2_multidet":
        mol = _li2_multidet()
    elif name == "li2_sd20":
        mol = qi.make_li2(n_mo=6, n_det=20)
    else:
        mol = qi.make_molecule(name)
    wf = O.Wavefunction(mol)
    r = _walkers(mol, 6)
    assert _rel(O.local_energy(wf, r), O.local_energy_ad(wf, r)) < 1e-11


def _li2_multidet():
    """Li2 with backflow and a small multi-determinant expansion (the
    multi-det + backflow path of eq. delta_sigma with its cross term)."""
    mol = qi.make_li2(n_mo=6)
    dets = [(qi.ground_exc(), qi.ground_exc()), ((1, 2, -1, 3, -1), qi.ground_exc()),
            (qi.ground_exc(), (1, 1, -1, 4, -1)), ((1, 2, -1, 5, -1), (1, 2, -1, 3, -1)),
            ((2, 1, 2, 3, 5), qi.ground_exc())]
    mol.det_exc = qi._dets_array(dets)
    mol.det_weight = np.array([0.9, 0.3, -0.2, 0.25, 0.1])
    return mol


def test_backflow_formula_reduces_without_backflow():
    mol = qi.make_lih()
    wf = O.Wavefunction(mol)
    r = _walkers(mol, 8)
    S1, gS, lS = O.slater_derivs_explicit(wf, r)
    S2, dS, d2S = O.slater_derivs_backflow(wf, r)
    assert _rel(S1, S2) < 1e-13
    assert _rel(gS.reshape(8, -1), dS) < 1e-12
    assert _rel(lS, d2S.sum(-1)) < 1e-12


def test_backflow_jacobian_finite_difference():
    wf = O.Wavefunction(qi.make_li2())
    r = _walkers(wf.mol, 4)
    _, J1, J2 = O.backflow_derivs(wf, r)
    h = 1e-5
    N = wf.n_elec
    for k in range(N):
        for e in range(3):
            d = torch.zeros_like(r)
            d[:, k, e] = h
            fd1 = (O.backflow(wf, r + d) - O.backflow(wf, r - d)) / (2 * h)
            assert _rel(J1[:, :, :, k, e], fd1) < 1e-7
            J1p = O.backflow_derivs(wf, r + d)[1][:, :, :, k, e]
            J1m = O.backflow_derivs(wf, r - d)[1][:, :, :, k, e]
            assert _rel(J2[:, :, :, k, e], (J1p - J1m) / (2 * h)) < 1e-6


@pytest.mark.parametrize("manybody", [False, True])
def test_jastrow_derivatives_finite_difference(manybody):
    mol = qi.make_lih()
    wf = O.Wavefunction(qi.with_manybody_jastrow(mol) if manybody else mol)
    r = _walkers(wf.mol, 8)
    J, gJ, lJ = O.jastrow(wf, r)
    h = 1e-5
    for i in range(wf.n_elec):
        for d in range(3):
            e = torch.zeros_like(r)
            e[:, i, d] = h
            Jp, gp, _ = O.jastrow(wf, r + e)
            Jm, gm, _ = O.jastrow(wf, r - e)
            assert _rel(gJ[:, i, d], (Jp - Jm) / (2 * h)) < 1e-7
            if d == 0:
                lap = 0
            lap = lap + (gp[:, i, d] - gm[:, i, d]) / (2 * h)
        assert _rel(lJ[:, i], lap) < 1e-6


# --------------------------------------------------------------------------
# table method and matrix identities (App. F, G, H)


def _random_phi(W=16, n=5, n_mo=9, seed=0):
    g = torch.Generator().manual_seed(seed)
    return torch.randn(W, n, n_mo, dtype=torch.float64, generator=g), torch.randn(W, n, n_mo, dtype=torch.float64, generator=g)


EXC = [(0, -1, -1, -1, -1), (1, 1, -1, 6, -1), (1, 4, -1, 5, -1), (2, 0, 3, 5, 8), (2, 2, 4, 6, 7)]


@pytest.mark.parametrize("rec", EXC)
def test_table_trace_matches_explicit_inverse(rec):
    Phi, B = _random_phi()
    n = Phi.shape[1]
    AX = O.excited_matrix(Phi, rec, n)
    BX = O.excited_matrix(B, rec, n)
    ref_tr = torch.einsum("wab,wba->w", torch.linalg.inv(AX), BX)
    ref_ratio = torch.linalg.det(AX) / torch.linalg.det(Phi[..., :n])
    tr, ratio = O.table_trace(Phi, B, rec)
    assert _rel(tr, ref_tr) < 1e-9
    assert _rel(ratio, ref_ratio) < 1e-11


@pytest.mark.parametrize("rec", EXC)
def test_table_squared_matches_explicit_inverse(rec):
    Phi, B = _random_phi(seed=1)
    n = Phi.shape[1]
    X = torch.linalg.inv(O.excited_matrix(Phi, rec, n)) @ O.excited_matrix(B, rec, n)
    ref = torch.einsum("wab,wba->w", X, X)
    assert _rel(O.table_trace_squared(Phi, B, rec), ref) < 1e-8


@pytest.mark.parametrize("rec", EXC[1:])
def test_woodbury_inverse(rec):
    Phi, _ = _random_phi(seed=2)
    n = Phi.shape[1]
    ref = torch.linalg.inv(O.excited_matrix(Phi, rec, n))
    assert _rel(O.woodbury_inverse(Phi, rec), ref) < 1e-9


def test_single_row_trace_identity():
    """App. G: for dA with one non-zero row, Tr(A^-1 dA)^2 = Tr((A^-1 dA)^2)."""
    A, dA = _random_phi(n=6, n_mo=6, seed=4)
    dA[:, [0, 1, 3, 4, 5]] = 0.0
    X = torch.linalg.inv(A) @ dA
    t = X.diagonal(dim1=-2, dim2=-1).sum(-1)
    assert _rel(t * t, torch.einsum("wab,wba->w", X, X)) < 1e-10


def test_table_local_energy_matches_explicit():
    mol = qi.make_co(n_det=30)
    wf = O.Wavefunction(mol)
    r = _walkers(mol, 8)
    assert _rel(O.local_energy_table(wf, r), O.local_energy(wf, r)) < 1e-11


# --------------------------------------------------------------------------
# physics invariants


def test_antisymmetry_same_spin_swap():
    for mol in (qi.make_lih(), qi.make_co(n_det=20), qi.make_li2(), qi.with_manybody_jastrow(qi.make_lih())):
        wf = O.Wavefunction(mol)
        r = _walkers(mol, 8)
        rs = r.clone()
        rs[:, [0, 1]] = r[:, [1, 0]]
        lp, sg = O.log_psi(wf, r)
        lps, sgs = O.log_psi(wf, rs)
        assert torch.allclose(lp, lps, atol=1e-12, rtol=0)
        assert torch.all(sg == -sgs)
        assert _rel(O.local_energy(wf, rs), O.local_energy(wf, r)) < 1e-11


def test_electron_electron_cusp_antiparallel():
    """Opposite-spin coalescence with u'(0) = 1/2: the kinetic -2 u'(0)/r12
    cancels +1/r12, so r12 E_L -> 0; without the Jastrow r12 E_L -> 1."""
    mol = qi.make_h2()
    base = _walkers(mol, 4)
    for jas, target in ((True, 0.0), (False, 1.0)):
        m = qi.make_h2()
        if not jas:
            m.jastrow_w0_anti = 0.0
            m.jastrow_w0_par = 0.0
        wf = O.Wavefunction(m)
        for eps in (1e-5, 1e-7):
            r = base.clone()
            r[:, 1] = r[:, 0] + eps * torch.tensor([0.6, 0.0, 0.8], dtype=torch.float64)
            val = eps * O.local_energy(wf, r)
            assert torch.allclose(val, torch.full_like(val, target), atol=50 * eps)


def test_translation_invariance():
    for mol in (qi.make_lih(), qi.make_co(n_det=10), qi.make_li2()):
        wf = O.Wavefunction(mol)
        r = _walkers(mol, 6)
        shift = np.array([0.3, -1.1, 0.7])
        wf2 = O.Wavefunction(mol.with_geometry(mol.atom_xyz + shift))
        assert _rel(O.local_energy(wf2, r + torch.tensor(shift)), O.local_energy(wf, r)) < 1e-11


def test_rotation_invariance_s_basis():
    mol = qi.make_h2()
    wf = O.Wavefunction(mol)
    r = _walkers(mol, 8)
    th = 0.7
    R = np.array([[1, 0, 0], [0, math.cos(th), -math.sin(th)], [0, math.sin(th), math.cos(th)]])
    wf2 = O.Wavefunction(mol.with_geometry(mol.atom_xyz @ R.T))
    assert _rel(O.local_energy(wf2, r @ torch.tensor(R.T)), O.local_energy(wf, r)) < 1e-12


# --------------------------------------------------------------------------
# gradient and force estimators against finite differences


@pytest.mark.parametrize("name", ["li2", "co_sd20", "lih_mbj"])
def test_grad_log_psi_finite_difference(name):
    """The oracle's autograd d log|Psi| / d theta against central
    differences, for the backflow single determinant (Li2), a 20-determinant
    CO expansion (CI weights, occupied and virtual MO columns) and LiH with
    the many-body Jastrow of App. D (its K_en and K_een parameters)."""
    mol = (qi.make_li2() if name == "li2" else qi.make_co(n_det=20) if name == "co_sd20"
           else qi.with_manybody_jastrow(qi.make_lih()))
    wf = O.Wavefunction(mol, requires_grad=True)
    r = _walkers(mol, 3)
    G = O.grad_log_psi(wf, r)
    params = list(wf.params().values())
    h = 1e-5
    off = 0
    rng = np.random.default_rng(0)
    extra = {"mo_coeff": [3 * mol.n_mo + 2, 5 * mol.n_mo + 10, 40 * mol.n_mo + 12], "det_weight": [1, 2, 7]}
    for key, p in zip(wf.params().keys(), params):
        n = p.numel()
        picks = [0, n - 1] + list(rng.integers(0, n, size=4)) + [j for j in extra.get(key, []) if j < n]
        for j in sorted(set(picks)):
            def central(step):
                with torch.no_grad():
                    flat = p.view(-1)
                    old = flat[j].item()
                    flat[j] = old + step
                    lp_p = O.log_psi(wf, r)[0]
                    flat[j] = old - step
                    lp_m = O.log_psi(wf, r)[0]
                    flat[j] = old
                return (lp_p - lp_m) / (2 * step)

            fd = (4.0 * central(h / 2) - central(h)) / 3.0  # Richardson: O(h^4)
            assert torch.allclose(G[:, off + j], fd, rtol=1e-6, atol=1e-7), (off, j)
        off += n


def test_force_and_gradient_estimators_finite_difference():
    mol = qi.make_li2()
    wf = O.Wavefunction(mol, requires_grad=True)
    r = _walkers(mol, 4)
    Ev, var, grad, F = O.energy_grad(wf, r)
    h = 1e-5
    M = r.shape[0]
    with torch.no_grad():
        E0, lp0, _ = O.local_energy(wf, r, return_parts=True)
        dE = E0 - E0.mean()
        for a in range(2):
            xyz = wf.atom_xyz
            old = xyz[a, 2].item()
            xyz[a, 2] = old + h
            Ep, lpp, _ = O.local_energy(wf, r, return_parts=True)
            xyz[a, 2] = old - h
            Em, lpm, _ = O.local_energy(wf, r, return_parts=True)
            xyz[a, 2] = old
            dEL = (Ep - Em) / (2 * h)
            dlr = 2 * (lpp - lpm) / (2 * h)
            Fz = -(dEL + dE * dlr).sum() / M
            assert abs(Fz.item() - F[a, 2].item()) < 1e-6 * max(1.0, abs(Fz.item()))
        # gradient estimator: backflow parameter (last entry)
        w = wf.backflow_w
        old = w.item()
        w.fill_(old + h)
        lpp = O.log_psi(wf, r)[0]
        w.fill_(old - h)
        lpm = O.log_psi(wf, r)[0]
        w.fill_(old)
        g_fd = (2 * (lpp - lpm) / (2 * h) * dE).sum() / M
        assert abs(g_fd.item() - grad[-1].item()) < 1e-6 * max(1.0, abs(g_fd.item()))
    assert abs(Ev.item() - E0.mean().item()) < 1e-12 and var.item() > 0


# --------------------------------------------------------------------------
# Metropolis sampler


def test_metropolis_counter_resume_and_batch_independence():
    mol = qi.make_h2()
    wf = O.Wavefunction(mol)
    r = _walkers(mol, 10)
    full, lp_full, acc_full = O.metropolis(wf, r, 12, 0.2, seed=99)
    half, _, acc1 = O.metropolis(wf, r, 7, 0.2, seed=99)
    rest, _, acc2 = O.metropolis(wf, half, 5, 0.2, seed=99, step_offset=7)
    assert torch.equal(rest, full) and torch.equal(acc1 + acc2, acc_full)
    a, _, _ = O.metropolis(wf, r[:4], 12, 0.2, seed=99)
    b, _, _ = O.metropolis(wf, r[4:], 12, 0.2, seed=99, first_walker=4)
    assert torch.equal(torch.cat([a, b]), full)


def test_metropolis_hydrogen_radial_distribution():
    """Exact 1s: |Psi|^2 radial density 4 r^2 exp(-2r); chi-square test."""
    from scipy import stats

    mol = qi.make_hydrogenic(1.0, 1.0)
    wf = O.Wavefunction(mol)
    r = _walkers(mol, 4000, seed=11)
    r, _, acc = O.metropolis(wf, r, 150, 0.6, seed=5)
    rr = r[:, 0].norm(dim=-1).numpy()
    edges = np.array([0, 0.3, 0.6, 0.9, 1.2, 1.6, 2.0, 2.6, 3.4, 5.0, np.inf])
    cdf = lambda x: 1 - np.exp(-2 * x) * (1 + 2 * x + 2 * x * x)
    expected = np.diff(np.where(np.isinf(edges), 1.0, cdf(np.minimum(edges, 1e9)))) * len(rr)
    observed = np.histogram(rr, bins=edges)[0]
    chi2 = ((observed - expected) ** 2 / expected).sum()
    assert stats.chi2.sf(chi2, len(expected) - 1) > 1e-3
    assert 0.2 < acc.float().mean() / 150 < 0.95


def test_metropolis_helium_mean_energy_within_3_sigma():
    mol = qi.make_helium(1.6875)
    wf = O.Wavefunction(mol)
    r = _walkers(mol, 3000, seed=12)
    r, _, _ = O.metropolis(wf, r, 120, 0.5, seed=6)
    Es = []
    for k in range(4):
        r, _, _ = O.metropolis(wf, r, 25, 0.5, seed=6, step_offset=120 + 25 * k)
        Es.append(O.local_energy(wf, r))
    per_walker = torch.stack(Es).mean(0)
    mean = per_walker.mean().item()
    err = per_walker.std().item() / math.sqrt(per_walker.numel())
    assert abs(mean - (-2.84765625)) < 3 * err, (mean, err)


# --------------------------------------------------------------------------
# planted mistakes: the pins above must catch them


def test_planted_mistake_in_jastrow_laplacian_is_caught(monkeypatch):
    mol = qi.make_lih()
    wf = O.Wavefunction(mol)
    r = _walkers(mol, 4)
    good = O.local_energy_ad(wf, r)
    real = O.jastrow

    def wrong(wf_, r_):
        J, gJ, lJ = real(wf_, r_)
        return J, gJ, 0.5 * lJ  # drop half of the pair Laplacian

    monkeypatch.setattr(O, "jastrow", wrong)
    assert _rel(O.local_energy(wf, r), good) > 1e-6


def test_planted_mistake_in_transposed_inverse_is_caught(monkeypatch):
    mol = qi.make_lih()
    wf = O.Wavefunction(mol)
    r = _walkers(mol, 4)
    good = O.local_energy_ad(wf, r)
    real_inv = torch.linalg.inv
    monkeypatch.setattr(torch.linalg, "inv", lambda A: real_inv(A).transpose(-1, -2))
    assert _rel(O.local_energy(wf, r), good) > 1e-6


def test_energy_gradient_sums_assemble_to_the_estimator():
    """The per-batch sums assembled by the closed formulas give the same
    estimator as the direct one, with the batch mean as E_v (Eq. nabla_loss,
    Eq. force); and splitting the batch into two parts and adding their sums
    changes nothing (the sums are additive)."""
    mol = qi.make_lih()
    wf = O.Wavefunction(mol, requires_grad=True)
    r = torch.tensor(qi.walkers(mol, 24, seed=52))
    Ev, var, grad, F = O.energy_grad(wf, r)
    n_param = sum(p.numel() for p in wf.params().values())
    whole = O.energy_grad_sums(wf, r)
    parts = O.energy_grad_sums(wf, r[:10]) + O.energy_grad_sums(wf, r[10:])
    assert whole.shape[0] == 3 + 2 * n_param + 9 * mol.n_atom
    for sums in (whole, parts):
        ev2, var2, g2, f2 = O.assemble_energy_grad(sums, n_param, mol.n_atom)
        assert abs(float(ev2 - Ev)) <= 1e-12 * abs(float(Ev))
        assert abs(float(var2 - var)) <= 1e-10 * float(var)
        assert float((g2 - grad).abs().max()) <= 1e-12 * float(grad.abs().max())
        assert float((f2 - F).abs().max()) <= 1e-12 * max(1.0, float(F.abs().max()))
