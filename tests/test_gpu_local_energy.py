"""GPU parity of qmc_local_energy against the CPU oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import qmc_inputs as qi
from oracle import qmc_oracle as O

from gpu_common import fp64_check, oracle_reference, reduced_check

pytestmark = pytest.mark.gpu

MOLS = {
    "h2": lambda: qi.make_h2(),
    "lih": lambda: qi.make_lih(),
    "co": lambda: qi.make_co(),
}


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2506_09743_gb300 as p

    return p


def _run(pkg, mol, r, precision, ldw_pad=0):
    wf = pkg.Wavefunction(mol, precision=precision)
    x = torch.zeros(3 * mol.n_elec, r.shape[0] + ldw_pad, dtype=torch.float64, device="cuda")
    x[:, : r.shape[0]] = torch.tensor(qi.to_soa(r), device="cuda")
    e, lp = wf.local_energy(x, n_walkers=r.shape[0])
    torch.cuda.synchronize()
    out = e.cpu().numpy(), lp.cpu().numpy()
    wf.close()
    return out


# 1000 walkers: several 64/128-walker tiles and a ragged tail
@pytest.mark.parametrize("name", ["h2", "lih", "co"])
def test_fp64_parity(pkg, name):
    mol = MOLS[name]()
    r = qi.walkers(mol, 1000, seed=21)
    E_ref, lp_ref, sens = oracle_reference(mol, r)
    E, lp = _run(pkg, mol, r, "fp64", ldw_pad=7)
    st = fp64_check(E, E_ref, sens)
    assert np.all(np.abs(lp - lp_ref) <= 128 * 2.0 ** -53 * sens * np.maximum(1, np.abs(lp_ref)))
    print(f"{name} fp64 rel err {st}")


@pytest.mark.parametrize("name", ["h2", "lih", "co"])
@pytest.mark.parametrize("precision", ["fp32", "mixed_tf32", "fp32x2"])
def test_reduced_precision_parity(pkg, name, precision):
    mol = MOLS[name]()
    r = qi.walkers(mol, 1000, seed=22)
    E_ref, lp_ref, sens = oracle_reference(mol, r)
    E, lp = _run(pkg, mol, r, precision)
    st = reduced_check(precision, E, E_ref, sens)
    print(f"{name} {precision} |dE| Ha {st}")


def _co_with_general_shells():
    """CO plus AOs outside the complete s/p/d shells: a Cartesian f shell on C
    (l = 3), an incomplete d shell (xy, zz) and a lone p_x on O, with small
    random MO coefficients on the new AOs."""
    import dataclasses

    mol = qi.make_co(n_det=20)
    rng = np.random.default_rng(17)
    extra = [(0, (3, 0, 0)), (0, (2, 1, 0)), (0, (2, 0, 1)), (0, (1, 2, 0)), (0, (1, 1, 1)),
             (0, (1, 0, 2)), (0, (0, 3, 0)), (0, (0, 2, 1)), (0, (0, 1, 2)), (0, (0, 0, 3)),
             (1, (1, 1, 0)), (1, (0, 0, 2)), (1, (1, 0, 0))]
    atom, pw, start = list(mol.ao_atom), [list(p) for p in mol.ao_pow], list(mol.ao_prim_start)
    pexp, pcoef = list(mol.prim_exp), list(mol.prim_coef)
    groups = {}
    for k, (a, (x, y, z)) in enumerate(extra):
        key = (a, x + y + z, k >= 12)
        if key not in groups:
            groups[key] = (np.sort(np.exp(rng.uniform(np.log(0.3), np.log(8.0), size=2)))[::-1],
                           rng.uniform(0.2, 1.0, size=2))
        al, c = groups[key]
        atom.append(a)
        pw.append([x, y, z, 0])
        pexp.extend(al)
        pcoef.extend(c)
        start.append(len(pexp))
    mo = np.vstack([mol.mo_coeff, 0.05 * rng.standard_normal((len(extra), mol.n_mo))])
    return dataclasses.replace(
        mol, name="co_general_shells", ao_atom=np.asarray(atom, np.int32),
        ao_kind=np.concatenate([mol.ao_kind, np.full(len(extra), qi.GTO, np.int32)]),
        ao_pow=np.asarray(pw, np.int32), ao_prim_start=np.asarray(start, np.int32),
        prim_exp=np.asarray(pexp), prim_coef=np.asarray(pcoef), mo_coeff=mo)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed_tf32", "fp32x2"])
def test_general_shells_parity(pkg, precision):
    """f shells and incomplete shells take the general angular path of the AO
    stages (the tensor-core stage evaluates complete s/p/d shells in a
    canonical column order and everything else by powers)."""
    mol = _co_with_general_shells()
    r = qi.walkers(mol, 300, seed=23)
    E_ref, _, sens = oracle_reference(mol, r)
    E, _ = _run(pkg, mol, r, precision)
    if precision == "fp64":
        fp64_check(E, E_ref, sens, min_within=0.98)
    else:
        reduced_check(precision, E, E_ref, sens)


@pytest.mark.parametrize("precision", ["fp64", "mixed_tf32", "fp32x2"])
@pytest.mark.parametrize("n_det", [1, 100, 1716])
def test_explicit_method_parity(pkg, precision, n_det):
    """Explicit per-excitation LU (the baseline of the paper's comparison,
    Sec. 2.2 / App. A) against the oracle, and against the table method."""
    mol = qi.make_co(n_det=n_det)
    r = qi.walkers(mol, 200, seed=24)
    E_ref, lp_ref, sens = oracle_reference(mol, r)
    out = {}
    for method in ("explicit", "table"):
        wf = pkg.Wavefunction(mol, precision=precision)
        wf.set_det_method(method)
        x = torch.tensor(qi.to_soa(r), device="cuda")
        e, lp = wf.local_energy(x)
        torch.cuda.synchronize()
        out[method] = (e.cpu().numpy(), lp.cpu().numpy())
        wf.close()
    E, lp = out["explicit"]
    if precision == "fp64":
        fp64_check(E, E_ref, sens, min_within=0.97)
        scale = np.maximum(1.0, np.abs(lp_ref))
        assert np.all(np.abs(lp - lp_ref) <= 128 * 2.0 ** -53 * sens * scale)
    else:
        reduced_check(precision, E, E_ref, sens)
    # both methods see the same MO values; they differ by rounding only
    Et = out["table"][0]
    bound = 128 * (2.0 ** -53) * sens * np.maximum(1.0, np.abs(E_ref))
    if precision == "fp64":
        assert np.all(np.abs(E - Et) <= 2 * bound)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed_tf32", "fp32x2"])
@pytest.mark.parametrize("name", ["lih", "co"])
def test_manybody_jastrow_parity(pkg, name, precision):
    """Electron-nucleus and electron-electron-nucleus Jastrow kernels (App. D)
    in every precision form against the oracle."""
    base = qi.make_lih() if name == "lih" else qi.make_co(n_det=20)
    mol = qi.with_manybody_jastrow(base)
    r = qi.walkers(mol, 300 if name == "lih" else 150, seed=25)
    E_ref, lp_ref, sens = oracle_reference(mol, r)
    E, lp = _run(pkg, mol, r, precision)
    if precision == "fp64":
        fp64_check(E, E_ref, sens, min_within=0.98)
        scale = np.maximum(1.0, np.abs(lp_ref))
        assert np.all(np.abs(lp - lp_ref) <= 128 * 2.0 ** -53 * sens * scale + 1e-13 * scale)
    else:
        reduced_check(precision, E, E_ref, sens)
    # the terms change the energy (the test is not vacuous)
    E0, _, _ = oracle_reference(base, r)
    assert np.abs(E_ref - E0).max() > 1e-3


def test_manybody_jastrow_hydrogen_closed_form_on_gpu(pkg):
    import dataclasses

    w0, w1, w2 = -0.2, 0.03, 0.8
    mol = dataclasses.replace(qi.make_hydrogenic(1.0, 1.0), jastrow_en=np.array([w0, w1, w2]))
    r = qi.walkers(mol, 200, seed=26)
    x = np.linalg.norm(r[:, 0], axis=-1)
    d = 1 + w2 * x
    K1 = (w0 + w1 * x * (2 + w2 * x)) / d ** 2
    K2 = 2 * (w1 - w0 * w2) / d ** 3
    ref = -0.5 * ((K1 - 1) ** 2 + K2 + 2 * (K1 - 1) / x) - 1 / x
    E, _ = _run(pkg, mol, r, "fp64")
    assert np.abs(E - ref).max() < 1e-12 * np.abs(ref).max()


def test_manybody_jastrow_scope(pkg):
    from paper_2506_09743_gb300 import QmcError

    wf = pkg.Wavefunction(qi.with_manybody_jastrow(qi.make_lih()), precision="fp64")
    x = torch.tensor(qi.to_soa(qi.walkers(qi.make_lih(), 16, seed=1)), device="cuda")
    with pytest.raises(QmcError):
        wf.energy_grad(x)
    with pytest.raises(QmcError):
        wf.set_manybody_jastrow([0.1, 0.0, -1.0], None)  # pole: w2 < 0
    wf.set_manybody_jastrow(None, None)  # off again: the plain Pade energy
    e, _ = wf.local_energy(x)
    ref = pkg.Wavefunction(qi.make_lih(), precision="fp64")
    e0, _ = ref.local_energy(x)
    assert torch.equal(e, e0)
    wf.close()
    ref.close()
    with pytest.raises(QmcError):
        pkg.Wavefunction(qi.with_manybody_jastrow(qi.make_li2()), precision="fp64")


def _h_chain(n_atom, n_terms):
    """Linear H chain, one 1s STO per atom, n_atom electrons, with the
    many-body Jastrow of n_terms e-e-n terms."""
    bb = qi._BasisBuilder()
    for a in range(n_atom):
        bb.add(a, qi.STO, 0, 0, 0, 0, [1.1], [1.0])
    xyz = np.zeros((n_atom, 3))
    xyz[:, 2] = 1.6 * (np.arange(n_atom) - (n_atom - 1) / 2)
    z = np.ones(n_atom)
    nu = n_atom // 2
    mo = qi.random_orthonormal(n_atom, nu, np.random.default_rng(3))
    mol = qi.Molecule(name=f"h{n_atom}", atom_xyz=xyz, atom_z=z, n_up=nu, n_down=n_atom - nu, **bb.arrays(),
                      mo_coeff=mo, det_weight=np.ones(1),
                      det_exc=qi._dets_array([(qi.ground_exc(), qi.ground_exc())]),
                      electron_home=qi.electron_homes(z, nu, n_atom - nu))
    return qi.with_manybody_jastrow(mol, n_terms=n_terms)


def test_manybody_een_shared_memory_limit(pkg):
    """The e-e-n tables of 12 electrons x 12 atoms x 8 terms need 266 KB per
    block in FP64 (refused) and 133 KB in FP32 (accepted)."""
    from paper_2506_09743_gb300 import QmcError

    mol = _h_chain(12, 8)
    with pytest.raises(QmcError):
        pkg.Wavefunction(mol, precision="fp64")
    wf = pkg.Wavefunction(mol, precision="mixed_tf32")
    r = qi.walkers(mol, 300, seed=6)
    e, _ = wf.local_energy(torch.tensor(qi.to_soa(r), device="cuda"))
    wf.close()
    E_ref, _, sens = oracle_reference(mol, r)
    reduced_check("mixed_tf32", e.cpu().numpy(), E_ref, sens)


def test_closed_forms_on_gpu(pkg):
    mol = qi.make_hydrogenic(1.0, 1.0)
    r = qi.walkers(mol, 333, seed=4)
    E, _ = _run(pkg, mol, r, "fp64")
    assert np.abs(E + 0.5).max() < 1e-13
    he = qi.make_helium(1.6875)
    r = qi.walkers(he, 257, seed=5)
    z = 1.6875
    r1, r2 = np.linalg.norm(r[:, 0], axis=-1), np.linalg.norm(r[:, 1], axis=-1)
    r12 = np.linalg.norm(r[:, 0] - r[:, 1], axis=-1)
    ref = -z * z + (z - 2) * (1 / r1 + 1 / r2) + 1 / r12
    # FP32X2: the electron-electron term 1/r12 is a refined FP32 reciprocal
    # (within 2^-22 of itself); the rest is exact to the pairs' 2^-44
    for prec, tol in (("fp64", 1e-12), ("mixed_tf32", 1e-4), ("fp32x2", 2.0 ** -21)):
        E, _ = _run(pkg, he, r, prec)
        assert np.abs(E - ref).max() < tol * np.maximum(1, np.abs(ref)).max(), prec


@pytest.mark.parametrize("W", [1, 31, 129])
def test_small_and_ragged_batches(pkg, W):
    mol = qi.make_co(n_det=20)
    r = qi.walkers(mol, W, seed=6)
    E_ref, _, sens = oracle_reference(mol, r)
    for prec in ("fp64", "mixed_tf32", "fp32x2"):
        E, _ = _run(pkg, mol, r, prec, ldw_pad=3)
        if prec == "fp64":
            fp64_check(E, E_ref, sens, min_within=0.0 if W < 100 else 0.99)
        else:
            reduced_check(prec, E, E_ref, sens)


def test_zero_walkers_is_a_noop(pkg):
    mol = qi.make_h2()
    wf = pkg.Wavefunction(mol)
    x = torch.zeros(6, 4, dtype=torch.float64, device="cuda")
    e = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    wf.local_energy(x, n_walkers=0, e_loc=e, log_psi=e)
    assert e.item() == 7.0


def test_caller_workspace_and_too_small_workspace(pkg):
    from paper_2506_09743_gb300 import QmcError

    mol = qi.make_lih()
    r = qi.walkers(mol, 300, seed=8)
    wf = pkg.Wavefunction(mol)
    x = torch.tensor(qi.to_soa(r), device="cuda")
    need = wf.workspace_size(300)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    e1, _ = wf.local_energy(x, workspace=ws)
    e2, _ = wf.local_energy(x)
    torch.cuda.synchronize()
    assert torch.equal(e1, e2)
    with pytest.raises(QmcError) as ei:
        wf.local_energy(x, workspace=ws[: need // 2])
    assert "workspace" in str(ei.value)


@pytest.mark.parametrize("precision", ["mixed_tf32", "fp32", "fp64"])
def test_set_params_rebuilds_every_table(pkg, precision):
    """New exponents, MO coefficients, CI weights and Jastrow b installed with
    qmc_set_params give the energies of a wavefunction built from them (the
    tensor-core operand, shell tables and excitation weights are rebuilt)."""
    import dataclasses

    mol = qi.make_co(n_det=20)
    r = qi.walkers(mol, 257, seed=27)
    wf = pkg.Wavefunction(mol, precision=precision)
    n, off = wf.param_layout()
    rng = np.random.default_rng(3)
    p = np.concatenate([mol.prim_exp, mol.mo_coeff.reshape(-1), mol.det_weight, [mol.jastrow_b, 0.0]])
    assert p.shape[0] == n
    p2 = p.copy()
    p2[off[0]:off[1]] *= rng.uniform(0.9, 1.1, off[1] - off[0])
    p2[off[1]:off[2]] += 0.01 * rng.standard_normal(off[2] - off[1])
    p2[off[2]:off[3]] *= rng.uniform(0.8, 1.2, off[3] - off[2])
    p2[off[3]] = 0.8
    wf.set_params(p2)
    x = torch.tensor(qi.to_soa(r), device="cuda")
    e1, lp1 = wf.local_energy(x)
    mol2 = dataclasses.replace(mol, prim_exp=p2[off[0]:off[1]].copy(),
                               mo_coeff=p2[off[1]:off[2]].reshape(mol.mo_coeff.shape).copy(),
                               det_weight=p2[off[2]:off[3]].copy(), jastrow_b=0.8)
    fresh = pkg.Wavefunction(mol2, precision=precision)
    e2, lp2 = fresh.local_energy(x)
    torch.cuda.synchronize()
    assert torch.equal(e1, e2) and torch.equal(lp1, lp2)
    wf.close()
    fresh.close()


def _host_buffers(soa, W, pinned):
    """(walkers, e_loc, log_psi) host arrays, page-locked or pageable."""
    if not pinned:
        return soa, np.empty(W), np.empty(W)
    bufs = [torch.from_numpy(soa).pin_memory(), torch.empty(W, dtype=torch.float64).pin_memory(),
            torch.empty(W, dtype=torch.float64).pin_memory()]
    return tuple(b.numpy() for b in bufs)


@pytest.mark.parametrize("W,pinned", [(500, False), (70001, False), (500, True), (70001, True)])
def test_host_entry_point_matches_device(pkg, W, pinned):
    """The host-buffer entry point gives the device call's results bit for
    bit, from pageable host memory (uploaded before the first kernel) and
    from page-locked memory (read by the first kernel over the host link)."""
    mol = qi.make_co(n_det=30)
    r = qi.walkers(mol, W, seed=9)
    wf = pkg.Wavefunction(mol, precision="mixed_tf32")
    soa = np.ascontiguousarray(qi.to_soa(r))
    x_h, e_h, lp_h = _host_buffers(soa, W, pinned)
    wf.local_energy_host(x_h, e_loc=e_h, log_psi=lp_h)
    e_d, lp_d = wf.local_energy(torch.tensor(soa, device="cuda"))
    torch.cuda.synchronize()
    assert np.array_equal(e_h, e_d.cpu().numpy()) and np.array_equal(lp_h, lp_d.cpu().numpy())
    wf.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed_tf32"])
def test_host_entry_point_pinned_manybody(pkg, precision):
    """Page-locked host walkers with the many-body Jastrow (its second kernel
    reads the device copy the first one wrote), both precision forms."""
    mol = qi.with_manybody_jastrow(qi.make_lih())
    W = 4099
    r = qi.walkers(mol, W, seed=12)
    wf = pkg.Wavefunction(mol, precision=precision)
    soa = np.ascontiguousarray(qi.to_soa(r))
    x_h, e_h, lp_h = _host_buffers(soa, W, True)
    for _ in range(2):  # the second call reuses the staging buffer
        wf.local_energy_host(x_h, e_loc=e_h, log_psi=lp_h)
        e_d, lp_d = wf.local_energy(torch.tensor(soa, device="cuda"))
        torch.cuda.synchronize()
        assert np.array_equal(e_h, e_d.cpu().numpy()) and np.array_equal(lp_h, lp_d.cpu().numpy())
        soa = np.ascontiguousarray(soa[:, ::-1])
        x_h[...] = soa
    wf.close()


def test_full_size_co_sampled_parity(pkg):
    """CO at its full 262,144-walker size in the launch configuration the
    benchmark times; 256 sampled walkers checked against the oracle."""
    mol = qi.make_co()
    W = qi.WORKLOAD_WALKERS["co"]
    r = qi.walkers(mol, W, seed=qi.SEED_WALKERS)
    idx = np.random.default_rng(0).choice(W, size=256, replace=False)
    E_ref, _, sens = oracle_reference(mol, r[idx])
    x = torch.tensor(qi.to_soa(r), device="cuda")
    for prec in ("fp64", "mixed_tf32", "fp32x2"):
        wf = pkg.Wavefunction(mol, precision=prec)
        e, _ = wf.local_energy(x)
        torch.cuda.synchronize()
        E = e.cpu().numpy()
        assert np.isfinite(E).mean() > 0.999
        if prec == "fp64":
            fp64_check(E[idx], E_ref, sens)
        else:
            print(prec, reduced_check(prec, E[idx], E_ref, sens))
        wf.close()


def test_set_geometry_matches_fresh_wavefunction(pkg):
    mol = qi.make_lih()
    r = qi.walkers(mol, 200, seed=10)
    stretched = mol.with_bond_scale(1.7)
    wf = pkg.Wavefunction(mol)
    wf.set_geometry(stretched.atom_xyz)
    x = torch.tensor(qi.to_soa(r), device="cuda")
    e1, _ = wf.local_energy(x)
    e2, _ = _run(pkg, stretched, r, "fp64")
    torch.cuda.synchronize()
    assert np.allclose(e1.cpu().numpy(), e2, rtol=0, atol=0)


@pytest.mark.parametrize("name", ["co", "lih"])
def test_fp32x2_near_a_nucleus(pkg, name):
    """Electrons within 2^-12 bohr of a nucleus (here within 1.7e-4 bohr,
    |E_L| up to 1e5 Ha): the FP32X2 tensor-core AO stage takes its row scales
    from the shells one by one there (outside the per-atom bound tables);
    such walkers meet the same 2e-4 Ha gate."""
    from gpu_common import gated_check

    mol = MOLS[name]()
    r = qi.walkers(mol, 200, seed=23)
    rng = np.random.default_rng(5)
    for w in range(0, 200, 2):  # every other walker: one electron next to a nucleus
        a = w % mol.n_atom
        i = (w // 2) % mol.n_elec
        r[w, i] = mol.atom_xyz[a] + rng.uniform(-1e-4, 1e-4, size=3)
    E_ref, _, sens = oracle_reference(mol, r)
    E, _ = _run(pkg, mol, r, "fp32x2")
    st = gated_check(E, E_ref, sens)
    print(name, "near-nucleus fp32x2", st)


@pytest.mark.parametrize("name", ["co", "lih"])
def test_fp32x2_near_coalescence(pkg, name):
    """Electron pairs of opposite spin within 1e-4 bohr: the FP32X2 Coulomb
    stage sums 1/r_ij of such pairs in pairs of FP32 (an FP32 term would cost
    2^-22 of 1e4 Ha); the walkers meet the same 2e-4 Ha gate."""
    from gpu_common import gated_check

    mol = MOLS[name]()
    r = qi.walkers(mol, 200, seed=24)
    rng = np.random.default_rng(6)
    for w in range(0, 200, 2):
        i = (w // 2) % mol.n_up
        j = mol.n_up + (w // 2) % mol.n_down
        r[w, j] = r[w, i] + rng.uniform(-1e-4, 1e-4, size=3)
    E_ref, _, sens = oracle_reference(mol, r)
    E, _ = _run(pkg, mol, r, "fp32x2")
    st = gated_check(E, E_ref, sens)
    print(name, "near-coalescence fp32x2", st)


def _co_rows(n_up, n_down, n_det=100):
    """The CO basis, MOs and Jastrow with n_up / n_down electrons and 100
    determinants of SD over its 14 orbitals (up to 5 active holes per spin)."""
    import dataclasses

    co = qi.make_co()
    all_dets = qi.sd_expansion(n_up, n_down, 14, max(0, min(n_up, n_down) - 5))
    dets = qi._dets_array(qi._select_dets(all_dets, n_det, np.random.default_rng(qi.SEED_DETS)))
    return dataclasses.replace(
        co, name=f"co_rows_{n_up}_{n_down}", n_up=n_up, n_down=n_down, det_exc=dets,
        det_weight=qi._ci_weights(len(dets), np.random.default_rng(qi.SEED_CI)),
        electron_home=qi.electron_homes(co.atom_z, n_up, n_down))


# Spin blocks of 4 to 8 rows, equal and unequal per spin: the FP64 stage of
# these expansions costs 3,522 to 7,544 flops per walker, so the FP32X2 form
# runs its pair-of-FP32 determinant stage (one instantiation per block size;
# two spin groups of a warp with different row counts), the FP64 form k_det.
@pytest.mark.parametrize("n_up,n_down", [(4, 4), (5, 4), (6, 6), (7, 6), (8, 8)])
def test_determinant_stage_block_sizes(pkg, n_up, n_down):
    mol = _co_rows(n_up, n_down)
    r = qi.walkers(mol, 300, seed=23)
    E_ref, lp_ref, sens = oracle_reference(mol, r)
    E64, lp64 = _run(pkg, mol, r, "fp64", ldw_pad=5)
    st64 = fp64_check(E64, E_ref, sens)
    assert np.all(np.abs(lp64 - lp_ref) <= 128 * 2.0 ** -53 * sens * np.maximum(1, np.abs(lp_ref)))
    E, lp = _run(pkg, mol, r, "fp32x2")
    st = reduced_check("fp32x2", E, E_ref, sens)
    # log|Psi|: the FP32X2 Jastrow sums FP32 pair terms |u| <= w0 / b = 0.5
    # (a few ulp each, 2^-21 allowed), the pair-of-FP32 orbitals and
    # determinants add about 2^-44 s (2^-40 s allowed)
    n = mol.n_up + mol.n_down
    tol_lp = 2.0 ** -21 * (n * (n - 1) // 2) * 0.5 + 2.0 ** -40 * sens
    assert np.all(np.abs(lp - lp_ref) <= tol_lp), float(np.max(np.abs(lp - lp_ref) / tol_lp))
    print(f"rows {n_up}/{n_down} fp64 {st64} fp32x2 {st}")
