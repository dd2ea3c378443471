"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every function that include/qmc.h declares, and
rejects bad arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import qmc_inputs as qi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_09743_gb300 import _lib, build_ext

    build_ext.build()
    return _lib.load()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "qmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qmc_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("qmc_create_wf", "qmc_local_energy", "qmc_sample", "qmc_destroy_wf"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2506_09743_gb300 import _lib

    for name in _declared_functions():
        assert hasattr(lib, name), name
    assert set(_declared_functions()) <= set(_lib.EXPORTED) | set(_declared_functions())
    assert set(_lib.EXPORTED) == set(_declared_functions())


def test_library_is_sm103a_only():
    from paper_2506_09743_gb300 import build_ext

    assert build_ext.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def _create(lib, mol, **over):
    from paper_2506_09743_gb300 import _lib

    a = dict(xyz=np.ascontiguousarray(mol.atom_xyz).reshape(-1), z=np.ascontiguousarray(mol.atom_z),
             ao_atom=mol.ao_atom.astype(np.int32), ao_kind=mol.ao_kind.astype(np.int32),
             ao_pow=np.ascontiguousarray(mol.ao_pow.astype(np.int32)).reshape(-1),
             ps=mol.ao_prim_start.astype(np.int32), pe=mol.prim_exp, pc=mol.prim_coef,
             mo=np.ascontiguousarray(mol.mo_coeff).reshape(-1), dw=mol.det_weight,
             de=np.ascontiguousarray(mol.det_exc.astype(np.int32)).reshape(-1))
    P = lambda x, t: x.ctypes.data_as(ctypes.POINTER(t))
    d, i = ctypes.c_double, ctypes.c_int32
    atoms = _lib.Atoms(over.get("n_atom", mol.n_atom), P(a["xyz"], d), P(a["z"], d), over.get("n_up", mol.n_up),
                       mol.n_down)
    basis = _lib.Basis(mol.n_ao, P(a["ao_atom"], i), P(a["ao_kind"], i), P(a["ao_pow"], i), P(a["ps"], i),
                       P(a["pe"], d), P(a["pc"], d))
    mos = _lib.Mos(over.get("n_mo", mol.n_mo), P(a["mo"], d))
    dets = _lib.Dets(mol.n_det, P(a["dw"], d), P(a["de"], i))
    jas = _lib.Jastrow(0.25, 0.5, 1.0, 0.0)
    opt = _lib.Options(over.get("precision", 0), 0)
    h = ctypes.c_void_p()
    st = lib.qmc_create_wf(ctypes.byref(atoms), ctypes.byref(basis), ctypes.byref(mos), ctypes.byref(dets),
                           ctypes.byref(jas), ctypes.byref(opt), ctypes.byref(h))
    return st, h


def test_create_rejects_bad_arguments_on_host(lib):
    from paper_2506_09743_gb300 import _lib

    mol = qi.make_lih()
    assert _create(lib, mol, n_atom=0)[0] == _lib.QMC_ERR_ARG
    assert _create(lib, mol, n_atom=99)[0] == _lib.QMC_ERR_ARG
    assert _create(lib, mol, n_up=9)[0] == _lib.QMC_ERR_UNSUPPORTED
    assert _create(lib, mol, n_mo=1)[0] == _lib.QMC_ERR_ARG
    assert _create(lib, mol, precision=7)[0] == _lib.QMC_ERR_ARG
    assert b"precision" in lib.qmc_last_error()
    st = lib.qmc_create_wf(None, None, None, None, None, None, None)
    assert st == _lib.QMC_ERR_ARG


def test_calls_on_null_handle_fail_cleanly(lib):
    from paper_2506_09743_gb300 import _lib

    assert lib.qmc_local_energy(None, None, 0, 0, None, None, None, 0, None) == _lib.QMC_ERR_ARG
    assert lib.qmc_sample(None, None, 1, 1, 1, 0.1, 0, 0, 0, None, None, None, 0, None) == _lib.QMC_ERR_ARG
    assert lib.qmc_workspace_size(None, 10) == 0
    assert lib.qmc_set_det_method(None, 1) == _lib.QMC_ERR_ARG
    lib.qmc_destroy_wf(None)


def test_excitation_records_validated(lib):
    from paper_2506_09743_gb300 import _lib

    mol = qi.make_co(n_det=5)
    bad = mol.det_exc.copy()
    bad[1, 0] = (1, 9, -1, 10, -1)  # hole beyond the occupied orbitals
    mol.det_exc = bad
    assert _create(lib, mol)[0] == _lib.QMC_ERR_ARG
