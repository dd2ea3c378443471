"""Helpers shared by the GPU parity tests (oracle references and tolerances).

Tolerances (per walker):
* FP64 form: |dE| <= 1e-10 * max(1, |E|) for walkers whose rounding
  sensitivity s (max 1-norm condition number of the reference Slater
  matrices times the CI cancellation factor sum|d_n D_n| / |sum d_n D_n|) is
  at most 1e4; the remaining near-node walkers (expected well under 1%) must
  still agree to 1e-10 * s.  FP64 rounding of the trace formulas is of order
  1e-16 * s times the term magnitudes (|kinetic terms| <~ 1e3 Ha), which
  these bounds contain with margin.
* FP32 / mixed forms: |dE| <= 2e-4 Ha for walkers with s <= 1e3, the rest
  counted and reported.  FP32 AO and MO channels carry a relative error of
  about 6e-8 times the term magnitudes, amplified by s through the
  determinant ratios.
"""
import numpy as np
import torch

import qmc_inputs as qi
from oracle import qmc_oracle as O

_CACHE = {}


def oracle_reference(mol, r):
    """(E_L, log|Psi|, sensitivity) from the oracle, cached per input."""
    key = (mol.name, mol.n_det, r.shape, float(r.sum()), float(mol.atom_xyz.sum()))
    if key not in _CACHE:
        wf = O.Wavefunction(mol)
        rt = torch.tensor(r)
        E, lp, _ = O.local_energy(wf, rt, return_parts=True)
        s = O.sensitivity(wf, rt)
        _CACHE[key] = (E.numpy(), lp.numpy(), s.numpy())
    return _CACHE[key]


def fp64_check(E_gpu, E_ref, sens, s_max=1e4, rel=1e-10, max_excluded=0.01):
    err = np.abs(E_gpu - E_ref) / np.maximum(1.0, np.abs(E_ref))
    good = sens <= s_max
    assert np.isfinite(E_gpu[good]).all()
    assert good.mean() >= 1.0 - max_excluded, good.mean()
    worst = float(err[good].max()) if good.any() else 0.0
    assert worst <= rel, worst
    assert np.all(err[~good] <= rel * sens[~good]), err[~good].max()
    return worst


def mixed_check(E_gpu, E_ref, sens, s_max=1e3, tol=2e-4, max_excluded=0.01):
    err = np.abs(E_gpu - E_ref)
    good = sens <= s_max
    assert good.mean() >= 1.0 - max_excluded, good.mean()
    assert np.isfinite(E_gpu[good]).all()
    stats = dict(median=float(np.median(err[good])), p99=float(np.quantile(err[good], 0.99)),
                 max=float(err[good].max()), excluded=int((~good).sum()))
    assert stats["max"] <= tol, stats
    return stats
