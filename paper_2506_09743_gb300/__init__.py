"""GB300-native variational Monte Carlo local-energy engine (QMCTorch method).

Python side of the C ABI declared in ``include/qmc.h``: argument marshalling
only.  Every step of the computation runs in the CUDA library
``libqmc_gb300.so``; PyTorch provides device memory and streams.

    from paper_2506_09743_gb300 import Wavefunction
    wf = Wavefunction(molecule, precision="mixed_tf32")
    e_loc, log_psi = wf.local_energy(walkers_soa)      # torch CUDA float64 [3N, W]
    wf.sample(walkers_soa, n_steps=50, step=0.2, seed=1)
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import PRECISIONS, QmcError  # noqa: F401

__all__ = ["Wavefunction", "QmcError", "PRECISIONS", "library"]


def library():
    """The loaded ctypes library (raises if it has not been built)."""
    return _lib.load()


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _stream_handle(stream):
    if stream is None:
        import torch

        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Wavefunction:
    """A device-resident Slater-Jastrow(-backflow) wavefunction.

    ``mol`` is a ``qmc_inputs.Molecule`` (plain arrays).  ``precision`` is one
    of ``fp64``, ``fp32``, ``mixed_tf32``, ``fp32x2`` (``mixed_bf16`` is
    declared but not built: QMC_ERR_UNSUPPORTED).
    """

    def __init__(self, mol, precision: str = "fp64", device: int = 0):
        lib = library()
        self.mol = mol
        self.precision = precision
        self.device = device
        self.n_elec = mol.n_up + mol.n_down
        # keep the marshalled arrays alive for the duration of the call
        self._arrays = a = dict(
            xyz=np.ascontiguousarray(mol.atom_xyz, dtype=np.float64).reshape(-1),
            z=np.ascontiguousarray(mol.atom_z, dtype=np.float64),
            ao_atom=np.ascontiguousarray(mol.ao_atom, dtype=np.int32),
            ao_kind=np.ascontiguousarray(mol.ao_kind, dtype=np.int32),
            ao_pow=np.ascontiguousarray(mol.ao_pow, dtype=np.int32).reshape(-1),
            ao_prim_start=np.ascontiguousarray(mol.ao_prim_start, dtype=np.int32),
            prim_exp=np.ascontiguousarray(mol.prim_exp, dtype=np.float64),
            prim_coef=np.ascontiguousarray(mol.prim_coef, dtype=np.float64),
            mo=np.ascontiguousarray(mol.mo_coeff, dtype=np.float64).reshape(-1),
            det_w=np.ascontiguousarray(mol.det_weight, dtype=np.float64),
            det_exc=np.ascontiguousarray(mol.det_exc, dtype=np.int32).reshape(-1),
        )
        atoms = _lib.Atoms(mol.n_atom, _ptr(a["xyz"], ctypes.c_double), _ptr(a["z"], ctypes.c_double),
                           mol.n_up, mol.n_down)
        basis = _lib.Basis(mol.n_ao, _ptr(a["ao_atom"], ctypes.c_int32), _ptr(a["ao_kind"], ctypes.c_int32),
                           _ptr(a["ao_pow"], ctypes.c_int32), _ptr(a["ao_prim_start"], ctypes.c_int32),
                           _ptr(a["prim_exp"], ctypes.c_double), _ptr(a["prim_coef"], ctypes.c_double))
        mos = _lib.Mos(mol.n_mo, _ptr(a["mo"], ctypes.c_double))
        dets = _lib.Dets(mol.n_det, _ptr(a["det_w"], ctypes.c_double), _ptr(a["det_exc"], ctypes.c_int32))
        jas = _lib.Jastrow(mol.jastrow_w0_par, mol.jastrow_w0_anti, mol.jastrow_b, mol.backflow_w)
        opt = _lib.Options(PRECISIONS[precision], device)
        handle = ctypes.c_void_p()
        _lib.check(lib.qmc_create_wf(ctypes.byref(atoms), ctypes.byref(basis), ctypes.byref(mos),
                                     ctypes.byref(dets), ctypes.byref(jas), ctypes.byref(opt),
                                     ctypes.byref(handle)))
        self._h = handle
        self._lib = lib
        jen, jeen = getattr(mol, "jastrow_en", None), getattr(mol, "jastrow_een", None)
        if jen is not None or jeen is not None:
            self.set_manybody_jastrow(jen, jeen)

    def set_manybody_jastrow(self, en=None, een=None):
        """Electron-nucleus kernel (w0, w1, w2) and electron-electron-nucleus
        terms [n, 7] = (c, a1, b1, a2, b2, a3, b3) of App. D; None = off."""
        e = None if en is None else np.ascontiguousarray(en, dtype=np.float64).reshape(3)
        t = None if een is None else np.ascontiguousarray(een, dtype=np.float64).reshape(-1, 7)
        _lib.check(self._lib.qmc_set_manybody_jastrow(
            self._h, None if e is None else _ptr(e, ctypes.c_double), 0 if t is None else t.shape[0],
            None if t is None else _ptr(t, ctypes.c_double)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.qmc_destroy_wf(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------
    def set_geometry(self, xyz):
        a = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1)
        _lib.check(self._lib.qmc_set_geometry(self._h, _ptr(a, ctypes.c_double)))

    def workspace_size(self, n_walkers: int) -> int:
        return int(self._lib.qmc_workspace_size(self._h, int(n_walkers)))

    def param_layout(self):
        n = ctypes.c_int64()
        off = (ctypes.c_int64 * 6)()
        _lib.check(self._lib.qmc_param_layout(self._h, ctypes.byref(n), off))
        return int(n.value), [int(v) for v in off]

    def set_params(self, params):
        """Replace the variational parameters (flat, param_layout order)."""
        a = np.ascontiguousarray(params, dtype=np.float64).reshape(-1)
        n, _ = self.param_layout()
        assert a.shape[0] == n, (a.shape, n)
        _lib.check(self._lib.qmc_set_params(self._h, _ptr(a, ctypes.c_double)))

    def energy_grad(self, walkers, n_walkers: int | None = None, want_grad: bool = True, want_forces: bool = True,
                    stream=None):
        """(E mean, E variance, gradient [n_param] (Eq. nabla_loss), forces [n_atom, 3] (Eq. force)) for
        CUDA float64 walkers [3N, ldw]; gradient and forces are CUDA tensors (or None)."""
        import torch

        assert walkers.is_cuda and walkers.dtype == torch.float64 and walkers.stride(1) == 1
        W = walkers.shape[1] if n_walkers is None else int(n_walkers)
        n, _ = self.param_layout()
        grad = torch.empty(n, dtype=torch.float64, device=walkers.device) if want_grad else None
        forces = torch.empty(self.mol.n_atom, 3, dtype=torch.float64, device=walkers.device) if want_forces else None
        stats = np.zeros(2, dtype=np.float64)
        _lib.check(self._lib.qmc_energy_grad(self._h, _dptr(walkers), W, walkers.stride(0),
                                             stats.ctypes.data_as(ctypes.c_void_p), _dptr(grad), _dptr(forces),
                                             _stream_handle(stream)))
        return float(stats[0]), float(stats[1]), grad, forces

    def energy_grad_sums(self, walkers, n_walkers: int | None = None, sums=None, stream=None):
        """Per-batch sums of the energy-gradient estimators (device float64
        [qmc_energy_grad_sums_size]), stream-ordered: all-reduce them across
        shards, then assemble with _lib.assemble_energy_grad."""
        import torch

        W = walkers.shape[1] if n_walkers is None else int(n_walkers)
        n = int(self._lib.qmc_energy_grad_sums_size(self._h))
        if sums is None:
            sums = torch.empty(n, dtype=torch.float64, device=walkers.device)
        _lib.check(self._lib.qmc_energy_grad_sums(self._h, _dptr(walkers), W, walkers.stride(0), _dptr(sums),
                                                  _stream_handle(stream)))
        return sums

    def optimize(self, walkers, n_iter: int, n_equil: int, n_resample: int, step: float, seed: int,
                 lr: float = 1e-2, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, mask=None,
                 n_walkers: int | None = None, stream=None):
        """The optimisation loop of App. B (qmc_optimize): equilibrate, then per step
        the Eq. nabla_loss gradient, one ADAM update and n_resample Metropolis steps.
        walkers (CUDA float64 [3N, ldw]) are updated in place; returns the history
        [n_iter, 3] (E mean, E variance, acceptance) as a numpy array."""
        import torch

        assert walkers.is_cuda and walkers.dtype == torch.float64 and walkers.stride(1) == 1
        W = walkers.shape[1] if n_walkers is None else int(n_walkers)
        hist = np.zeros((max(n_iter, 1), 3), dtype=np.float64)
        m = None
        if mask is not None:
            m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8))
            assert m.shape == (self.param_layout()[0],)
        cfg = _lib.OptConfig(n_iter, n_equil, n_resample, 0, step, seed, lr, beta1, beta2, eps,
                             None if m is None else m.ctypes.data)
        _lib.check(self._lib.qmc_optimize(self._h, _dptr(walkers), W, walkers.stride(0), ctypes.byref(cfg),
                                          hist.ctypes.data_as(ctypes.c_void_p), _stream_handle(stream)))
        return hist[:n_iter]

    def force_batches(self, walkers, n_batches: int, symmetrize: bool = True, n_walkers: int | None = None,
                      stream=None):
        """Per-batch (E mean [n_batches], forces [n_batches, n_atom, 3]) of Eq. force, each batch
        optionally symmetrised about the z axis (qmc_force_batches)."""
        import torch

        assert walkers.is_cuda and walkers.dtype == torch.float64 and walkers.stride(1) == 1
        W = walkers.shape[1] if n_walkers is None else int(n_walkers)
        e = np.zeros(n_batches, dtype=np.float64)
        f = np.zeros((n_batches, self.mol.n_atom, 3), dtype=np.float64)
        _lib.check(self._lib.qmc_force_batches(self._h, _dptr(walkers), W, walkers.stride(0), n_batches,
                                               1 if symmetrize else 0, e.ctypes.data_as(ctypes.c_void_p),
                                               f.ctypes.data_as(ctypes.c_void_p), _stream_handle(stream)))
        return e, f

    def set_det_method(self, method: str):
        """'table' (default, Eq. table) or 'explicit' (LU of every distinct
        excited matrix; the baseline of the paper's comparison)."""
        code = {"table": 0, "explicit": 1}[method]
        _lib.check(self._lib.qmc_set_det_method(self._h, code))

    def check_status(self, stream=None):
        """Raise QmcError(QMC_ERR_TIMEOUT) if a bounded device wait gave up
        since the last check (waits for the stream first)."""
        _lib.check(self._lib.qmc_check_status(self._h, _stream_handle(stream)))

    def set_wait_limit(self, cycles: int):
        """Testing aid: budget of each bounded device wait in SM cycles (0 = give up at once)."""
        _lib.check(self._lib.qmc_set_wait_limit(self._h, int(cycles)))

    def set_timing(self, enable: bool = True):
        """Record per-stage CUDA events on the call's stream (tracing aid)."""
        _lib.check(self._lib.qmc_set_timing(self._h, 1 if enable else 0))

    def last_stage_ms(self):
        """[Jastrow+Coulomb, AO+MO, det+assembly] ms of the last timed call."""
        ms = (ctypes.c_float * 3)()
        _lib.check(self._lib.qmc_last_stage_ms(self._h, ms, 3))
        return [float(v) for v in ms]

    # ------------------------------------------------------------------
    def local_energy(self, walkers, n_walkers: int | None = None, e_loc=None, log_psi=None, workspace=None,
                     stream=None, want_log_psi: bool = True):
        """E_L (and log|Psi|) for walkers given as a CUDA float64 tensor [3N, ldw]."""
        import torch

        assert walkers.is_cuda and walkers.dtype == torch.float64 and walkers.dim() == 2
        assert walkers.stride(1) == 1 and walkers.shape[0] == 3 * self.n_elec
        W = walkers.shape[1] if n_walkers is None else int(n_walkers)
        ldw = walkers.stride(0)
        if e_loc is None:
            e_loc = torch.empty(W, dtype=torch.float64, device=walkers.device)
        if log_psi is None and want_log_psi:
            log_psi = torch.empty(W, dtype=torch.float64, device=walkers.device)
        ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
        _lib.check(self._lib.qmc_local_energy(self._h, _dptr(walkers), W, ldw, _dptr(e_loc), _dptr(log_psi),
                                              _dptr(workspace), ws_bytes, _stream_handle(stream)))
        return e_loc, log_psi

    def local_energy_noalloc(self, walkers, n_walkers: int | None = None, e_loc=None, log_psi=None, stream=None,
                             want_log_psi: bool = True):
        """As local_energy, for callers that must not allocate device memory
        during a call: the scratch is the library's static device array (see
        qmc_local_energy_noalloc in include/qmc.h for the batch limit and the
        rule that overlapping calls race on that array)."""
        import torch

        assert walkers.is_cuda and walkers.dtype == torch.float64 and walkers.dim() == 2
        assert walkers.stride(1) == 1 and walkers.shape[0] == 3 * self.n_elec
        W = walkers.shape[1] if n_walkers is None else int(n_walkers)
        if e_loc is None:
            e_loc = torch.empty(W, dtype=torch.float64, device=walkers.device)
        if log_psi is None and want_log_psi:
            log_psi = torch.empty(W, dtype=torch.float64, device=walkers.device)
        _lib.check(self._lib.qmc_local_energy_noalloc(self._h, _dptr(walkers), W, walkers.stride(0), _dptr(e_loc),
                                                      _dptr(log_psi), _stream_handle(stream)))
        return e_loc, log_psi

    def local_energy_host(self, walkers: np.ndarray, e_loc: np.ndarray | None = None,
                          log_psi: np.ndarray | None = None, stream=None):
        """E_L from HOST buffers: walkers float64 [3N, W] C-contiguous (pinned
        memory is fastest); results are on the host when this returns."""
        W = walkers.shape[1]
        assert walkers.dtype == np.float64 and walkers.flags.c_contiguous and walkers.shape[0] == 3 * self.n_elec
        if e_loc is None:
            e_loc = np.empty(W, dtype=np.float64)
        _lib.check(self._lib.qmc_local_energy_host(
            self._h, walkers.ctypes.data_as(ctypes.c_void_p), W, e_loc.ctypes.data_as(ctypes.c_void_p),
            None if log_psi is None else log_psi.ctypes.data_as(ctypes.c_void_p),
            ctypes.c_void_p(0) if stream is None else _stream_handle(stream)))
        return e_loc, log_psi

    def sample(self, walkers, n_steps: int, step: float, seed: int, first_walker: int = 0, step_offset: int = 0,
               n_walkers: int | None = None, log_psi=None, n_accept=None, workspace=None, stream=None):
        """Metropolis steps, updating the CUDA float64 walkers [3N, ldw] in place."""
        import torch

        assert walkers.is_cuda and walkers.dtype == torch.float64 and walkers.stride(1) == 1
        W = walkers.shape[1] if n_walkers is None else int(n_walkers)
        ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
        _lib.check(self._lib.qmc_sample(self._h, _dptr(walkers), W, walkers.stride(0), int(n_steps), float(step),
                                        int(seed), int(first_walker), int(step_offset), _dptr(log_psi),
                                        _dptr(n_accept), _dptr(workspace), ws_bytes, _stream_handle(stream)))
        return walkers


def _torch_energy_function():
    import torch

    class VariationalEnergy(torch.autograd.Function):
        """E_v = <E_L> over the given walkers as a differentiable function of
        the variational parameters and the nuclear coordinates.  Forward sets
        them on the device wavefunction and runs qmc_energy_grad; backward
        returns the low-variance gradient estimator (Eq. nabla_loss) for the
        parameters and minus the force estimator (Eq. force) for the nuclei
        (the walkers are held fixed, as in the paper's estimators)."""

        @staticmethod
        def forward(ctx, params, atom_xyz, wf, walkers):
            wf.set_params(params.detach().cpu().numpy())
            wf.set_geometry(atom_xyz.detach().cpu().numpy())
            e_mean, e_var, grad, forces = wf.energy_grad(walkers)
            ctx.save_for_backward(grad.to(params.device), forces.to(atom_xyz.device))
            ctx.e_var = e_var
            return params.new_tensor(e_mean)

        @staticmethod
        def backward(ctx, g):
            grad, forces = ctx.saved_tensors
            return g * grad, -g * forces, None, None

    return VariationalEnergy


def variational_energy(params, atom_xyz, wf: Wavefunction, walkers):
    """Differentiable <E_L> (torch.autograd.Function over qmc_energy_grad)."""
    return _torch_energy_function().apply(params, atom_xyz, wf, walkers)
