"""ctypes declarations of the C ABI in ``include/qmc.h``.

Loading fails loudly (``RuntimeError``) if the shared library is missing:
there is no CPU fallback anywhere in the package.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int32, c_int64, c_size_t, c_uint64, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqmc_gb300.so")

QMC_OK, QMC_ERR_ARG, QMC_ERR_OOM, QMC_ERR_CUDA, QMC_ERR_TIMEOUT, QMC_ERR_UNSUPPORTED, QMC_ERR_CANCELLED = range(7)
STATUS_NAMES = {0: "QMC_OK", 1: "QMC_ERR_ARG", 2: "QMC_ERR_OOM", 3: "QMC_ERR_CUDA", 4: "QMC_ERR_TIMEOUT",
                5: "QMC_ERR_UNSUPPORTED", 6: "QMC_ERR_CANCELLED"}
QMC_FP64, QMC_FP32, QMC_MIXED_TF32, QMC_MIXED_BF16, QMC_FP32X2 = range(5)
NOALLOC_SCRATCH_BYTES = 64 << 20  # QMC_NOALLOC_SCRATCH_BYTES of include/qmc.h
PRECISIONS = {"fp64": QMC_FP64, "fp32": QMC_FP32, "mixed_tf32": QMC_MIXED_TF32, "mixed_bf16": QMC_MIXED_BF16,
              "fp32x2": QMC_FP32X2}

# every exported symbol declared in include/qmc.h
EXPORTED = (
    "qmc_create_wf", "qmc_destroy_wf", "qmc_set_geometry", "qmc_workspace_size", "qmc_local_energy",
    "qmc_local_energy_host", "qmc_local_energy_noalloc", "qmc_sample", "qmc_param_layout", "qmc_energy_grad",
    "qmc_set_params", "qmc_server_create", "qmc_server_destroy", "qmc_server_add_wf", "qmc_server_submit",
    "qmc_server_progress", "qmc_server_results", "qmc_server_cancel", "qmc_server_set_policy", "qmc_server_free_bytes", "qmc_server_clock",
    "qmc_server_last_error", "qmc_set_timing", "qmc_last_stage_ms", "qmc_set_det_method", "qmc_optimize", "qmc_force_batches", "qmc_set_manybody_jastrow",
    "qmc_check_status", "qmc_set_wait_limit", "qmc_energy_grad_sums_size", "qmc_energy_grad_sums",
    "qmc_assemble_energy_grad", "qmc_measure_rates", "qmc_last_error",
)

PD = POINTER(c_double)
PI32 = POINTER(c_int32)


class Atoms(ctypes.Structure):
    _fields_ = [("n_atom", c_int32), ("xyz", PD), ("z", PD), ("n_up", c_int32), ("n_down", c_int32)]


class Basis(ctypes.Structure):
    _fields_ = [("n_ao", c_int32), ("ao_atom", PI32), ("ao_kind", PI32), ("ao_pow", PI32),
                ("ao_prim_start", PI32), ("prim_exp", PD), ("prim_coef", PD)]


class Mos(ctypes.Structure):
    _fields_ = [("n_mo", c_int32), ("coeff", PD)]


class Dets(ctypes.Structure):
    _fields_ = [("n_det", c_int32), ("weight", PD), ("exc", PI32)]


class Jastrow(ctypes.Structure):
    _fields_ = [("w0_par", c_double), ("w0_anti", c_double), ("b", c_double), ("backflow_w", c_double)]


class Options(ctypes.Structure):
    _fields_ = [("precision", c_int32), ("device", c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("wf_id", c_int32), ("n_walkers", c_int64), ("n_steps", c_int32), ("step", c_double),
                ("seed", c_uint64), ("walkers", c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("ticket", c_int64), ("status", c_int32), ("wf_id", c_int32), ("n_walkers", c_int64),
                ("e_mean", c_double), ("e_var", c_double), ("accept_rate", c_double), ("t_submit", c_double),
                ("t_admit", c_double), ("t_done", c_double), ("n_nonfinite", c_int64)]


class OptConfig(ctypes.Structure):
    _fields_ = [("n_iter", c_int32), ("n_equil", c_int32), ("n_resample", c_int32), ("reserved", c_int32),
                ("step", c_double), ("seed", c_uint64), ("lr", c_double), ("beta1", c_double), ("beta2", c_double),
                ("eps", c_double), ("mask", c_void_p)]


class QmcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load the shared library once; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    lib.qmc_create_wf.argtypes = [POINTER(Atoms), POINTER(Basis), POINTER(Mos), POINTER(Dets), POINTER(Jastrow),
                                  POINTER(Options), POINTER(c_void_p)]
    lib.qmc_create_wf.restype = c_int32
    lib.qmc_destroy_wf.argtypes = [c_void_p]
    lib.qmc_destroy_wf.restype = None
    lib.qmc_set_geometry.argtypes = [c_void_p, PD]
    lib.qmc_set_geometry.restype = c_int32
    lib.qmc_workspace_size.argtypes = [c_void_p, c_int64]
    lib.qmc_workspace_size.restype = c_size_t
    lib.qmc_local_energy.argtypes = [c_void_p, c_void_p, c_int64, c_int64, c_void_p, c_void_p, c_void_p, c_size_t,
                                     c_void_p]
    lib.qmc_local_energy.restype = c_int32
    lib.qmc_local_energy_host.argtypes = [c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p]
    lib.qmc_local_energy_host.restype = c_int32
    lib.qmc_local_energy_noalloc.argtypes = [c_void_p, c_void_p, c_int64, c_int64, c_void_p, c_void_p, c_void_p]
    lib.qmc_local_energy_noalloc.restype = c_int32
    lib.qmc_sample.argtypes = [c_void_p, c_void_p, c_int64, c_int64, c_int32, c_double, c_uint64, c_uint64,
                               c_uint64, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]
    lib.qmc_sample.restype = c_int32
    lib.qmc_param_layout.argtypes = [c_void_p, POINTER(c_int64), POINTER(c_int64)]
    lib.qmc_param_layout.restype = c_int32
    lib.qmc_energy_grad.argtypes = [c_void_p, c_void_p, c_int64, c_int64, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.qmc_energy_grad.restype = c_int32
    lib.qmc_set_params.argtypes = [c_void_p, PD]
    lib.qmc_set_params.restype = c_int32
    lib.qmc_set_timing.argtypes = [c_void_p, c_int32]
    lib.qmc_set_timing.restype = c_int32
    lib.qmc_set_det_method.argtypes = [c_void_p, c_int32]
    lib.qmc_set_det_method.restype = c_int32
    lib.qmc_set_manybody_jastrow.argtypes = [c_void_p, PD, c_int32, PD]
    lib.qmc_set_manybody_jastrow.restype = c_int32
    lib.qmc_optimize.argtypes = [c_void_p, c_void_p, c_int64, c_int64, POINTER(OptConfig), c_void_p, c_void_p]
    lib.qmc_optimize.restype = c_int32
    lib.qmc_force_batches.argtypes = [c_void_p, c_void_p, c_int64, c_int64, c_int32, c_int32, c_void_p, c_void_p,
                                      c_void_p]
    lib.qmc_force_batches.restype = c_int32
    lib.qmc_last_stage_ms.argtypes = [c_void_p, POINTER(ctypes.c_float), c_int32]
    lib.qmc_last_stage_ms.restype = c_int32
    lib.qmc_server_create.argtypes = [c_int32, c_size_t, c_int32, POINTER(c_void_p)]
    lib.qmc_server_create.restype = c_int32
    lib.qmc_server_destroy.argtypes = [c_void_p]
    lib.qmc_server_destroy.restype = None
    lib.qmc_server_add_wf.argtypes = [c_void_p, c_void_p, POINTER(c_int32)]
    lib.qmc_server_add_wf.restype = c_int32
    lib.qmc_server_submit.argtypes = [c_void_p, POINTER(Request), POINTER(c_int64)]
    lib.qmc_server_submit.restype = c_int32
    lib.qmc_server_progress.argtypes = [c_void_p, POINTER(c_int32), POINTER(c_int32)]
    lib.qmc_server_progress.restype = c_int32
    lib.qmc_server_results.argtypes = [c_void_p, POINTER(Result), c_int32, POINTER(c_int32)]
    lib.qmc_server_results.restype = c_int32
    lib.qmc_server_cancel.argtypes = [c_void_p, c_int64]
    lib.qmc_server_cancel.restype = c_int32
    lib.qmc_server_set_policy.argtypes = [c_void_p, c_int64, c_int32]
    lib.qmc_server_set_policy.restype = c_int32
    lib.qmc_server_free_bytes.argtypes = [c_void_p]
    lib.qmc_server_free_bytes.restype = c_size_t
    lib.qmc_server_clock.argtypes = []
    lib.qmc_server_clock.restype = c_double
    lib.qmc_server_last_error.argtypes = []
    lib.qmc_server_last_error.restype = c_char_p
    lib.qmc_check_status.argtypes = [c_void_p, c_void_p]
    lib.qmc_check_status.restype = c_int32
    lib.qmc_set_wait_limit.argtypes = [c_void_p, c_int64]
    lib.qmc_set_wait_limit.restype = c_int32
    lib.qmc_energy_grad_sums_size.argtypes = [c_void_p]
    lib.qmc_energy_grad_sums_size.restype = c_int64
    lib.qmc_energy_grad_sums.argtypes = [c_void_p, c_void_p, c_int64, c_int64, c_void_p, c_void_p]
    lib.qmc_energy_grad_sums.restype = c_int32
    lib.qmc_assemble_energy_grad.argtypes = [c_int64, c_int32, PD, PD, PD, PD]
    lib.qmc_assemble_energy_grad.restype = c_int32
    lib.qmc_measure_rates.argtypes = [PD, c_void_p]
    lib.qmc_measure_rates.restype = c_int32
    lib.qmc_last_error.argtypes = []
    lib.qmc_last_error.restype = c_char_p
    _lib = lib
    return lib


def check(status: int):
    if status != QMC_OK:
        msg = _lib.qmc_last_error().decode() if _lib is not None else ""
        raise QmcError(status, msg)


def check_server(status: int):
    if status != QMC_OK:
        msg = _lib.qmc_server_last_error().decode() if _lib is not None else ""
        raise QmcError(status, msg)


def assemble_energy_grad(sums, n_param: int, n_atom: int):
    """qmc_assemble_energy_grad on host sums (e.g. after an all-reduce over
    the shards): returns (E_v, variance, grad [n_param], forces [n_atom, 3])."""
    import numpy as np

    lib = load()
    s = np.ascontiguousarray(sums, dtype=np.float64)
    e = np.empty(2)
    g = np.empty(max(n_param, 1))
    f = np.empty((n_atom, 3))
    check(lib.qmc_assemble_energy_grad(int(n_param), int(n_atom), s.ctypes.data_as(PD), e.ctypes.data_as(PD),
                                       g.ctypes.data_as(PD), f.ctypes.data_as(PD)))
    return float(e[0]), float(e[1]), g[:n_param], f


def measure_rates(stream=None) -> dict:
    """qmc_measure_rates: the GPU's FP64 FMA, FP32 FMA and FP64 exp / sqrt /
    reciprocal rates per second, measured by the library's probe kernels."""
    import numpy as np

    lib = load()
    out = np.zeros(5, dtype=np.float64)
    h = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    check(lib.qmc_measure_rates(out.ctypes.data_as(PD), h))
    keys = ("fp64_fma_per_s", "fp32_fma_per_s", "fp64_exp_per_s", "fp64_sqrt_per_s", "fp64_recip_per_s")
    return {k: float(v) for k, v in zip(keys, out)}
