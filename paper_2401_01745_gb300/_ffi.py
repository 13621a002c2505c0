"""ctypes declarations of the C ABI in include/emrkc.h (argument marshalling only)."""

from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libemrkc.so")

EMRKC_OK = 0
ERRORS = {1: "EMRKC_ERR_ARG", 2: "EMRKC_ERR_CUDA", 3: "EMRKC_ERR_OOM", 4: "EMRKC_ERR_NONFINITE",
          5: "EMRKC_ERR_TIMEOUT", 6: "EMRKC_ERR_STATE"}
NUM_PHASES = 5
PHASES = ("stage", "inner", "power_F", "power_S", "other")


class Matrix(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.POINTER(C.c_int64)),
                ("col", C.POINTER(C.c_int32)), ("K", C.POINTER(C.c_double)),
                ("lumped_mass", C.POINTER(C.c_double))]


class OwnedMatrix(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.POINTER(C.c_int64)),
                ("col", C.POINTER(C.c_int32)), ("K", C.POINTER(C.c_double)),
                ("lumped_mass", C.POINTER(C.c_double))]


class Tissue(C.Structure):
    _fields_ = [("chi", C.c_double), ("Cm", C.c_double)]


class Stimulus(C.Structure):
    _fields_ = [("node_mask", C.POINTER(C.c_uint8)), ("amplitude", C.c_double),
                ("t_on", C.c_double), ("t_off", C.c_double)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("rho_every", C.c_int), ("rho_F", C.c_double),
                ("rho_S", C.c_double), ("eps", C.c_double), ("safety", C.c_double),
                ("pow_tol", C.c_double), ("pow_eps", C.c_double), ("pow_max_iter", C.c_int),
                ("seed", C.c_uint64), ("act_threshold", C.c_double), ("cuda_stream", C.c_void_p),
                ("device", C.c_int), ("profile", C.c_int), ("use_graphs", C.c_int),
                ("rho_S_min", C.c_double), ("method", C.c_int), ("lin_rtol", C.c_double),
                ("lin_max_iter", C.c_int), ("pow_tol_cold", C.c_double), ("pow_max_iter_cold", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("t", C.c_double), ("steps", C.c_int64), ("s", C.c_int), ("m", C.c_int),
                ("eta", C.c_double), ("rho_F", C.c_double), ("rho_S", C.c_double),
                ("pow_iters_F", C.c_int), ("pow_iters_S", C.c_int), ("total_pow_iters", C.c_int64),
                ("launches", C.c_int64), ("matrix_entries", C.c_int64), ("matrix_slots", C.c_int64),
                ("phase_ms", C.c_double * NUM_PHASES),
                ("phase_launches", C.c_int64 * NUM_PHASES), ("lin_iters", C.c_int),
                ("total_lin_iters", C.c_int64), ("lin_residual", C.c_double)]


class BatchInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("N", C.c_int), ("model", C.c_int), ("s", C.c_int), ("m", C.c_int),
                ("t", C.c_double), ("steps", C.c_int64), ("device_bytes", C.c_int64)]


class BatchStats(C.Structure):
    _fields_ = [("instances", C.c_int), ("total_nodes", C.c_int64), ("items", C.c_int64),
                ("tile", C.c_int), ("block", C.c_int), ("grid", C.c_int), ("launches", C.c_int64),
                ("device_bytes", C.c_int64), ("schedule", C.c_int), ("threads_per_sm", C.c_int)]


_P = C.c_void_p
_PD = C.POINTER(C.c_double)

SIGNATURES = {
    "emrkc_default_options": (C.c_int, [C.POINTER(Options)]),
    "emrkc_num_vars": (C.c_int, [C.c_int]),
    "emrkc_num_gates": (C.c_int, [C.c_int]),
    "emrkc_rkc_stages": (C.c_int, [C.c_double, C.c_double, C.c_double, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "emrkc_rkc_coeffs": (C.c_int, [C.c_int, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                   C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "emrkc_assemble_p1": (C.c_int, [C.c_int, C.c_int64, _PD, C.c_int64, C.POINTER(C.c_int64), _PD,
                                    C.POINTER(OwnedMatrix)]),
    "emrkc_free_matrix": (None, [C.POINTER(OwnedMatrix)]),
    "emrkc_set_stimulus": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint8), C.c_int64, C.c_double, C.c_double,
                                     C.c_double]),
    "emrkc_set_stimulus_async": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint8), C.c_int64, C.c_double, C.c_double,
                                           C.c_double]),
    "emrkc_get_state_async": (C.c_int, [_P, C.c_int, _PD, C.c_int64]),
    "emrkc_create": (C.c_int, [C.POINTER(Matrix), C.POINTER(Tissue), C.c_int, C.POINTER(Stimulus),
                               C.POINTER(Options), C.POINTER(_P)]),
    "emrkc_step": (C.c_int, [_P, C.c_double]),
    "emrkc_run": (C.c_int, [_P, C.c_double, C.c_double]),
    "emrkc_sync": (C.c_int, [_P]),
    "emrkc_get_state": (C.c_int, [_P, C.c_int, _PD, C.c_int64]),
    "emrkc_set_state": (C.c_int, [_P, C.c_int, _PD, C.c_int64]),
    "emrkc_get_state_device": (C.c_int, [_P, C.c_int, C.c_void_p, C.c_int64]),
    "emrkc_set_state_device": (C.c_int, [_P, C.c_int, C.c_void_p, C.c_int64]),
    "emrkc_get_activation_times": (C.c_int, [_P, _PD, C.c_int64]),
    "emrkc_estimate_rho": (C.c_int, [_P, _PD, _PD, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "emrkc_set_time": (C.c_int, [_P, C.c_double, C.c_int64]),
    "emrkc_estimate_rho_F_noalloc": (C.c_int, [_P, C.c_void_p, C.c_void_p, C.c_int64, C.c_double, _PD,
                                               C.POINTER(C.c_int)]),
    "emrkc_get_stats": (C.c_int, [_P, C.POINTER(Stats)]),
    "emrkc_last_error": (C.c_char_p, [_P]),
    "emrkc_destroy": (None, [_P]),
    "emrkc_batch_create": (C.c_int, [C.POINTER(Options), C.POINTER(_P)]),
    "emrkc_batch_add": (C.c_int, [_P, C.POINTER(Matrix), C.POINTER(Tissue), C.c_int, C.POINTER(Stimulus),
                                  C.POINTER(Options), C.POINTER(C.c_int)]),
    "emrkc_batch_remove": (C.c_int, [_P, C.c_int]),
    "emrkc_batch_step": (C.c_int, [_P, C.c_double]),
    "emrkc_batch_sync": (C.c_int, [_P]),
    "emrkc_batch_get_state": (C.c_int, [_P, C.c_int, C.c_int, _PD, C.c_int64]),
    "emrkc_batch_set_state": (C.c_int, [_P, C.c_int, C.c_int, _PD, C.c_int64]),
    "emrkc_batch_get_activation_times": (C.c_int, [_P, C.c_int, _PD, C.c_int64]),
    "emrkc_batch_get_info": (C.c_int, [_P, C.c_int, C.POINTER(BatchInfo)]),
    "emrkc_batch_get_stats": (C.c_int, [_P, C.POINTER(BatchStats)]),
    "emrkc_batch_set_config": (C.c_int, [_P, C.c_int, C.c_int]),
    "emrkc_batch_set_spin_limit": (C.c_int, [_P, C.c_int64]),
    "emrkc_batch_set_schedule": (C.c_int, [_P, C.c_int]),
    "emrkc_batch_set_occupancy": (C.c_int, [_P, C.c_int]),
    "emrkc_batch_autotune": (C.c_int, [_P, C.c_double, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                       C.POINTER(C.c_double)]),
    "emrkc_batch_set_stimulus_async": (C.c_int, [_P, C.POINTER(C.c_uint8), C.c_int64]),
    "emrkc_batch_get_V_async": (C.c_int, [_P, _PD, C.c_int64]),
    "emrkc_batch_get_V32_async": (C.c_int, [_P, C.POINTER(C.c_float), C.c_int64]),
    "emrkc_batch_ids": (C.c_int, [_P, C.POINTER(C.c_int), C.c_int]),
    "emrkc_batch_set_profile": (C.c_int, [_P, C.c_int]),
    "emrkc_batch_get_kernel_time": (C.c_int, [_P, _PD, C.POINTER(C.c_int64)]),
    "emrkc_instance_bytes": (C.c_int64, [C.c_int64, C.c_double, C.c_int]),
    "emrkc_batch_last_error": (C.c_char_p, [_P]),
    "emrkc_batch_destroy": (None, [_P]),
}

_lib = None


def load(path: str | None = None):
    """Load the shared library; raises if it has not been built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"the emRKC CUDA library is not built ({p}); run paper_2401_01745_gb300.build()")
    lib = C.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        if not hasattr(lib, name):
            continue
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = lib
    return lib
