"""ctypes declarations of the C ABI in include/polfmm.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpolfmm.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "polfmm.h")

OK = 0
ERR_INVALID_ARG = 1
ERR_COINCIDENT = 2
ERR_NOT_CONVERGED = 3
ERR_OUT_OF_MEMORY = 4
ERR_CUDA = 5
ERR_STATE = 6

FP64 = 0
MIXED = 1
SOLVER_PCG = 0
SOLVER_JACOBI = 1
M2L_AUTO = 0
M2L_SIMT = 1
M2L_TENSOR = 2
M2L_FFMA = 3
NOALLOC_MAX_SITES = 262144


class Options(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_int),
        ("solver", ctypes.c_int),
        ("max_iter", ctypes.c_int),
        ("coulomb_k", ctypes.c_double),
        ("use_root_box", ctypes.c_int),
        ("root_lo", ctypes.c_double * 3),
        ("root_side", ctypes.c_double),
        ("m2l_impl", ctypes.c_int),
        ("profile", ctypes.c_int),
        ("cuda_stream", ctypes.c_void_p),
        ("no_graphs", ctypes.c_int),
        ("dipole_dl", ctypes.c_double),
        ("no_pdl", ctypes.c_int),
        ("dipole_tree", ctypes.c_int),
    ]


_lock = threading.Lock()
_lib = None

P = ctypes.c_void_p
I = ctypes.c_int
I64 = ctypes.c_int64
D = ctypes.c_double

SIGNATURES = {
    "fmm_default_options": (None, [ctypes.POINTER(Options)]),
    "fmm_build": (I, [ctypes.POINTER(P), I64, P, P, P, I, I, ctypes.POINTER(Options), I]),
    "fmm_solve_induced_dipoles": (I, [P, D, ctypes.POINTER(I), ctypes.POINTER(D)]),
    "fmm_energy_forces": (I, [P, P, P, P, P, I]),
    "fmm_energy": (I, [P, P]),
    "fmm_get_dipoles": (I, [P, P, I]),
    "fmm_set_dipoles": (I, [P, P, I]),
    "fmm_update_positions": (I, [P, P, I]),
    "fmm_set_field_charges": (I, [P, P, I]),
    "fmm_set_exclusions": (I, [P, I64, P, I]),
    "fmm_field_charge_gradient": (I, [P, P, I]),
    "fmm_set_thole": (I, [P, D]),
    "fmm_set_dipole_predictor": (I, [P, I]),
    "fmm_reset_dipoles": (I, [P]),
    "fmm_static_field": (I, [P, P, P, I]),
    "fmm_dipole_field": (I, [P, P, P, I]),
    "fmm_total_field": (I, [P, P, P, P, P, I]),
    "fmm_leaf_cells": (I, [P, P, I]),
    "fmm_tree_info": (I, [P, P]),
    "fmm_root_box": (I, [P, P, P]),
    "fmm_profile_get": (I, [P, ctypes.c_char_p, ctypes.POINTER(D), ctypes.POINTER(I64)]),
    "fmm_profile_reset": (I, [P]),
    "fmm_launch_count": (I64, [P]),
    "fmm_testing_alloc_hook": (I64, [I64]),
    "fmm_testing_m2l_plan": (I, [I, I, I, P, P, P, P, P]),
    "fmm_measure_peak": (I, [I, P, ctypes.POINTER(D)]),
    "fmm_kdtree_fields": (I, [I64, P, P, P, I, D, I, I, D, D, P, P, P, P, P, I]),
    "fmm_wall_create": (I, [ctypes.POINTER(P), I64, P]),
    "fmm_wall_forces": (I, [P, P, I64, D, D, P, P]),
    "fmm_md_kinetic": (I, [P, P, P, I64, D, P]),
    "fmm_md_momentum": (I, [P, P, P, I64, P]),
    "fmm_md_kick": (I, [P, P, P, D, I64, P]),
    "fmm_md_drift": (I, [P, P, D, I64, P]),
    "fmm_wall_destroy": (None, [P]),
    "fmm_destroy": (None, [P]),
    "fmm_sort_sites_noalloc": (I, [I64, P, I, P, P, P, P, P, P]),
    "fmm_status_string": (ctypes.c_char_p, [I]),
    "fmm_last_error": (ctypes.c_char_p, []),
}


def header_functions() -> list[str]:
    """Names of every function the public header declares."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"POLFMM_API\s+[\w\s\*]*?\b(fmm_\w+)\s*\(", txt)))


def load(path: str | None = None):
    """Load libpolfmm.so.  Raises if the CUDA library has not been built: there
    is no fallback implementation."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(
                f"CUDA library {p} is missing; build it with paper_1408_6527_gb300.build() "
                "(nvcc, sm_103a). There is no CPU fallback.")
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = lib
        return lib


class PolFMMError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        try:
            msg = load().fmm_status_string(status).decode()
            if status == ERR_CUDA:
                msg += ": " + load().fmm_last_error().decode()
        except Exception:  # pragma: no cover
            msg = f"status {status}"
        super().__init__(f"{where}: {msg} ({status})")


def check(status: int, where: str, allow=()):
    if status != OK and status not in allow:
        raise PolFMMError(status, where)
    return status
