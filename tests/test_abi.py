"""The C ABI library builds for sm_103a, loads without a GPU and exports every
function the public header declares.  No compute call is made here."""
import ctypes
import os
import shutil

import pytest

from paper_1408_6527_gb300 import _lib


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_lib.LIB_PATH):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available to build the library")
        import paper_1408_6527_gb300

        paper_1408_6527_gb300.build()
    return ctypes.CDLL(_lib.LIB_PATH)


def test_header_declares_the_three_calls():
    names = _lib.header_functions()
    for f in ("fmm_build", "fmm_solve_induced_dipoles", "fmm_energy_forces", "fmm_destroy"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    names = _lib.header_functions()
    assert len(names) >= 18
    for name in names:
        assert hasattr(lib, name), name


def test_binding_signatures_cover_the_header():
    assert set(_lib.header_functions()) <= set(_lib.SIGNATURES)


def test_status_strings_without_gpu(lib):
    lib.fmm_status_string.restype = ctypes.c_char_p
    assert lib.fmm_status_string(0) == b"ok"
    assert lib.fmm_status_string(3) == b"dipole solve not converged"


def test_default_options_without_gpu(lib):
    o = _lib.Options()
    lib.fmm_default_options(ctypes.byref(o))
    assert o.mode == _lib.FP64 and o.max_iter == 100 and o.coulomb_k == 1.0 and o.solver == _lib.SOLVER_PCG


def test_invalid_arguments_rejected_before_any_device_work(lib):
    lib.fmm_build.argtypes = _lib.SIGNATURES["fmm_build"][1]
    h = ctypes.c_void_p()
    import numpy as np

    x = np.zeros(6)
    q = np.zeros(2)
    a = np.ones(2)
    ptr = lambda v: v.ctypes.data_as(ctypes.c_void_p)
    # order out of range, depth out of range, n < 1, negative polarizability, NaN
    assert lib.fmm_build(ctypes.byref(h), 2, ptr(x), ptr(q), ptr(a), 11, 3, None, 0) == 1
    assert lib.fmm_build(ctypes.byref(h), 2, ptr(x), ptr(q), ptr(a), 4, 9, None, 0) == 1
    assert lib.fmm_build(ctypes.byref(h), 0, ptr(x), ptr(q), ptr(a), 4, 3, None, 0) == 1
    a2 = np.array([1.0, -0.5])
    assert lib.fmm_build(ctypes.byref(h), 2, ptr(x), ptr(q), ptr(a2), 4, 3, None, 0) == 1
    x2 = x.copy()
    x2[4] = float("nan")
    assert lib.fmm_build(ctypes.byref(h), 2, ptr(x2), ptr(q), ptr(a), 4, 3, None, 0) == 1
    assert not h.value
