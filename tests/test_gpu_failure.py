"""Failure handling of the solver and of the allocator, made on the host (no
GPU fault is provoked): an indefinite dipole operator, a diverging fixed-point
iteration and a planted out-of-memory at every allocation of a build.

Point dipoles without damping pass the polarization catastrophe when
alpha^1/2 T alpha^1/2 has an eigenvalue above 1 (Sec. II.A: the dipole
equations then have no positive-definite solution); the 400-site random
cluster with polarizabilities up to 2 A^3 is such a case (smallest eigenvalue
of diag(1/alpha) - T about -0.04, checked in the oracle pins)."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1408_6527_gb300 import PolFMM, PolFMMError, _lib  # noqa: E402


def _catastrophe():
    return synth.small_random(2024, 400, box=16.0, alpha_range=(0.3, 2.0))


def test_indefinite_operator_stops_with_the_last_good_dipoles():
    pos, q, alpha = _catastrophe()
    lo, side = oracle.root_box(pos)
    ev = np.linalg.eigvalsh(oracle.dipole_matrix(pos) * -1.0 + np.diag(np.repeat(1.0 / alpha, 3)))
    assert ev[0] < 0.0  # the operator is indefinite
    with PolFMM(pos, q, alpha, p=6, depth=3, mode="fp64", max_iter=200) as f:
        info = f.solve(1e-12)
        mu_stop = f.dipoles()
    assert info["status"] == _lib.ERR_NOT_CONVERGED and info["iterations"] < 200
    assert np.all(np.isfinite(mu_stop)) and np.isfinite(info["residual"])
    # the direction of non-positive curvature is not applied: the dipoles equal
    # those after one iteration fewer
    with PolFMM(pos, q, alpha, p=6, depth=3, mode="fp64", max_iter=info["iterations"] - 1) as g:
        info2 = g.solve(1e-12)
        mu_prev = g.dipoles()
    assert info2["iterations"] == info["iterations"] - 1
    np.testing.assert_array_equal(mu_stop, mu_prev)
    assert info["residual"] == info2["residual"]


def test_diverging_fixed_point_stops_on_residual_growth():
    pos, q, alpha = _catastrophe()
    with PolFMM(pos, q, alpha, p=6, depth=3, mode="fp64", solver="jacobi", max_iter=500) as f:
        info = f.solve(1e-10)
    assert info["status"] == _lib.ERR_NOT_CONVERGED
    assert info["iterations"] < 500


def test_converging_solves_are_not_stopped_as_stagnating():
    pos, q, alpha = synth.small_random(2024, 400, box=16.0, alpha_range=(0.3, 1.2))
    for solver in ("pcg", "jacobi"):
        with PolFMM(pos, q, alpha, p=6, depth=3, mode="fp64", solver=solver, max_iter=500) as f:
            info = f.solve(1e-10)
        assert info["converged"], (solver, info)


def test_out_of_memory_at_every_allocation_of_a_build():
    """fmm_build must return out-of-memory, leave *ctx NULL and free what it
    had allocated, whichever allocation fails."""
    lib = _lib.load()
    w = synth.workload(1)
    x, qv, av = (np.ascontiguousarray(a, dtype=np.float64) for a in (w.pos, w.q, w.alpha))
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    opt = _lib.Options()
    lib.fmm_default_options(ctypes.byref(opt))
    opt.mode = _lib.MIXED  # the mode with the most allocations (tensor-core M2L state)

    def build():
        h = ctypes.c_void_p()
        st = lib.fmm_build(ctypes.byref(h), w.n, ptr(x), ptr(qv), ptr(av), 6, 3, ctypes.byref(opt), 0)
        return st, h

    lib.fmm_testing_alloc_hook(-1)
    st, h = build()  # warm-up: module load, first context
    assert st == 0
    lib.fmm_destroy(h)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    lib.fmm_testing_alloc_hook(-1)
    st, h = build()
    assert st == 0
    lib.fmm_destroy(h)
    count = lib.fmm_testing_alloc_hook(-1)
    assert count > 20
    for k in range(count):
        lib.fmm_testing_alloc_hook(k)
        st, h = build()
        assert st == _lib.ERR_OUT_OF_MEMORY, (k, st)
        assert not h.value, k
    lib.fmm_testing_alloc_hook(-1)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert abs(free1 - free0) <= 4 << 20, (free0, free1)
    st, h = build()  # the library is still usable
    assert st == 0
    lib.fmm_destroy(h)


def test_energy_call_is_the_stationary_energy():
    w = synth.workload(1)
    with PolFMM(w.pos, w.q, w.alpha, p=4, depth=3) as f:
        with pytest.raises(PolFMMError) as e:
            f.energy()
        assert e.value.status == _lib.ERR_STATE
        f.solve(1e-12)
        e1 = f.energy()
        out = f.energy_forces(forces=False, dq=False, dalpha=False)
        lo, side = f.root_box()
    ref = oracle.polarizable_energy(w.pos, w.q, w.alpha, method="fmm", p=4, depth=3, root=(lo, side), tol=1e-13)
    assert e1["U"] == pytest.approx(ref["U"], rel=1e-10)
    assert e1["Uqq"] == pytest.approx(ref["Uqq"], rel=1e-12)
    # stationary and full forms agree at convergence
    assert e1["Upol"] == pytest.approx(out["Upol"], rel=1e-9)
