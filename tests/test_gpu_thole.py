"""Thole damping of the dipole-dipole interaction on the GPU (NEXT-2; reading:
Thole's exponential model as used by AMOEBA, a = 0.39) against the oracle's
FMM with the same damped-minus-undamped pair terms, same order and tree: the
converged energy, dipoles and every gradient, with exclusions and field
charges too; the MIXED gate; a rebuild; switching it off; bad arguments."""
import numpy as np
import pytest

import oracle
import synth
from oracle import polaris

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1408_6527_gb300 import PolFMM, PolFMMError, _lib  # noqa: E402
from siteerr import max_site_err  # noqa: E402

A = 0.39


def dev(a):
    return torch.as_tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy() if isinstance(t, torch.Tensor) else np.asarray(t)


def _system(n=300, seed=11, box=14.0):
    pos, q, alpha = synth.small_random(seed, n, box=box, alpha_range=(0.5, 2.0))
    rng = np.random.default_rng(seed + 1)
    qE = q + rng.normal(0.0, 0.1, n)
    alpha = alpha.copy()
    alpha[rng.choice(n, n // 6, replace=False)] = 0.0
    d = np.linalg.norm(pos[:, None] - pos[None], axis=2)
    np.fill_diagonal(d, np.inf)
    excl = sorted({tuple(sorted((i, int(np.argmin(d[i]))))) for i in range(0, n, 3)})
    return pos, q, qE, alpha, excl


@pytest.mark.parametrize("with_excl,with_qE", [(False, False), (True, True)])
def test_damped_energy_dipoles_and_gradients_fp64(with_excl, with_qE):
    pos, q, qE, alpha, excl = _system()
    p, depth = 6, 3
    ex = excl if with_excl else []
    qe = qE if with_qE else q
    with PolFMM(dev(pos), dev(q), dev(alpha), p=p, depth=depth, max_iter=500) as f:
        if with_excl:
            f.set_exclusions(ex)
        if with_qE:
            f.set_field_charges(dev(qE))
        f.set_thole(A)
        info = f.solve(1e-13)
        out = f.energy_forces()
        mu = host(f.dipoles())
        root = f.root_box()
    assert info["converged"]
    ref = polaris.polaris_energy(pos, q, qe, alpha, ex, method="fmm", p=p, depth=depth, root=root, solve="pcg",
                                 tol=1e-13, thole=A)
    und = polaris.polaris_energy(pos, q, qe, alpha, ex, method="fmm", p=p, depth=depth, root=root, solve="pcg",
                                 tol=1e-13)
    assert abs(ref["U"] - und["U"]) > 1e-4 * abs(und["U"])  # the damping matters here
    assert out["U"] == pytest.approx(ref["U"], rel=1e-10)
    assert out["Upol"] == pytest.approx(ref["Upol"], rel=1e-9)
    assert oracle.rel_rms(mu, ref["mu"]) < 1e-9 and max_site_err(mu, ref["mu"]) < 1e-7
    checks = [("F", host(out["F"]), ref["F"]), ("dUdalpha", host(out["dUdalpha"]), ref["dUdalpha"])]
    if not with_qE:
        checks.append(("dUdq", host(out["dUdq"]), ref["dUdq"] + ref["dUdqE"]))
    for k, a, b in checks:
        assert oracle.rel_rms(a, b) < 1e-9, k
        assert max_site_err(a, b) < 1e-7, k


def test_damping_survives_a_rebuild_and_switches_off():
    pos, q, qE, alpha, excl = _system(n=200, seed=13)
    moved = pos + 0.05 * np.random.default_rng(3).normal(size=pos.shape)
    root = (oracle.root_box(pos)[0] - 1.0, oracle.root_box(pos)[1] + 2.0)
    with PolFMM(dev(pos), dev(q), dev(alpha), p=5, depth=3, root_box=root) as f:
        f.set_thole(A)
        f.solve(1e-12)
        f.update_positions(dev(moved))
        f.reset_dipoles()
        f.solve(1e-12)
        a = f.energy_forces()
        f.set_thole(0.0)
        f.reset_dipoles()
        f.solve(1e-12)
        off = f.energy_forces()
    with PolFMM(dev(moved), dev(q), dev(alpha), p=5, depth=3, root_box=root) as g:
        g.set_thole(A)
        g.solve(1e-12)
        b = g.energy_forces()
    with PolFMM(dev(moved), dev(q), dev(alpha), p=5, depth=3, root_box=root) as h:
        h.solve(1e-12)
        c = h.energy_forces()
    assert a["U"] == pytest.approx(b["U"], rel=1e-12)
    assert oracle.rel_rms(host(a["F"]), host(b["F"])) < 1e-11
    assert off["U"] == pytest.approx(c["U"], rel=1e-12)
    assert oracle.rel_rms(host(off["F"]), host(c["F"])) < 1e-11


def test_mixed_gate_with_damping():
    """The 30k globule with Thole damping: MIXED (FP32 pair corrections in the
    solve) against FP64 on the same tree."""
    w = synth.workload(2)
    res = {}
    for mode, tol in (("fp64", 1e-8), ("mixed", 1e-7)):
        with PolFMM(dev(w.pos), dev(w.q), dev(w.alpha), p=w.p, depth=w.depth, mode=mode, max_iter=500) as f:
            f.set_thole(A)
            info = f.solve(tol)
            assert info["converged"], (mode, info)
            out = f.energy_forces()
            res[mode] = (host(out["F"]), host(f.dipoles()), out["U"])
    (F64, mu64, U64), (Fmx, mumx, Umx) = res["fp64"], res["mixed"]
    print(f"MIXED vs FP64 with Thole damping: F {oracle.rel_rms(Fmx, F64):.2e} mu {oracle.rel_rms(mumx, mu64):.2e} "
          f"U {abs(Umx - U64) / abs(U64):.2e}")
    assert oracle.rel_rms(Fmx, F64) < 1e-5
    assert oracle.rel_rms(mumx, mu64) < 1e-5
    assert abs(Umx - U64) < 1e-6 * abs(U64)


def test_invalid_thole_parameter():
    pos, q, qE, alpha, excl = _system(n=50, seed=17, box=10.0)
    with PolFMM(pos, q, alpha, p=4, depth=2) as f:
        for bad in (-0.1, float("nan"), float("inf")):
            with pytest.raises(PolFMMError) as e:
                f.set_thole(bad)
            assert e.value.status == _lib.ERR_INVALID_ARG
