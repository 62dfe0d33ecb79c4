"""Exclusion lists and field charges on the GPU (Sec. II.A starred sums; Sec.
III, the field charges q^E) against the oracle's FMM with the same exclusion
correction (FMM over all pairs minus the excluded pairs' direct terms), same
order and tree: single passes, the converged energy and every gradient, the
MIXED precision gate, and the lists kept across a rebuild."""
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


def dev(a):
    return torch.as_tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy() if isinstance(t, torch.Tensor) else np.asarray(t)


def _system(n=300, seed=11, box=15.0):
    pos, q, alpha = synth.small_random(seed, n, box=box, alpha_range=(0.3, 1.0))
    rng = np.random.default_rng(seed + 1)
    qE = q + rng.normal(0.0, 0.1, n)
    alpha = alpha.copy()
    alpha[rng.choice(n, n // 5, replace=False)] = 0.0
    # excluded pairs: every site with its nearest neighbour and a second, farther
    # partner (pairs in the near field and, at depth 3, some in the far field)
    d = np.linalg.norm(pos[:, None] - pos[None], axis=2)
    np.fill_diagonal(d, np.inf)
    order = np.argsort(d, axis=1)
    excl = sorted({tuple(sorted((i, int(order[i, 0])))) for i in range(n)} |
                  {tuple(sorted((i, int(order[i, 40])))) for i in range(0, n, 7)})
    return pos, q, qE, alpha, excl


def _oracle_fields(pos, excl, p, depth, root, w=None, mu=None):
    f = oracle.fmm_fields(pos, w, mu, p=p, depth=depth, root=root)
    phi, E, G = f["phi"].copy(), f["E"].copy(), f["G"].copy()
    if w is not None:
        c = polaris._excluded_correction(pos, excl, w)
        phi, E, G = phi - c[0], E - c[1], G - c[2]
    if mu is not None:
        c = polaris._excluded_correction(pos, excl, None, mu)
        phi, E, G = phi - c[0], E - c[1], G - c[2]
    return phi, E, G


def test_passes_without_the_excluded_pairs_fp64():
    pos, q, qE, alpha, excl = _system()
    p, depth = 6, 3
    mu = 0.3 * np.random.default_rng(2).normal(size=pos.shape)
    with PolFMM(dev(pos), dev(q), dev(alpha), p=p, depth=depth) as f:
        f.set_exclusions(excl)
        st = f.static_field()
        Emu = host(f.dipole_field(dev(mu)))
        tot = f.total_field(dev(mu))
        root = f.root_box()
    phi, E, _ = _oracle_fields(pos, excl, p, depth, root, w=q)
    for a, b in ((host(st["phi"]), phi), (host(st["E"]), E)):
        assert oracle.rel_rms(a, b) < 1e-10 and max_site_err(a, b) < 1e-8
    _, Em, _ = _oracle_fields(pos, excl, p, depth, root, mu=mu)
    assert oracle.rel_rms(Emu, Em) < 1e-10 and max_site_err(Emu, Em) < 1e-8
    phit, Et, Gt = _oracle_fields(pos, excl, p, depth, root, w=q, mu=mu)
    for a, b in ((host(tot["phi"]), phit), (host(tot["E"]), Et), (host(tot["G"]), Gt)):
        assert oracle.rel_rms(a, b) < 1e-10 and max_site_err(a, b) < 1e-8
    # the exclusions matter at this size: the field without them differs
    full = oracle.fmm_fields(pos, q, None, p=p, depth=depth, root=root)["E"]
    assert oracle.rel_rms(full, E) > 1e-2


@pytest.mark.parametrize("with_excl,with_qE", [(True, True), (True, False), (False, True)])
def test_converged_energy_and_gradients_fp64(with_excl, with_qE):
    pos, q, qE, alpha, excl = _system()
    p, depth = 6, 3
    ex = excl if with_excl else []
    qe = qE if with_qE else q
    with PolFMM(dev(pos), dev(q), dev(alpha), p=p, depth=depth, max_iter=500) as f:
        if with_excl:
            f.set_exclusions(ex)
        if with_qE:
            f.set_field_charges(dev(qE))
        info = f.solve(1e-13)
        e_st = f.energy()
        out = f.energy_forces()
        mu = host(f.dipoles())
        dqE = host(f.field_charge_gradient()) if with_qE else None
        root = f.root_box()
    assert info["converged"]
    ref = polaris.polaris_energy(pos, q, qe, alpha, ex, method="fmm", p=p, depth=depth, root=root, solve="pcg",
                                 tol=1e-13)
    assert out["U"] == pytest.approx(ref["U"], rel=1e-10)
    assert out["Uqq"] == pytest.approx(ref["Uqq"], rel=1e-12)
    assert out["Upol"] == pytest.approx(ref["Upol"], rel=1e-9)
    assert e_st["U"] == pytest.approx(ref["U"], rel=1e-9)
    assert oracle.rel_rms(mu, ref["mu"]) < 1e-9 and max_site_err(mu, ref["mu"]) < 1e-7
    checks = [("F", host(out["F"]), ref["F"]), ("dUdalpha", host(out["dUdalpha"]), ref["dUdalpha"])]
    if with_qE:
        checks += [("dUdq", host(out["dUdq"]), ref["dUdq"]), ("dUdqE", dqE, ref["dUdqE"])]
    else:  # one charge set in both roles: dU/dq is the total potential
        checks += [("dUdq", host(out["dUdq"]), ref["dUdq"] + ref["dUdqE"])]
    for k, a, b in checks:
        assert oracle.rel_rms(a, b) < 1e-9, k
        assert max_site_err(a, b) < 1e-7, k


def test_mixed_gate_with_exclusions_and_field_charges():
    """The 30k globule with a bond stand-in (each site excluded with its nearest
    neighbour) and field charges: MIXED against FP64 on the same tree."""
    w = synth.workload(2)
    rng = np.random.default_rng(5)
    qE = w.q + rng.normal(0.0, 0.05, w.n)
    from scipy.spatial import cKDTree

    _, nn = cKDTree(w.pos).query(w.pos, k=2)
    excl = np.unique(np.sort(np.stack([np.arange(w.n), nn[:, 1]], 1), axis=1), axis=0)
    res = {}
    # tolerances of the plain MIXED gate test: the force error at a MIXED solve
    # tolerance of 1e-6 is dominated by the solve, not by the arithmetic
    for mode, tol in (("fp64", 1e-8), ("mixed", 1e-7)):
        with PolFMM(dev(w.pos), dev(w.q), dev(w.alpha), p=w.p, depth=w.depth, mode=mode, max_iter=500) as f:
            f.set_exclusions(excl)
            f.set_field_charges(dev(qE))
            info = f.solve(tol)
            assert info["converged"], (mode, info)
            out = f.energy_forces()
            res[mode] = (host(out["F"]), host(f.dipoles()), out["U"], host(f.field_charge_gradient()))
    F64, mu64, U64, g64 = res["fp64"]
    Fmx, mumx, Umx, gmx = res["mixed"]
    print(f"MIXED vs FP64 with exclusions and field charges: F {oracle.rel_rms(Fmx, F64):.2e} "
          f"mu {oracle.rel_rms(mumx, mu64):.2e} U {abs(Umx - U64) / abs(U64):.2e} dU/dqE {oracle.rel_rms(gmx, g64):.2e}")
    assert oracle.rel_rms(Fmx, F64) < 1e-5
    assert oracle.rel_rms(mumx, mu64) < 1e-5
    assert abs(Umx - U64) < 1e-6 * abs(U64)
    assert oracle.rel_rms(gmx, g64) < 1e-5


def test_exclusions_and_field_charges_survive_a_rebuild():
    pos, q, qE, alpha, excl = _system(n=200, seed=13)
    moved = pos + 0.05 * np.random.default_rng(3).normal(size=pos.shape)
    root = (oracle.root_box(pos)[0] - 1.0, oracle.root_box(pos)[1] + 2.0)
    outs = []
    with PolFMM(dev(pos), dev(q), dev(alpha), p=5, depth=3, root_box=root) as f:
        f.set_exclusions(excl)
        f.set_field_charges(dev(qE))
        f.solve(1e-12)
        f.update_positions(dev(moved))
        f.reset_dipoles()
        f.solve(1e-12)
        o = f.energy_forces()
        outs.append((o["U"], host(o["F"]), host(f.field_charge_gradient())))
    with PolFMM(dev(moved), dev(q), dev(alpha), p=5, depth=3, root_box=root) as g:
        g.set_exclusions(excl)
        g.set_field_charges(dev(qE))
        g.solve(1e-12)
        o = g.energy_forces()
        outs.append((o["U"], host(o["F"]), host(g.field_charge_gradient())))
    assert outs[0][0] == pytest.approx(outs[1][0], rel=1e-12)
    assert oracle.rel_rms(outs[0][1], outs[1][1]) < 1e-11
    assert oracle.rel_rms(outs[0][2], outs[1][2]) < 1e-11


def test_invalid_exclusions_and_state():
    pos, q, qE, alpha, excl = _system(n=50, seed=17, box=10.0)
    with PolFMM(pos, q, alpha, p=4, depth=2) as f:
        for bad in ([(0, 0)], [(0, 50)], [(-1, 3)]):
            with pytest.raises(PolFMMError) as e:
                f.set_exclusions(bad)
            assert e.value.status == _lib.ERR_INVALID_ARG
        f.set_field_charges(qE)
        with pytest.raises(PolFMMError) as e:
            f.field_charge_gradient()  # no force pass yet
        assert e.value.status == _lib.ERR_STATE
        f.set_exclusions(excl)
        f.set_exclusions([])  # cleared: back to all pairs
        f.solve(1e-12)
        a = f.energy_forces()
    with PolFMM(pos, q, alpha, p=4, depth=2) as g:
        g.set_field_charges(qE)
        g.solve(1e-12)
        b = g.energy_forces()
    assert a["U"] == pytest.approx(b["U"], rel=1e-13)
