"""Pins of the exclusion-list / field-charge oracle (Sec. II.A, Sec. III):
reduction to the pinned path, finite differences of every gradient, full
exclusion of a site = its removal, no field charges = no polarization,
Newton's third law, and the FMM with its exclusion correction."""
import numpy as np
import pytest

import oracle
import synth
from oracle import polaris

# the coupled-site closed forms and the main path are pinned in test_oracle_pins.py


def _system(n=60, seed=3):
    pos, q, alpha = synth.small_random(seed, n, box=10.0, alpha_range=(0.3, 1.0))
    rng = np.random.default_rng(seed + 1)
    qE = q + rng.normal(0.0, 0.1, n)
    alpha = alpha.copy()
    alpha[rng.choice(n, n // 5, replace=False)] = 0.0  # some sites without polarizability
    # excluded pairs: each site with its nearest neighbour (a bond list stand-in)
    d = np.linalg.norm(pos[:, None] - pos[None], axis=2)
    np.fill_diagonal(d, np.inf)
    excl = sorted({tuple(sorted((i, int(np.argmin(d[i]))))) for i in range(n)})
    return pos, q, qE, alpha, excl


def test_without_exclusions_and_with_qE_equal_q_it_is_the_pinned_path():
    pos, q, _, alpha, _ = _system()
    a = polaris.polaris_energy(pos, q, q, alpha)
    b = oracle.polarizable_energy(pos, q, alpha, method="direct", solve="dense")
    assert abs(a["U"] - b["U"]) < 1e-12 * abs(b["U"])
    for k_a, k_b in (("F", "F"), ("dUdalpha", "dUdalpha"), ("mu", "mu")):
        assert oracle.rel_rms(a[k_a], b[k_b]) < 1e-11, k_a
    # with qE = q the two charge gradients add up to the total potential
    assert oracle.rel_rms(a["dUdq"] + a["dUdqE"], b["dUdq"]) < 1e-11


def test_gradients_are_finite_differences_of_the_energy():
    pos, q, qE, alpha, excl = _system()
    ref = polaris.polaris_energy(pos, q, qE, alpha, excl)
    U = lambda **kw: polaris.polaris_energy(**{"pos": pos, "q": q, "qE": qE, "alpha": alpha,
                                               "exclusions": excl, **kw})["U"]
    rng = np.random.default_rng(9)
    h = 1e-5
    for i in rng.choice(pos.shape[0], 4, replace=False):
        for d in range(3):
            xp, xm = pos.copy(), pos.copy()
            xp[i, d] += h
            xm[i, d] -= h
            fd = -(U(pos=xp) - U(pos=xm)) / (2 * h)
            assert abs(fd - ref["F"][i, d]) < 1e-6 * np.abs(ref["F"]).max()
        for name, key in (("q", "dUdq"), ("qE", "dUdqE"), ("alpha", "dUdalpha")):
            vp = {"q": q, "qE": qE, "alpha": alpha}[name].copy()
            vm = vp.copy()
            vp[i] += h
            vm[i] -= h
            if name == "alpha" and vm[i] < 0:  # one-sided at alpha = 0
                fd = (U(**{name: vp}) - ref["U"]) / h
                assert abs(fd - ref[key][i]) < 1e-4 * np.abs(ref[key]).max()
                continue
            fd = (U(**{name: vp}) - U(**{name: vm})) / (2 * h)
            assert abs(fd - ref[key][i]) < 1e-6 * np.abs(ref[key]).max(), (name, i)


def test_excluding_every_pair_of_a_site_removes_it():
    pos, q, qE, alpha, excl = _system()
    k = int(np.nonzero(alpha > 0)[0][3])  # a polarizable site: its dipole must vanish too
    excl_k = sorted(set(excl) | {tuple(sorted((k, j))) for j in range(pos.shape[0]) if j != k})
    a = polaris.polaris_energy(pos, q, qE, alpha, excl_k)
    keep = np.arange(pos.shape[0]) != k
    old = np.nonzero(keep)[0]
    remap = {int(o): i for i, o in enumerate(old)}
    excl_rest = [(remap[i], remap[j]) for i, j in excl if i != k and j != k]
    b = polaris.polaris_energy(pos[keep], q[keep], qE[keep], alpha[keep], excl_rest)
    assert abs(a["U"] - b["U"]) < 1e-12 * abs(b["U"])
    assert np.abs(a["mu"][k]).max() == 0.0
    assert oracle.rel_rms(a["F"][keep], b["F"]) < 1e-11
    assert np.abs(a["F"][k]).max() == 0.0


def test_without_field_charges_there_is_no_polarization():
    pos, q, _, alpha, excl = _system()
    a = polaris.polaris_energy(pos, q, np.zeros_like(q), alpha, excl)
    assert np.abs(a["mu"]).max() == 0.0 and a["Upol"] == 0.0
    assert abs(a["U"] - a["Uqq"]) == 0.0


def test_stationary_energy_and_newtons_third_law():
    pos, q, qE, alpha, excl = _system()
    a = polaris.polaris_energy(pos, q, qE, alpha, excl)
    assert abs(a["Upol"] - a["Upol_stationary"]) < 1e-10 * abs(a["Upol"])
    assert np.abs(a["F"].sum(0)).max() < 1e-11 * np.abs(a["F"]).sum()


def test_fmm_with_the_exclusion_correction_matches_the_pair_sums():
    """An FMM over all pairs minus the excluded pairs' direct terms: exact when
    every pair is in the near field (depth 1), and with a far field (depth 2)
    no less accurate than the same FMM without exclusions."""
    pos, q, qE, alpha, excl = _system(n=120, seed=5)
    lo, side = oracle.root_box(pos)
    a = polaris.polaris_energy(pos, q, qE, alpha, excl)
    b = polaris.polaris_energy(pos, q, qE, alpha, excl, method="fmm", p=8, depth=1, root=(lo, side))
    assert abs(a["U"] - b["U"]) < 1e-13 * abs(a["U"])
    assert oracle.rel_rms(b["F"], a["F"]) < 1e-13
    err = {}
    for ex in ((), excl):
        d = polaris.polaris_energy(pos, q, qE, alpha, ex)
        f = polaris.polaris_energy(pos, q, qE, alpha, ex, method="fmm", p=8, depth=2, root=(lo, side))
        err[len(ex) > 0] = oracle.rel_rms(f["F"], d["F"])
    assert 0.0 < err[True] < 1.5 * err[False]


def test_pcg_solve_reproduces_the_dense_solve():
    """The conjugate-gradient solve of the same (exactly symmetric) dense
    operator gives the Cholesky dipoles, energy and gradients."""
    pos, q, qE, alpha, excl = _system()
    a = polaris.polaris_energy(pos, q, qE, alpha, excl)
    b = polaris.polaris_energy(pos, q, qE, alpha, excl, solve="pcg", tol=1e-14)
    assert abs(a["U"] - b["U"]) < 1e-12 * abs(a["U"])
    for k in ("F", "dUdq", "dUdqE", "dUdalpha", "mu"):
        assert oracle.rel_rms(b[k], a[k]) < 1e-10, k


# ---------------------------------------------------------------------------
# Thole damping of the dipole-dipole tensor (reading: Thole's exponential model
# as used by AMOEBA; the paper cites Thole without printing the form)
# ---------------------------------------------------------------------------

def test_thole_factors_closed_form_and_limits():
    pos = np.array([[0.0, 0.0, 0.0], [1.5, 0.0, 0.0], [40.0, 0.0, 0.0]])
    alpha = np.array([1.0, 8.0, 1.0])
    r, ri = polaris._pairs(pos)
    th = polaris.thole_factors(r, ri, alpha, 0.39, polaris._mask(3, []))
    u = 1.5 / (1.0 * 8.0) ** (1 / 6)
    au3 = 0.39 * u ** 3
    assert th["l3"][0, 1] == pytest.approx(1 - np.exp(-au3), rel=1e-14)
    assert th["l5"][0, 1] == pytest.approx(1 - (1 + au3) * np.exp(-au3), rel=1e-14)
    # far apart: undamped to FP64; symmetric in i, j
    assert th["l3"][0, 2] == 1.0 and th["l5"][0, 2] == 1.0
    np.testing.assert_array_equal(th["l3"], th["l3"].T)
    # a site without polarizability is never damped
    th0 = polaris.thole_factors(r, ri, np.array([0.0, 8.0, 1.0]), 0.39, polaris._mask(3, []))
    assert th0["l3"][0, 1] == 1.0 and th0["l5"][0, 1] == 1.0 and th0["d3r"][0, 1] == 0.0


def test_thole_damping_gradients_are_finite_differences_of_the_energy():
    pos, q, qE, alpha, excl = _system()
    a = 0.39
    ref = polaris.polaris_energy(pos, q, qE, alpha, excl, thole=a)
    und = polaris.polaris_energy(pos, q, qE, alpha, excl)
    assert abs(ref["U"] - und["U"]) > 1e-5 * abs(und["U"])  # the damping acts on this system
    U = lambda **kw: polaris.polaris_energy(**{"pos": pos, "q": q, "qE": qE, "alpha": alpha,
                                               "exclusions": excl, "thole": a, **kw})["U"]
    rng = np.random.default_rng(10)
    h = 1e-5
    for i in rng.choice(np.nonzero(alpha > 0)[0], 4, replace=False):
        for d in range(3):
            xp, xm = pos.copy(), pos.copy()
            xp[i, d] += h
            xm[i, d] -= h
            fd = -(U(pos=xp) - U(pos=xm)) / (2 * h)
            assert abs(fd - ref["F"][i, d]) < 1e-6 * np.abs(ref["F"]).max()
        ap, am = alpha.copy(), alpha.copy()
        ap[i] += h
        am[i] -= h
        fd = (U(alpha=ap) - U(alpha=am)) / (2 * h)
        assert abs(fd - ref["dUdalpha"][i]) < 1e-6 * np.abs(ref["dUdalpha"]).max()
    # Newton's third law survives the damping
    assert np.abs(ref["F"].sum(0)).max() < 1e-10 * np.abs(ref["F"]).max()


def test_thole_fmm_correction_matches_the_damped_pair_sums():
    """FMM over all pairs plus the damped-minus-undamped pair terms: exact when
    every pair is in the near field (depth 1), and with a far field (depth 2)
    no less accurate than the same FMM without damping."""
    pos, q, qE, alpha, excl = _system(n=120, seed=5)
    lo, side = oracle.root_box(pos)
    a = polaris.polaris_energy(pos, q, qE, alpha, excl, thole=0.39)
    b = polaris.polaris_energy(pos, q, qE, alpha, excl, method="fmm", p=8, depth=1, root=(lo, side), thole=0.39)
    assert abs(a["U"] - b["U"]) < 1e-13 * abs(a["U"])
    for k in ("F", "dUdalpha", "mu"):
        assert oracle.rel_rms(b[k], a[k]) < 1e-12, k
    err = {}
    for th in (0.0, 0.39):
        d = polaris.polaris_energy(pos, q, qE, alpha, excl, thole=th)
        f = polaris.polaris_energy(pos, q, qE, alpha, excl, method="fmm", p=8, depth=2, root=(lo, side), thole=th)
        err[th] = oracle.rel_rms(f["F"], d["F"])
    assert 0.0 < err[0.39] < 1.5 * err[0.0]
