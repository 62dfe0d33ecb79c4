"""Pins of the CPU oracle against closed forms, symbolic algebra, exact
identities and the paper's own constructions -- never against itself.

Each test names the passage of Coles & Masella (arXiv:1408.6527) it pins.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------------------
# derivative tensor of the Green's function 1/r (Sec. II.B, App. D)
# ---------------------------------------------------------------------------

def test_derivatives_match_symbolic_differentiation():
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z", real=True)
    f = 1 / sp.sqrt(x * x + y * y + z * z)
    R = (sp.Rational(7, 10), sp.Rational(-13, 10), sp.Rational(21, 10))
    p = 6
    got = oracle.derivatives([float(v) for v in R], p)
    mi = oracle.multi_indices(p)
    for c, (a, b, cc) in enumerate(mi):
        expr = f
        if a:
            expr = sp.diff(expr, x, int(a))
        if b:
            expr = sp.diff(expr, y, int(b))
        if cc:
            expr = sp.diff(expr, z, int(cc))
        ref = float(expr.subs({x: R[0], y: R[1], z: R[2]}))
        assert abs(got[c] - ref) <= 1e-12 * max(1.0, abs(ref)), (a, b, cc, got[c], ref)


def test_derivatives_low_order_closed_forms():
    R = np.array([0.3, -1.1, 0.8])
    r = np.linalg.norm(R)
    xx, yy, zz = R
    a = oracle.derivatives(R, 3)
    mi = [tuple(v) for v in oracle.multi_indices(3)]
    ref = {
        (0, 0, 0): 1 / r,
        (1, 0, 0): -xx / r**3,
        (0, 0, 1): -zz / r**3,
        (2, 0, 0): 3 * xx * xx / r**5 - 1 / r**3,
        (1, 1, 0): 3 * xx * yy / r**5,
        (3, 0, 0): -15 * xx**3 / r**7 + 9 * xx / r**5,
        (2, 1, 0): -15 * xx * xx * yy / r**7 + 3 * yy / r**5,
        (1, 1, 1): -15 * xx * yy * zz / r**7,
    }
    for k, v in ref.items():
        assert a[mi.index(k)] == pytest.approx(v, rel=1e-13, abs=1e-15)


def test_derivatives_are_harmonic():
    """1/r is harmonic: a_{n+2x} + a_{n+2y} + a_{n+2z} = 0 for every n."""
    p = 10
    a = oracle.derivatives([1.3, 0.4, -0.9], p)
    mi = [tuple(v) for v in oracle.multi_indices(p)]
    pos = {k: i for i, k in enumerate(mi)}
    scale = np.abs(a).max()
    for (nx, ny, nz) in mi:
        if nx + ny + nz > p - 2:
            continue
        s = a[pos[(nx + 2, ny, nz)]] + a[pos[(nx, ny + 2, nz)]] + a[pos[(nx, ny, nz + 2)]]
        assert abs(s) <= 1e-12 * scale


# ---------------------------------------------------------------------------
# single-box operators (Sec. II.B)
# ---------------------------------------------------------------------------

def _cluster(rng, centre, radius, m):
    u = rng.normal(size=(m, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    return np.asarray(centre) + radius * u * rng.random((m, 1)) ** (1 / 3)


def test_far_field_expansion_converges_to_direct():
    """P2M -> M2L -> L2P reproduces the direct potential, field and field
    gradient of a remote cluster of charges and point dipoles, with an error
    that falls geometrically with p (the truncated two-centre Taylor
    expansion of Sec. II.B)."""
    rng = _rng(1)
    zA = np.array([0.0, 0.0, 0.0])
    zB = np.array([6.0, -3.0, 4.0])
    xs = _cluster(rng, zA, 0.8, 12)
    q = rng.normal(size=12)
    mu = rng.normal(size=(12, 3))
    xt = _cluster(rng, zB, 0.8, 5)
    errs = []
    for p in (2, 4, 6, 8, 10, 12):
        M = oracle.p2m(p, zA, xs, q, mu)
        F = oracle.m2l(p, zB - zA, M)
        e = []
        for x in xt:
            phi, dphi, ddphi = oracle.l2p(p, x - zB, F)
            d = oracle.direct_fields(np.vstack([x, xs]), np.concatenate([[0.0], q]),
                                     np.vstack([[0, 0, 0], mu]), targets=[0])
            e.append(max(abs(phi - d["phi"][0]) / abs(d["phi"][0]),
                         np.linalg.norm(-dphi - d["E"][0]) / np.linalg.norm(d["E"][0]),
                         np.linalg.norm(-ddphi - d["G"][0]) / np.linalg.norm(d["G"][0])))
        errs.append(max(e))
    # |r_a| + |r_b| <= 1.6, |z_B - z_A| = 7.8: ratio ~0.2 per order, so at
    # least a factor 0.2 for every two orders; the field gradient has
    # effective order p - 2
    for a, b in zip(errs, errs[1:]):
        assert b < a * 0.2
    assert errs[-1] < 2e-6


def test_dipole_multipole_is_the_paper_charge_pair_limit():
    """Sec. II.C: a point dipole mu is a pair +-q^mu at x +- dl with
    mu = 2 |q^mu| dl.  The dipole multipole must equal the pair's multipole
    up to O(dl^2)."""
    rng = _rng(2)
    p = 6
    z = np.zeros(3)
    x = np.array([0.3, -0.2, 0.45])
    mu = rng.normal(size=3)
    dl_len = 1e-4
    dl = mu / np.linalg.norm(mu) * dl_len
    qmu = np.linalg.norm(mu) / (2 * dl_len)
    Mpair = oracle.p2m(p, z, np.vstack([x + dl, x - dl]), np.array([qmu, -qmu]))
    Mdip = oracle.p2m(p, z, x[None], None, mu[None])
    scale = np.abs(Mdip).max()
    assert np.abs(Mpair - Mdip).max() < 1e-6 * scale


def test_m2m_is_exact():
    """Shifting multipoles keeps every term (k <= n), so P2M at the child centre
    followed by M2M equals P2M at the parent centre (Sec. II.B)."""
    rng = _rng(3)
    p = 7
    zc = np.array([0.25, -0.25, 0.25])
    zp = np.zeros(3)
    xs = _cluster(rng, zc, 0.2, 9)
    q = rng.normal(size=9)
    mu = rng.normal(size=(9, 3))
    Mc = oracle.p2m(p, zc, xs, q, mu)
    Mp = oracle.m2m(p, zp - zc, Mc)
    Mref = oracle.p2m(p, zp, xs, q, mu)
    assert np.abs(Mp - Mref).max() <= 1e-13 * np.abs(Mref).max()


def test_l2l_preserves_the_local_polynomial():
    """A local expansion is a polynomial of degree p; re-expanding it about the
    child centre (L2L) and evaluating (L2P) gives the same values and
    derivatives as evaluating the parent expansion (Sec. II.B)."""
    rng = _rng(4)
    p = 6
    F = rng.normal(size=oracle.ncoef(p))
    zp = np.zeros(3)
    zc = np.array([-0.25, 0.25, 0.25])
    Fc = oracle.l2l(p, zc - zp, F)
    for _ in range(5):
        x = zc + 0.25 * (rng.random(3) * 2 - 1)
        a = oracle.l2p(p, x - zp, F)
        b = oracle.l2p(p, x - zc, Fc)
        assert b[0] == pytest.approx(a[0], rel=1e-12, abs=1e-12)
        np.testing.assert_allclose(b[1], a[1], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(b[2], a[2], rtol=1e-12, atol=1e-12)


def test_m2l_operator_is_symmetric():
    """Evaluating the same truncated expansion in both directions gives the
    mutual interaction (Sec. II.B, Newton's third law): for unit charges,
    sum_n (r_b^n/n!) F_n(B <- A) equals sum_n (r_a^n/n!) F_n(A <- B)."""
    p = 5
    zA = np.zeros(3)
    zB = np.array([2.0, 1.0, -2.0])
    xa = np.array([0.1, -0.2, 0.3])
    xb = zB + np.array([-0.3, 0.1, 0.2])
    FB = oracle.m2l(p, zB - zA, oracle.p2m(p, zA, xa[None], np.ones(1)))
    FA = oracle.m2l(p, zA - zB, oracle.p2m(p, zB, xb[None], np.ones(1)))
    assert oracle.l2p(p, xb - zB, FB)[0] == pytest.approx(oracle.l2p(p, xa - zA, FA)[0], rel=1e-14)


# ---------------------------------------------------------------------------
# direct sums and the induced dipoles: closed forms (Sec. II.A)
# ---------------------------------------------------------------------------

def test_two_charges_closed_form():
    x = np.array([[0.0, 0.0, 0.0], [1.2, -0.7, 2.0]])
    q = np.array([0.6, -1.3])
    r = np.linalg.norm(x[0] - x[1])
    out = oracle.polarizable_energy(x, q, np.zeros(2), method="direct", solve="dense")
    assert out["U"] == pytest.approx(q[0] * q[1] / r, rel=1e-14)
    F0 = q[0] * q[1] * (x[0] - x[1]) / r**3
    np.testing.assert_allclose(out["F"][0], F0, rtol=1e-13)
    np.testing.assert_allclose(out["F"][1], -F0, rtol=1e-13)
    np.testing.assert_allclose(out["dUdq"], [q[1] / r, q[0] / r], rtol=1e-14)


def test_charge_and_induced_dipole_closed_form():
    """Charge Q (alpha = 0) and a polarizable site alpha (q = 0) at distance r:
    mu = alpha Q rhat / r^2, U^pol = -alpha Q^2 / (2 r^4), force on the site
    -2 alpha Q^2 / r^5 rhat, dU/dalpha = -Q^2 / (2 r^4)."""
    Q, al, r = 0.8, 1.7, 3.1
    x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    for solve in ("dense", "pcg"):
        out = oracle.polarizable_energy(x, np.array([Q, 0.0]), np.array([0.0, al]), method="direct",
                                        solve=solve, tol=1e-14)
        np.testing.assert_allclose(out["mu"][1], [al * Q / r**2, 0, 0], rtol=1e-13)
        np.testing.assert_allclose(out["mu"][0], 0.0, atol=0)
        assert out["Upol"] == pytest.approx(-al * Q * Q / (2 * r**4), rel=1e-13)
        assert out["U"] == pytest.approx(-al * Q * Q / (2 * r**4), rel=1e-13)
        np.testing.assert_allclose(out["F"][1], [-2 * al * Q * Q / r**5, 0, 0], rtol=1e-12)
        np.testing.assert_allclose(out["F"][0], [2 * al * Q * Q / r**5, 0, 0], rtol=1e-12)
        assert out["dUdalpha"][1] == pytest.approx(-Q * Q / (2 * r**4), rel=1e-12)


def _two_site_solution(a1, a2, e1, e2, c):
    """mu1 = a1 (e1 + c mu2), mu2 = a2 (e2 + c mu1), solved by hand."""
    det = 1.0 - a1 * a2 * c * c
    m1 = (a1 * e1 + a1 * a2 * c * e2) / det
    m2 = (a2 * e2 + a1 * a2 * c * e1) / det
    return m1, m2


def test_two_polarizable_sites_closed_form():
    """Two coupled sites polarized by a charge: the dipole field couples the
    components along the pair axis by 2/r^3 and across it by -1/r^3
    (physical sign of the dipolar tensor of Sec. II.A)."""
    Q, h, s = 1.1, 2.5, 1.6
    a1, a2 = 1.4, 0.9
    x = np.array([[0.0, h, 0.0], [-s, 0.0, 0.0], [s, 0.0, 0.0]])
    r = 2 * s
    R = math.hypot(s, h)
    E1 = Q * (x[1] - x[0]) / R**3
    E2 = Q * (x[2] - x[0]) / R**3
    mx1, mx2 = _two_site_solution(a1, a2, E1[0], E2[0], 2 / r**3)
    my1, my2 = _two_site_solution(a1, a2, E1[1], E2[1], -1 / r**3)
    for solve in ("dense", "pcg"):
        out = oracle.polarizable_energy(x, np.array([Q, 0, 0]), np.array([0, a1, a2]), method="direct",
                                        solve=solve, tol=1e-15)
        np.testing.assert_allclose(out["mu"][1], [mx1, my1, 0], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(out["mu"][2], [mx2, my2, 0], rtol=1e-12, atol=1e-15)
        Upol = -0.5 * (mx1 * E1[0] + my1 * E1[1] + mx2 * E2[0] + my2 * E2[1])
        assert out["Upol"] == pytest.approx(Upol, rel=1e-12)


def test_fixed_dipole_dipole_energy_and_force():
    """U = [mu1.mu2 - 3 (mu1.rhat)(mu2.rhat)] / r^3 = -mu1 . E^{mu2}(x1); the force
    (mu1 . grad) E^{mu2} equals minus the gradient of that closed form."""
    rng = _rng(5)
    x1 = np.array([0.2, -0.1, 0.3])
    x2 = np.array([1.9, 1.1, -0.8])
    m1, m2 = rng.normal(size=3), rng.normal(size=3)

    def U(a):
        r = a - x2
        d = np.linalg.norm(r)
        return (m1 @ m2 - 3 * (m1 @ r) * (m2 @ r) / d**2) / d**3

    out = oracle.direct_fields(np.vstack([x1, x2]), None, np.vstack([np.zeros(3), m2]), targets=[0])
    assert -m1 @ out["E"][0] == pytest.approx(U(x1), rel=1e-13)
    G = out["G"][0]
    Gm = np.array([[G[0], G[1], G[2]], [G[1], G[3], G[4]], [G[2], G[4], G[5]]]) @ m1
    h = 1e-5
    fd = np.array([-(U(x1 + h * e) - U(x1 - h * e)) / (2 * h) for e in np.eye(3)])
    np.testing.assert_allclose(Gm, fd, rtol=1e-8)


# ---------------------------------------------------------------------------
# whole-system invariants: Newton's third law, stationarity (Sec. II.A, II.C)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def small_system():
    return synth.small_random(11, 40, box=9.0)


def test_newton_third_law_direct(small_system):
    pos, q, al = small_system
    out = oracle.polarizable_energy(pos, q, al, method="direct", solve="dense")
    F = out["F"]
    assert np.linalg.norm(F.sum(0)) <= 1e-12 * np.abs(F).sum()


def test_stationary_polarization_energy(small_system):
    """At the solution, U^pol = -1/2 sum mu.E^q (Eq. upol_derivatives with
    A = 1/2 sum |mu|^2/alpha)."""
    pos, q, al = small_system
    out = oracle.polarizable_energy(pos, q, al, method="direct", solve="dense")
    assert out["Upol"] == pytest.approx(out["Upol_stationary"], rel=1e-11)


def test_pcg_matches_dense_solve(small_system):
    pos, q, al = small_system
    a = oracle.polarizable_energy(pos, q, al, method="direct", solve="dense")
    b = oracle.polarizable_energy(pos, q, al, method="direct", solve="pcg", tol=1e-14)
    assert oracle.rel_rms(b["mu"], a["mu"]) < 1e-12
    assert b["U"] == pytest.approx(a["U"], rel=1e-13)


def test_gradients_match_finite_differences(small_system):
    """Because dU^pol/dmu = 0 at the solution, the analytic force, dU/dq and
    dU/dalpha need no derivative of the dipoles; central differences of U with
    the dipoles re-solved each time must agree (Sec. II.A, II.C)."""
    pos, q, al = small_system

    def U(p_, q_, a_):
        return oracle.polarizable_energy(p_, q_, a_, method="direct", solve="dense")["U"]

    base = oracle.polarizable_energy(pos, q, al, method="direct", solve="dense")
    h = 1e-5
    for i in (0, 7, 23):
        for d in range(3):
            pp = pos.copy(); pp[i, d] += h
            pm = pos.copy(); pm[i, d] -= h
            fd = -(U(pp, q, al) - U(pm, q, al)) / (2 * h)
            assert base["F"][i, d] == pytest.approx(fd, rel=1e-6, abs=1e-9)
        qp = q.copy(); qp[i] += h
        qm = q.copy(); qm[i] -= h
        assert base["dUdq"][i] == pytest.approx((U(pos, qp, al) - U(pos, qm, al)) / (2 * h), rel=1e-6, abs=1e-9)
        ap = al.copy(); ap[i] += h
        am = al.copy(); am[i] -= h
        assert base["dUdalpha"][i] == pytest.approx((U(pos, q, ap) - U(pos, q, am)) / (2 * h), rel=1e-5, abs=1e-9)


# ---------------------------------------------------------------------------
# the CPU FMM as a whole (Sec. II.B, Sec. III)
# ---------------------------------------------------------------------------

def test_fmm_exact_for_tight_remote_clusters():
    """Two tight clusters around the centres of non-adjacent level-2 boxes of a
    depth-4 tree: every far interaction goes P2M -> M2M -> M2L -> L2L -> L2P
    and converges fast, near pairs are direct.  At p = 12 the FMM equals the
    direct sum to ~1e-12."""
    rng = _rng(6)
    side = 16.0
    lo = np.zeros(3)
    cA = np.array([2.0, 2.0, 2.0])  # centre of level-2 box (0,0,0)
    cB = np.array([14.0, 10.0, 6.0])  # centre of level-2 box (3,2,1)
    xs = np.vstack([_cluster(rng, cA, 0.45, 20), _cluster(rng, cB, 0.45, 20)])
    q = rng.normal(size=40)
    mu = 0.3 * rng.normal(size=(40, 3))
    d = oracle.direct_fields(xs, q, mu)
    errs = []
    for p in (4, 8, 12):
        f = oracle.fmm_fields(xs, q, mu, p=p, depth=4, root=(lo, side))
        errs.append(max(oracle.rel_rms(f["E"], d["E"]), oracle.rel_rms(f["phi"], d["phi"]),
                        oracle.rel_rms(f["G"], d["G"])))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-11


def test_fmm_error_decays_with_order():
    w = synth.workload(1)
    d = oracle.direct_fields(w.pos, w.q)
    errs = [oracle.rel_rms(oracle.fmm_fields(w.pos, w.q, p=p, depth=3)["E"], d["E"]) for p in (2, 4, 6, 8)]
    for a, b in zip(errs, errs[1:]):
        assert b < 0.7 * a


def test_fmm_dipole_operator_is_symmetric():
    """a . T(b) = b . T(a) for the FMM dipole-field operator: the truncation
    |n| + |m| <= p is symmetric and the shift operators are exact, so the
    approximate operator stays symmetric (needed by conjugate gradients)."""
    pos, q, al = synth.small_random(12, 300, box=16.0)
    rng = _rng(7)
    a = rng.normal(size=(300, 3))
    b = rng.normal(size=(300, 3))
    Ta = oracle.fmm_fields(pos, None, a, p=4, depth=3)["E"]
    Tb = oracle.fmm_fields(pos, None, b, p=4, depth=3)["E"]
    assert np.sum(a * Tb) == pytest.approx(np.sum(b * Ta), rel=1e-12)


def test_fmm_forces_are_the_gradient_of_the_fmm_energy():
    """With the tree fixed, W = 1/2 sum (q Phi - mu.E) from the FMM is a smooth
    function of the positions whose exact gradient is -(q E + (grad E) mu)."""
    pos, q, al = synth.small_random(13, 200, box=14.0)
    rng = _rng(8)
    mu = 0.2 * rng.normal(size=(200, 3))
    lo, side = oracle.root_box(pos)
    lo = lo - 0.5
    side = side + 1.0
    p, depth = 4, 3

    def W(x):
        f = oracle.fmm_fields(x, q, mu, p=p, depth=depth, root=(lo, side))
        return 0.5 * (np.sum(q * f["phi"]) - np.sum(mu * f["E"]))

    f = oracle.fmm_fields(pos, q, mu, p=p, depth=depth, root=(lo, side))
    _, _, dUda = oracle.gradients(q, np.ones(200), mu, f)
    F, _, _ = oracle.gradients(q, np.ones(200), mu, f)
    h = 1e-5
    hcell = side / 2**depth
    checked = 0
    for i in range(200):
        u = (pos[i] - lo) / hcell
        if np.min(np.abs(u - np.round(u))) < 1e-3:
            continue
        for dd in range(3):
            pp = pos.copy(); pp[i, dd] += h
            pm = pos.copy(); pm[i, dd] -= h
            fd = -(W(pp) - W(pm)) / (2 * h)
            assert F[i, dd] == pytest.approx(fd, rel=2e-6, abs=1e-8)
        checked += 1
        if checked == 4:
            break
    assert checked == 4


def test_fmm_is_permutation_invariant():
    pos, q, al = synth.small_random(14, 250, box=15.0)
    rng = _rng(9)
    mu = rng.normal(size=(250, 3))
    perm = rng.permutation(250)
    a = oracle.fmm_fields(pos, q, mu, p=5, depth=3)
    b = oracle.fmm_fields(pos[perm], q[perm], mu[perm], p=5, depth=3)
    inv = np.argsort(perm)
    for k in ("phi", "E", "G"):
        np.testing.assert_allclose(b[k][inv], a[k], rtol=1e-11, atol=1e-12 * np.abs(a[k]).max())


def test_leaf_cells_brute_force():
    rng = _rng(10)
    x = rng.normal(size=(500, 3)) * 7
    lo, side = oracle.root_box(x)
    assert side == pytest.approx((x.max(0) - x.min(0)).max() * (1 + 1e-6), rel=1e-15)
    depth = 4
    c = oracle.leaf_cells(x, depth, lo, side)
    h = side / 2**depth
    assert c.min() >= 0 and c.max() < 2**depth
    assert np.all(lo + c * h <= x + 1e-12) and np.all(x < lo + (c + 1) * h + 1e-12)


def test_fmm_pcg_matches_direct_pcg_within_truncation():
    """The FMM-based solve converges to the direct solve's dipoles with an
    error of the order of the FMM truncation at that p (Sec. IV)."""
    pos, q, al = synth.small_random(15, 300, box=16.0)
    a = oracle.polarizable_energy(pos, q, al, method="direct", solve="dense")
    e = []
    for p in (3, 6, 9):
        b = oracle.polarizable_energy(pos, q, al, method="fmm", p=p, depth=3, tol=1e-12)
        e.append(oracle.rel_rms(b["F"], a["F"]))
    assert e[0] > e[1] > e[2]
    assert e[2] < 1e-2


# ---------------------------------------------------------------------------
# the paper's sphere test, qualitatively (Sec. IV.A)
# ---------------------------------------------------------------------------

def test_sphere_test_error_distribution_is_in_the_paper_range():
    """Sphere test of Sec. IV.A (4096 sites, r = 45 A, d_min = 2 A, +-e).  The
    paper reports, for its kd-tree at theta = 0.5 and p = 5, ~80 % of the
    per-atom force errors below 1e-4 and all below 1e-2 (tests/golden).  The
    octree rule used here is looser (theta ~ 0.87), so this checks the trend
    and the order of magnitude: at p = 5 most errors are below 1e-2 and
    raising p to 8 lowers the 80th percentile."""
    import json
    import os

    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_sphere_test.json")))
    rng = _rng(16)
    pos = synth.sites_sphere(rng, g["n_sites"], g["radius_A"], g["min_separation_A"])
    q = synth.charges_pm_equal(rng, pos.shape[0])
    d = oracle.direct_fields(pos, q)
    errs = {}
    for p in (5, 8):
        f = oracle.fmm_fields(pos, q, p=p, depth=3)
        errs[p] = oracle.per_site_rel_err(q[:, None] * f["E"], q[:, None] * d["E"])
    assert np.percentile(errs[5], 80) < 1e-2
    assert np.percentile(errs[8], 80) < np.percentile(errs[5], 80)
    assert np.max(errs[8]) < g["max_rel_force_error"] * 10


# ---------------------------------------------------------------------------
# the synthetic inputs
# ---------------------------------------------------------------------------

def test_workload1_inputs():
    w = synth.workload(1)
    assert w.n == 1000 and w.p == 4 and w.depth == 3
    from scipy.spatial import cKDTree
    dist, _ = cKDTree(w.pos).query(w.pos, k=2)
    assert dist[:, 1].min() >= 1.75
    assert abs(w.q.sum()) < 1e-12
    assert np.all(np.abs(w.q) <= 0.85)  # +-U(0.1, 0.8) shifted by the small mean
    assert w.alpha.min() >= 0.5 and w.alpha.max() <= 2.0
    w2 = synth.workload(1)
    np.testing.assert_array_equal(w.pos, w2.pos)


def test_workload1_dipole_matrix_is_positive_definite():
    """The dense dipole solve of Sec. II.A needs diag(1/alpha) - T positive
    definite (no polarization catastrophe); the cube workload must admit the
    Cholesky factorisation, and PCG with direct sums must reach 1e-10."""
    w = synth.workload(1)
    st = oracle.direct_fields(w.pos, w.q)
    mu = oracle.dense_dipole_solve(w.pos, w.alpha, st["E"])
    mu2, it, res, _ = oracle.pcg_dipole_solve(w.alpha, st["E"], lambda v: oracle.direct_fields(w.pos, None, v)["E"],
                                              tol=1e-10, max_iter=200)
    assert res <= 1e-10 and it < 120
    assert oracle.rel_rms(mu2, mu) < 1e-8


def test_smoke_input_is_positive_definite():
    """The induced-dipole equations (Sec. II.A) have a unique solution only where
    diag(1/alpha) - T is positive definite; the smoke cluster must lie there
    (dense eigenvalues of the 1200 x 1200 operator)."""
    import __graft_entry__ as g

    pos, q, alpha = synth.small_random(2024, 400, box=16.0, alpha_range=g.SMOKE_ALPHA)
    n = len(pos)
    r = pos[:, None, :] - pos[None, :, :]
    d = np.linalg.norm(r, axis=2)
    np.fill_diagonal(d, np.inf)
    T = (3 * r[:, :, :, None] * r[:, :, None, :] / d[:, :, None, None] ** 2 - np.eye(3)) / d[:, :, None, None] ** 3
    A = np.diag(np.repeat(1 / alpha, 3)) - T.transpose(0, 2, 1, 3).reshape(3 * n, 3 * n)
    assert np.linalg.eigvalsh(A)[0] > 0.1
