"""Pins of the kd-tree FMM oracle (Sec. III): tree invariants and pair coverage
by brute force, the direct-sum limit theta -> 0, error decay with p, momentum
conservation of the mutual walk, and the paper's own sphere-test accuracy."""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import kdtree

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _sphere(seed, n, radius):
    rng = _rng(seed)
    pos = synth.sites_sphere(rng, n, radius, 2.0)
    return pos, synth.charges_pm_equal(rng, pos.shape[0])


def test_tree_partitions_the_particles_and_splits_at_the_centre():
    pos, _ = _sphere(3, 700, 25.0)
    root = kdtree.build_tree(pos, n_bucket=8)
    seen = np.zeros(pos.shape[0], dtype=int)
    for c in kdtree.cells(root):
        pts = pos[c.idx]
        assert np.allclose(c.z, pts.mean(axis=0))
        # r_enc encloses every particle of the cell
        assert np.max(np.linalg.norm(pts - c.z, axis=1)) <= c.r_enc + 1e-12
        if c.leaf:
            assert 1 <= c.n <= 8
            seen[c.idx] += 1
            continue
        l, r = c.children
        assert sorted(np.concatenate([l.idx, r.idx]).tolist()) == sorted(c.idx.tolist())
        # split across the longest dimension of the cell's box at the centre
        d = int(np.argmax(pts.max(axis=0) - pts.min(axis=0)))
        cut = pts[:, d].mean()
        assert np.all(pos[l.idx, d] < cut) and np.all(pos[r.idx, d] >= cut)
    assert np.all(seen == 1)


@pytest.mark.parametrize("theta,n_direct,n,radius", [(0.9, 8, 500, 24.0), (0.5, 64, 2000, 36.0)])
def test_walk_covers_every_pair_exactly_once(theta, n_direct, n, radius):
    pos, _ = _sphere(4, n, radius)
    root = kdtree.build_tree(pos)
    direct, multipole = kdtree.walk(root, theta, n_direct)
    assert multipole, "the case must exercise the multipole branch"
    count = np.zeros((n, n), dtype=np.int16)
    for a, b in direct:
        if a is b:
            count[np.ix_(a.idx, a.idx)] += 1
            continue
        count[np.ix_(a.idx, b.idx)] += 1
        count[np.ix_(b.idx, a.idx)] += 1
    for a, b in multipole:
        assert a is not b
        assert theta * np.linalg.norm(a.z - b.z) > a.r_enc + b.r_enc  # Eq. mac
        count[np.ix_(a.idx, b.idx)] += 1
        count[np.ix_(b.idx, a.idx)] += 1
    # every site meets itself once, in the one self pair that is summed directly
    assert np.all(count.diagonal() == 1)
    np.fill_diagonal(count, 1)
    assert np.all(count == 1)


def test_theta_zero_is_the_direct_sum():
    pos, q = _sphere(5, 400, 20.0)
    mu = _rng(6).normal(0.0, 0.1, pos.shape)
    f = kdtree.kdtree_fields(pos, q, mu, p=4, theta=0.0)
    d = oracle.direct_fields(pos, q, mu)
    for k in ("phi", "E", "G"):
        assert oracle.rel_rms(f[k], d[k]) < 1e-13


def test_error_decays_with_order_for_charges_and_dipoles():
    pos, q = _sphere(7, 1500, 33.0)
    mu = _rng(8).normal(0.0, 0.1, pos.shape)
    d = oracle.direct_fields(pos, q, mu)
    errs = [oracle.rel_rms(kdtree.kdtree_fields(pos, q, mu, p=p, theta=0.7)["E"], d["E"]) for p in (2, 4, 6)]
    assert errs[0] > 3 * errs[1] > 9 * errs[2]
    assert errs[2] < 5e-4


def test_mutual_walk_conserves_momentum():
    """Sec. III accumulates the field tensors of both nodes of a multipole pair,
    'ensuring conservation of momentum': sum_i q_i E_i vanishes to rounding,
    far below the truncation error of the forces themselves."""
    pos, q = _sphere(9, 1500, 33.0)
    f = kdtree.kdtree_fields(pos, q, p=4, theta=0.7)
    F = q[:, None] * f["E"]
    d = q[:, None] * oracle.direct_fields(pos, q)["E"]
    assert np.linalg.norm(F.sum(axis=0)) / np.abs(F).sum() < 1e-14
    assert oracle.rel_rms(F, d) > 1e-6  # the forces themselves carry truncation error


def test_sphere_test_matches_the_paper():
    """Sec. IV.A: 4096 sites of +-e in a 45 A ball, 2 A apart, kd-tree with
    theta = 0.5 and p = 5. The paper prints ~80 % of the per-atom relative
    force errors below 1e-4 and all below 1e-2 (tests/golden)."""
    g = json.load(open(os.path.join(GOLDEN, "paper_sphere_test.json")))
    pos, q = _sphere(16, g["n_sites"], g["radius_A"])
    f = kdtree.kdtree_fields(pos, q, p=g["order_p"], theta=g["theta"])
    d = oracle.direct_fields(pos, q)
    e = oracle.per_site_rel_err(q[:, None] * f["E"], q[:, None] * d["E"])
    assert (e < 1e-4).mean() >= g["fraction_below_1e-4"]
    assert e.max() < g["max_rel_force_error"]


def _sphere_with_dipoles():
    g = json.load(open(os.path.join(GOLDEN, "paper_sphere_test.json")))
    pos, q = _sphere(16, g["n_sites"], g["radius_A"])
    mu = _rng(17).normal(0.0, 0.2, pos.shape)
    return g, pos, q, mu


def test_dipole_pairs_approach_the_analytic_multipole_as_dl_squared():
    """Sec. II.C: a dipole is the +-q pair with mu = 2 q_mu dl; its multipoles
    differ from the point dipole's by O(dl^2)."""
    g, pos, q, mu = _sphere_with_dipoles()
    a = kdtree.kdtree_fields(pos, q, mu, p=g["order_p"], theta=g["theta"])
    diff = [oracle.rel_rms(kdtree.kdtree_fields(pos, q, mu, p=g["order_p"], theta=g["theta"], dipole_dl=dl)["E"],
                           a["E"]) for dl in (1e-1, 1e-2)]
    assert 98.0 < diff[0] / diff[1] < 102.0


def test_dipole_pair_separation_leaves_the_error_distribution_unchanged():
    """Sec. IV.A, Fig. pol-radius: over dl = 1e-5 ... 1e-1 A the paper finds no
    difference in the force errors at theta = 0.5."""
    g, pos, q, mu = _sphere_with_dipoles()
    d = oracle.direct_fields(pos, q, mu)

    def dist(dl):
        f = kdtree.kdtree_fields(pos, q, mu, p=g["order_p"], theta=g["theta"], dipole_dl=dl)
        e = oracle.per_site_rel_err(f["E"], d["E"])
        return np.percentile(e, 80), (e < 1e-4).mean()

    p80, frac = dist(0.0)
    for dl in (1e-5, 1e-3, 1e-1):
        p80_dl, frac_dl = dist(dl)
        assert abs(p80_dl - p80) < 1e-3 * p80
        assert abs(frac_dl - frac) < 1e-3


def test_polarized_sphere_test_keeps_the_error_distribution():
    """Sec. IV.A, Fig. pol-test: with polarization enabled (alpha = 1 A^3 on all
    atoms, field charges q^E = +-e drawn separately) at theta = 0.5 the paper
    finds no significant change in the force errors. Forces F = q E^coul +
    q^E E^mu + (grad E^qE + grad E^mu) mu, the kd-tree FMM against direct sums,
    each solved by PCG to 1e-10 with its own operator."""
    g = json.load(open(os.path.join(GOLDEN, "paper_sphere_test.json")))
    pos, q = _sphere(16, g["n_sites"], g["radius_A"])
    qE = synth.charges_pm_equal(_rng(61), pos.shape[0])
    n = pos.shape[0]
    alpha = np.ones(n)

    def gmu(G, mu):
        return np.stack([G[:, 0] * mu[:, 0] + G[:, 1] * mu[:, 1] + G[:, 2] * mu[:, 2],
                         G[:, 1] * mu[:, 0] + G[:, 3] * mu[:, 1] + G[:, 4] * mu[:, 2],
                         G[:, 2] * mu[:, 0] + G[:, 4] * mu[:, 1] + G[:, 5] * mu[:, 2]], 1)

    def forces(field):
        st = field(qE, None)
        mu = oracle.pcg_dipole_solve(alpha, st["E"], lambda v: field(None, v)["E"], tol=1e-10, max_iter=200)[0]
        dm = field(None, mu)
        return q[:, None] * field(q, None)["E"] + qE[:, None] * dm["E"] + gmu(st["G"] + dm["G"], mu)

    Fd = forces(lambda qq, mm: oracle.direct_fields(pos, qq, mm))
    Fk = forces(lambda qq, mm: kdtree.kdtree_fields(pos, qq, mm, p=g["order_p"], theta=g["theta"]))
    e = oracle.per_site_rel_err(Fk, Fd)
    assert (e < 1e-4).mean() >= g["fraction_below_1e-4"]
    assert e.max() < g["max_rel_force_error"]
