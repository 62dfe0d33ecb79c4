"""The dipole solve on its own tree over the polarizable sites (T^mu, Sec. III;
polfmm_options.dipole_tree) against the oracle on the same two trees."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import polaris
from paper_1408_6527_gb300 import PolFMM

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)


def dev(a):
    return torch.as_tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy() if isinstance(t, torch.Tensor) else np.asarray(t)


def max_site_err(a, b):
    return float(np.max(oracle.per_site_rel_err(a, b)))


def _system(n, frac_pol, seed, box):
    """Random sites at 0.05-0.08 per cubic Angstrom, alpha in [0.3, 1.5] on a
    fraction of them (the solve converges in about 20-30 PCG iterations)."""
    pos, q, alpha = synth.small_random(seed, n, box=box, alpha_range=(0.3, 1.5))
    rng = np.random.default_rng(seed + 7)
    alpha = alpha.copy()
    off = rng.choice(n, n - int(round(frac_pol * n)), replace=False)
    alpha[off] = 0.0
    return pos, q, alpha


def dipole_tree_depth(n, m, depth):
    """The library's rule: the given depth less log8(n / m), rounded down."""
    r = n // m
    while r >= 8 and depth > 1:
        depth -= 1
        r //= 8
    return depth


def two_tree_reference(pos, q, alpha, p, depth, root, tol=1e-13):
    """The oracle on the same two trees: the field of the charges from the tree
    over all sites; the dipole solve with the dipole field of the tree over the
    polarizable sites (same root box, its own depth); the energy and gradients
    from the tree over all sites."""
    sel = alpha > 0
    m = int(sel.sum())
    st = oracle.fmm_fields(pos, q, None, p=p, depth=depth, root=root)
    Eq, phi_q = st["E"], st["phi"]
    dmu = dipole_tree_depth(len(q), m, depth)
    apply_T = lambda v: oracle.fmm_fields(pos[sel], None, v, p=p, depth=dmu, root=root)["E"]
    mu_s, it, res, _ = oracle.pcg_dipole_solve(alpha[sel], Eq[sel], apply_T, tol=tol, max_iter=500)
    mu = np.zeros_like(pos)
    mu[sel] = mu_s
    tot = oracle.fmm_fields(pos, q, mu, p=p, depth=depth, root=root)
    Uqq, Upol = oracle.energy_terms(q, alpha, mu, phi_q, Eq, tot["E"] - Eq)
    F, dUdq, dUda = oracle.gradients(q, alpha, mu, tot)
    return {"U": Uqq + Upol, "Upol": Upol, "mu": mu, "F": F, "dUdq": dUdq, "dUdalpha": dUda, "iterations": it,
            "depth_mu": dmu}


@pytest.mark.parametrize("frac_pol", [0.6, 0.1])
def test_dipole_tree_matches_the_oracle_on_the_same_trees(frac_pol):
    pos, q, alpha = _system(800, frac_pol, 61, 22.0)
    p, depth = 6, 3
    lo, side = oracle.root_box(pos)
    ref = two_tree_reference(pos, q, alpha, p, depth, (lo, side))
    if frac_pol < 0.125:
        assert ref["depth_mu"] == depth - 1  # the smaller tree is shallower
    with PolFMM(dev(pos), dev(q), dev(alpha), p=p, depth=depth, root_box=(lo, side), max_iter=500,
                dipole_tree=True) as f:
        info = f.solve(1e-13)
        out = f.energy_forces()
        mu = host(f.dipoles())
    assert info["converged"]
    assert np.all(mu[alpha == 0.0] == 0.0)
    sel = alpha > 0  # (the other sites carry no dipole on either side)
    assert oracle.rel_rms(mu, ref["mu"]) < 1e-9 and max_site_err(mu[sel], ref["mu"][sel]) < 1e-7
    assert out["U"] == pytest.approx(ref["U"], rel=1e-10)
    assert out["Upol"] == pytest.approx(ref["Upol"], rel=1e-9)
    for k in ("F", "dUdq", "dUdalpha"):
        assert oracle.rel_rms(host(out[k]), ref[k]) < 1e-9, k
        assert max_site_err(host(out[k]), ref[k]) < 1e-7, k


def test_dipole_tree_with_exclusions_and_thole_against_the_definition():
    """Exclusions (pairs of polarizable sites) and Thole damping reach the
    dipole tree. At depth 1 there is no far field, so both forms are the dense
    definition to round-off; at depth 3 the two-tree error against it is the
    octree's truncation error, of the same size as with one tree."""
    pos, q, alpha = _system(400, 0.5, 67, 18.0)
    d = np.linalg.norm(pos[:, None] - pos[None], axis=2)
    np.fill_diagonal(d, np.inf)
    excl = sorted({tuple(sorted((i, int(np.argmin(d[i]))))) for i in range(0, len(q), 3)})
    a = 0.39
    ref = polaris.polaris_energy(pos, q, q, alpha, excl, method="dense", solve="dense", thole=a)
    und = polaris.polaris_energy(pos, q, q, alpha, excl, method="dense", solve="dense")
    assert abs(ref["U"] - und["U"]) > 1e-4 * abs(und["U"])  # the damping matters here
    errs = {}
    for depth in (1, 3):
        for tree in (False, True):
            with PolFMM(dev(pos), dev(q), dev(alpha), p=8, depth=depth, max_iter=500, dipole_tree=tree) as f:
                f.set_exclusions(excl)
                f.set_thole(a)
                assert f.solve(1e-13)["converged"]
                out = f.energy_forces()
                errs[depth, tree] = (oracle.rel_rms(host(out["F"]), ref["F"]),
                                     oracle.rel_rms(host(f.dipoles()), ref["mu"]),
                                     abs(out["U"] - ref["U"]) / abs(ref["U"]))
    for k in range(3):
        assert errs[1, True][k] < 1e-9 and errs[1, False][k] < 1e-9, (k, errs)
        assert errs[3, True][k] < 1.5 * errs[3, False][k], (k, errs)


def test_dipole_tree_mixed_within_the_gate():
    w = synth.workload(2)
    alpha = w.alpha.copy()
    alpha[np.random.default_rng(5).random(w.n) < 0.5] = 0.0
    outs = {}
    # MIXED against FP64 on the same two trees (a different tree changes the truncation error)
    for mode in ("fp64", "mixed"):
        with PolFMM(dev(w.pos), dev(w.q), dev(alpha), p=w.p, depth=w.depth, mode=mode, dipole_tree=True) as f:
            assert f.solve(1e-8 if mode == "fp64" else 1e-7)["converged"]
            out = f.energy_forces()
            outs[mode] = (host(out["F"]), host(f.dipoles()), out["U"])
    assert oracle.rel_rms(outs["mixed"][0], outs["fp64"][0]) < 1e-5
    assert oracle.rel_rms(outs["mixed"][1], outs["fp64"][1]) < 1e-5
    assert outs["mixed"][2] == pytest.approx(outs["fp64"][2], rel=1e-6)


def test_dipole_tree_follows_positions_dipoles_and_the_predictor():
    """Along a path of positions (one root box for all of them), with the
    dipole predictor warm-starting each solve: every step equals the oracle on
    the same two trees. Set dipoles reach both trees."""
    pos, q, alpha = _system(600, 0.4, 71, 20.0)
    rng = np.random.default_rng(9)
    path = [pos + 0.03 * k * rng.normal(size=pos.shape) for k in range(1, 4)]
    lo, side = oracle.root_box(np.concatenate(path))
    lo, side = lo - 0.5, side + 1.0
    p, depth = 6, 3
    with PolFMM(dev(pos), dev(q), dev(alpha), p=p, depth=depth, root_box=(lo, side), max_iter=500,
                dipole_tree=True) as f:
        f.set_dipole_predictor(1)
        for x in path:
            f.update_positions(dev(x))
            assert f.solve(1e-12)["converged"]
            out = f.energy_forces()
            ref = two_tree_reference(x, q, alpha, p, depth, (lo, side))
            assert out["U"] == pytest.approx(ref["U"], rel=1e-9)
            assert oracle.rel_rms(host(f.dipoles()), ref["mu"]) < 1e-8
            assert oracle.rel_rms(host(out["F"]), ref["F"]) < 1e-8
        mu_set = 0.1 * rng.normal(size=pos.shape) * (alpha > 0)[:, None]
        f.set_dipoles(dev(mu_set))
        assert np.array_equal(host(f.dipoles()), mu_set)
        # a warm start from the set dipoles converges to the same solution
        assert f.solve(1e-12)["converged"]
        assert oracle.rel_rms(host(f.dipoles()), ref["mu"]) < 1e-8
        f.reset_dipoles()
        assert f.solve(1e-12)["converged"]
        assert oracle.rel_rms(host(f.dipoles()), ref["mu"]) < 1e-8


def test_dipole_tree_when_all_or_no_sites_are_polarizable():
    pos, q, alpha = _system(300, 1.0, 73, 16.0)
    out = {}
    for tree in (False, True):
        with PolFMM(dev(pos), dev(q), dev(alpha), p=6, depth=3, dipole_tree=tree) as f:
            info = f.solve(1e-10)
            out[tree] = (info["iterations"], host(f.dipoles()), f.energy_forces()["U"])
    # every site polarizable: the two trees coincide and one is used
    assert out[True][0] == out[False][0]
    assert np.array_equal(out[True][1], out[False][1]) and out[True][2] == out[False][2]
    with PolFMM(dev(pos), dev(q), dev(np.zeros_like(alpha)), p=6, depth=3, dipole_tree=True) as f:
        f.solve(1e-10)
        e = f.energy_forces()
        assert np.all(host(f.dipoles()) == 0.0)
        assert e["Upol"] == 0.0
