"""GPU path against the CPU oracle, through the C ABI.

FP64 mode must reproduce the oracle's FMM at the same order and tree to
round-off: 1e-10 relative RMS over all sites and 1e-8 at the worst single site
(per-site error with a floor of 1 % of the typical magnitude, so that one
wrong leaf or tile row cannot hide in the norm; the arithmetic is the same
truncated expansion, only evaluated in a different order and normalisation).
MIXED mode must stay within 1e-5 relative RMS force error of FP64.  Integer
work (leaf cells, root cube) must match bit for bit.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1408_6527_gb300 import PolFMM, PolFMMError  # noqa: E402
from siteerr import max_site_err  # noqa: E402

FP64_TOL = 1e-10
FP64_SITE_TOL = 1e-8
MIXED_FORCE_TOL = 1e-5
MIXED_SITE_TOL = 1e-3
MIXED_ENERGY_TOL = 1e-6


def dev(a):
    return torch.as_tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy() if isinstance(t, torch.Tensor) else np.asarray(t)


@pytest.fixture(scope="module")
def w1():
    return synth.workload(1)


@pytest.fixture(scope="module")
def w2():
    return synth.workload(2)


# ---------------------------------------------------------------------------
# tree: integer work is bit-exact
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("depth", [1, 3, 5])
def test_root_box_and_leaf_cells_bit_exact(w1, depth):
    with PolFMM(dev(w1.pos), dev(w1.q), dev(w1.alpha), p=4, depth=depth) as f:
        lo, side = f.root_box()
        cells = host(f.leaf_cells())
    rlo, rside = oracle.root_box(w1.pos)
    assert side == rside and np.array_equal(lo, rlo)
    np.testing.assert_array_equal(cells, oracle.leaf_cells(w1.pos, depth, rlo, rside))


def test_tree_box_counts(w2):
    with PolFMM(dev(w2.pos), dev(w2.q), dev(w2.alpha), p=6, depth=4) as f:
        info = f.tree_info()
        lo, side = f.root_box()
    cells = oracle.leaf_cells(w2.pos, 4, lo, side)
    for l in range(5):
        c = cells >> (4 - l)
        assert info["boxes"][l] == len(np.unique(c[:, 0] + 64 * (c[:, 1] + 64 * c[:, 2])))


# ---------------------------------------------------------------------------
# single passes, FP64 against the oracle FMM (same p, same tree)
# ---------------------------------------------------------------------------

def _static_case(pos, q, alpha, p, depth):
    with PolFMM(dev(pos), dev(q), dev(alpha), p=p, depth=depth) as f:
        st = f.static_field()
        lo, side = f.root_box()
    ref = oracle.fmm_fields(pos, q, None, p=p, depth=depth, root=(lo, side))
    return st, ref


@pytest.mark.parametrize("p,depth", [(1, 2), (4, 3), (6, 3), (8, 2), (10, 3)])
def test_static_field_fp64(w1, p, depth):
    st, ref = _static_case(w1.pos, w1.q, w1.alpha, p, depth)
    assert oracle.rel_rms(host(st["E"]), ref["E"]) < FP64_TOL
    assert oracle.rel_rms(host(st["phi"]), ref["phi"]) < FP64_TOL
    assert max_site_err(host(st["E"]), ref["E"]) < FP64_SITE_TOL
    assert max_site_err(host(st["phi"]), ref["phi"]) < FP64_SITE_TOL


def test_static_field_fp64_ragged_small():
    # 37 sites: one partly filled tile, empty boxes, leaves with a single site
    pos, q, alpha = synth.small_random(31, 37, box=10.0)
    st, ref = _static_case(pos, q, alpha, 5, 4)
    assert oracle.rel_rms(host(st["E"]), ref["E"]) < FP64_TOL
    assert max_site_err(host(st["E"]), ref["E"]) < FP64_SITE_TOL
    assert max_site_err(host(st["phi"]), ref["phi"]) < FP64_SITE_TOL


def test_static_field_fp64_globule_full_size(w2):
    st, ref = _static_case(w2.pos, w2.q, w2.alpha, w2.p, w2.depth)
    assert oracle.rel_rms(host(st["E"]), ref["E"]) < FP64_TOL
    assert oracle.rel_rms(host(st["phi"]), ref["phi"]) < FP64_TOL
    assert max_site_err(host(st["E"]), ref["E"]) < FP64_SITE_TOL
    assert max_site_err(host(st["phi"]), ref["phi"]) < FP64_SITE_TOL


@pytest.mark.parametrize("p,depth", [(4, 3), (6, 4)])
def test_dipole_field_fp64(w1, p, depth):
    rng = np.random.default_rng(3)
    mu = rng.normal(size=(w1.n, 3))
    with PolFMM(dev(w1.pos), dev(w1.q), dev(w1.alpha), p=p, depth=depth) as f:
        E = host(f.dipole_field(dev(mu)))
        lo, side = f.root_box()
    ref = oracle.fmm_fields(w1.pos, None, mu, p=p, depth=depth, root=(lo, side))
    assert oracle.rel_rms(E, ref["E"]) < FP64_TOL
    assert max_site_err(E, ref["E"]) < FP64_SITE_TOL


def test_total_field_fp64(w1):
    rng = np.random.default_rng(4)
    mu = 0.3 * rng.normal(size=(w1.n, 3))
    with PolFMM(dev(w1.pos), dev(w1.q), dev(w1.alpha), p=5, depth=3) as f:
        out = f.total_field(dev(mu))
        lo, side = f.root_box()
    ref = oracle.fmm_fields(w1.pos, w1.q, mu, p=5, depth=3, root=(lo, side))
    for k in ("phi", "E", "G"):
        assert oracle.rel_rms(host(out[k]), ref[k]) < FP64_TOL, k
        assert max_site_err(host(out[k]), ref[k]) < FP64_SITE_TOL, k


def test_host_buffers_match_device_buffers(w1):
    with PolFMM(w1.pos, w1.q, w1.alpha, p=4, depth=3) as f:
        a = f.static_field()
    with PolFMM(dev(w1.pos), dev(w1.q), dev(w1.alpha), p=4, depth=3) as g:
        b = g.static_field()
    np.testing.assert_array_equal(a["E"], host(b["E"]))


# ---------------------------------------------------------------------------
# the solve and the energy / forces
# ---------------------------------------------------------------------------

def _oracle_fmm_apply(pos, p, depth, root):
    return lambda v: oracle.fmm_fields(pos, None, v, p=p, depth=depth, root=root)["E"]


@pytest.mark.parametrize("iters", [1, 5])
def test_fixed_iteration_pcg_fp64(w1, iters):
    with PolFMM(dev(w1.pos), dev(w1.q), dev(w1.alpha), p=4, depth=3, max_iter=iters) as f:
        info = f.solve(0.0)
        mu = host(f.dipoles())
        lo, side = f.root_box()
        Eq = host(f.static_field()["E"])
    assert info["iterations"] == iters and not info["converged"]
    ref_mu, it, res, _ = oracle.pcg_dipole_solve(w1.alpha, Eq, _oracle_fmm_apply(w1.pos, 4, 3, (lo, side)),
                                                 tol=0.0, max_iter=iters)
    assert it == iters
    assert oracle.rel_rms(mu, ref_mu) < 1e-9
    assert max_site_err(mu, ref_mu) < 1e-7
    assert info["residual"] == pytest.approx(res, rel=1e-6)


def test_converged_energy_forces_fp64(w1):
    with PolFMM(dev(w1.pos), dev(w1.q), dev(w1.alpha), p=4, depth=3) as f:
        info = f.solve(1e-12)
        f_energy = f.energy()
        out = f.energy_forces()
        mu = host(f.dipoles())
        lo, side = f.root_box()
    assert info["converged"]
    ref = oracle.polarizable_energy(w1.pos, w1.q, w1.alpha, method="fmm", p=4, depth=3, root=(lo, side),
                                    tol=1e-13)
    assert oracle.rel_rms(mu, ref["mu"]) < 1e-9
    assert f_energy["U"] == pytest.approx(ref["U"], rel=1e-10)
    assert out["U"] == pytest.approx(ref["U"], rel=1e-10)
    assert out["Uqq"] == pytest.approx(ref["Uqq"], rel=1e-10)
    assert out["Upol"] == pytest.approx(ref["Upol"], rel=1e-9)
    assert oracle.rel_rms(host(out["F"]), ref["F"]) < 1e-9
    assert oracle.rel_rms(host(out["dUdq"]), ref["dUdq"]) < 1e-9
    assert oracle.rel_rms(host(out["dUdalpha"]), ref["dUdalpha"]) < 1e-9
    for k in ("F", "dUdq", "dUdalpha"):
        assert max_site_err(host(out[k]), ref[k]) < 1e-7, k
    assert max_site_err(mu, ref["mu"]) < 1e-7


def test_against_direct_sum_and_dense_solve(w1):
    """Against the exact definition (direct sums + dense dipole solve) the error
    is the FMM truncation error, which falls with p."""
    ref = oracle.polarizable_energy(w1.pos, w1.q, w1.alpha, method="direct", solve="dense")
    errs = []
    for p in (4, 6, 8):
        with PolFMM(dev(w1.pos), dev(w1.q), dev(w1.alpha), p=p, depth=3) as f:
            f.solve(1e-12)
            out = f.energy_forces()
            lo, side = f.root_box()
        e_gpu = oracle.rel_rms(host(out["F"]), ref["F"])
        fmm = oracle.polarizable_energy(w1.pos, w1.q, w1.alpha, method="fmm", p=p, depth=3, root=(lo, side),
                                        tol=1e-13)
        # same truncation as the oracle's FMM
        assert e_gpu == pytest.approx(oracle.rel_rms(fmm["F"], ref["F"]), rel=1e-6)
        errs.append(e_gpu)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.5 * errs[0]


def test_mixed_vs_fp64_force_error(w2):
    outs = {}
    for mode in ("fp64", "mixed"):
        with PolFMM(dev(w2.pos), dev(w2.q), dev(w2.alpha), p=w2.p, depth=w2.depth, mode=mode) as f:
            info = f.solve(1e-8 if mode == "fp64" else 1e-7)
            outs[mode] = (f.energy_forces(), host(f.dipoles()), info)
    F64, Fmx = host(outs["fp64"][0]["F"]), host(outs["mixed"][0]["F"])
    assert oracle.rel_rms(Fmx, F64) < MIXED_FORCE_TOL
    assert oracle.rel_rms(outs["mixed"][1], outs["fp64"][1]) < 1e-5
    assert max_site_err(Fmx, F64) < MIXED_SITE_TOL
    assert max_site_err(outs["mixed"][1], outs["fp64"][1]) < MIXED_SITE_TOL
    # U = U^qq' + U^pol: a sum of ~1e4 terms of both signs per site in FP32 whose
    # total is about 1e-2 of the sum of magnitudes; the MIXED solve tolerance
    # (1e-7 here) adds an error of the same order to U^pol
    assert outs["mixed"][0]["U"] == pytest.approx(outs["fp64"][0]["U"], rel=MIXED_ENERGY_TOL)


def test_deterministic_repeat(w1):
    res = []
    for _ in range(2):
        with PolFMM(dev(w1.pos), dev(w1.q), dev(w1.alpha), p=4, depth=3, mode="mixed") as f:
            f.solve(1e-7)
            res.append(host(f.energy_forces()["F"]))
    np.testing.assert_array_equal(res[0], res[1])


# ---------------------------------------------------------------------------
# edge cases and errors
# ---------------------------------------------------------------------------

def test_single_site():
    with PolFMM(np.zeros((1, 3)), np.array([0.7]), np.array([1.0]), p=3, depth=2) as f:
        info = f.solve(1e-10)
        out = f.energy_forces()
    assert info["iterations"] == 0
    assert out["U"] == 0.0 and np.all(out["F"] == 0.0)


def test_two_sites_closed_form():
    # depth 1: the two sites lie in adjacent leaves and interact directly
    x = np.array([[0.0, 0.0, 0.0], [2.5, 0.0, 0.0]])
    Q, al = 0.8, 1.7
    with PolFMM(x, np.array([Q, 0.0]), np.array([0.0, al]), p=4, depth=1) as f:
        f.solve(1e-14)
        out = f.energy_forces()
        mu = f.dipoles()
    np.testing.assert_allclose(mu[1], [al * Q / 2.5**2, 0, 0], rtol=1e-12)
    assert out["Upol"] == pytest.approx(-al * Q * Q / (2 * 2.5**4), rel=1e-12)


def test_coincident_sites_status():
    x = np.array([[0.0, 0.0, 0.0], [1.0, 1.0, 1.0], [1.0, 1.0, 1.0]])
    with pytest.raises(PolFMMError) as e:
        PolFMM(x, np.array([1.0, -0.5, -0.5]), np.ones(3), p=3, depth=2)
    assert e.value.status == 2


def test_energy_before_solve_is_a_state_error(w1):
    with PolFMM(w1.pos, w1.q, w1.alpha, p=4, depth=3) as f:
        with pytest.raises(PolFMMError) as e:
            f.energy_forces()
    assert e.value.status == 6


def test_iteration_cap_reports_not_converged(w1):
    with PolFMM(w1.pos, w1.q, w1.alpha, p=4, depth=3, max_iter=1) as f:
        info = f.solve(1e-12)
        assert not info["converged"] and info["status"] == 3 and info["iterations"] == 1
        f.energy_forces()  # dipoles stay usable


def test_alpha_zero_sites_carry_no_dipole(w1):
    alpha = w1.alpha.copy()
    alpha[::3] = 0.0
    with PolFMM(dev(w1.pos), dev(w1.q), dev(alpha), p=4, depth=3) as f:
        f.solve(1e-12)
        mu = host(f.dipoles())
        out = f.energy_forces()
        lo, side = f.root_box()
    assert np.all(mu[::3] == 0.0)
    ref = oracle.polarizable_energy(w1.pos, w1.q, alpha, method="fmm", p=4, depth=3, root=(lo, side), tol=1e-13)
    assert oracle.rel_rms(host(out["F"]), ref["F"]) < 1e-9
    assert oracle.rel_rms(host(out["dUdalpha"]), ref["dUdalpha"]) < 1e-9
    assert max_site_err(host(out["F"]), ref["F"]) < 1e-7
    assert max_site_err(host(out["dUdalpha"]), ref["dUdalpha"]) < 1e-7


# ---------------------------------------------------------------------------
# tensor-core multipole-to-local (MIXED) against the SIMT kernel and FP64
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["small", "cube", "globule"])
def test_tensor_core_m2l_matches_simt(case, w1, w2):
    if case == "small":
        pos, q, alpha = synth.small_random(41, 300, box=14.0)
        p, depth = 5, 3
    elif case == "cube":
        pos, q, alpha, p, depth = w1.pos, w1.q, w1.alpha, 4, 3
    else:
        pos, q, alpha, p, depth = w2.pos, w2.q, w2.alpha, 6, 4
    rng = np.random.default_rng(5)
    mu = 0.3 * rng.normal(size=(len(q), 3))
    out = {}
    for impl in ("simt", "tensor"):
        with PolFMM(dev(pos), dev(q), dev(alpha), p=p, depth=depth, mode="mixed", m2l=impl) as f:
            out[impl] = (host(f.dipole_field(dev(mu))), host(f.static_field()["E"]))
    with PolFMM(dev(pos), dev(q), dev(alpha), p=p, depth=depth, mode="fp64") as f:
        ref = host(f.dipole_field(dev(mu)))
    # 3xTF32 products carry FP32-level accuracy: both MIXED kernels sit at FP32
    # round-off of FP64 (a few 1e-6 relative after ~1e4 accumulated terms)
    assert oracle.rel_rms(out["tensor"][0], ref) < 5e-6
    assert oracle.rel_rms(out["tensor"][0], out["simt"][0]) < 5e-6
    assert oracle.rel_rms(out["tensor"][1], out["simt"][1]) < 5e-6
    assert max_site_err(out["tensor"][0], ref) < 1e-4
    assert max_site_err(out["tensor"][1], out["simt"][1]) < 1e-4


# ---------------------------------------------------------------------------
# FP32 CUDA-core multipole-to-local (MIXED, p <= 6) against SIMT and FP64
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["p1", "p2", "p3", "small", "cube", "globule", "deep"])
def test_ffma_m2l_matches_simt(case, w1, w2):
    if case in ("p1", "p2", "p3"):
        pos, q, alpha = synth.small_random(43, 500, box=16.0)
        p, depth = int(case[1]), 3
    elif case == "small":
        pos, q, alpha = synth.small_random(41, 300, box=14.0)
        p, depth = 5, 3
    elif case == "cube":
        pos, q, alpha, p, depth = w1.pos, w1.q, w1.alpha, 4, 3
    elif case == "globule":
        pos, q, alpha, p, depth = w2.pos, w2.q, w2.alpha, 6, 4
    else:
        # depth 6: 8^l maps, empty boxes and groups that straddle levels
        pos, q, alpha = synth.small_random(47, 6000, box=60.0, d_min=1.2)
        p, depth = 6, 6
    rng = np.random.default_rng(7)
    mu = 0.3 * rng.normal(size=(len(q), 3))
    out = {}
    for impl in ("simt", "ffma", "auto"):
        with PolFMM(dev(pos), dev(q), dev(alpha), p=p, depth=depth, mode="mixed", m2l=impl) as f:
            out[impl] = (host(f.dipole_field(dev(mu))), host(f.static_field()["E"]), host(f.static_field()["phi"]))
    with PolFMM(dev(pos), dev(q), dev(alpha), p=p, depth=depth, mode="fp64") as f:
        ref = host(f.dipole_field(dev(mu)))
        ref_s = f.static_field()
        ref_e, ref_phi = host(ref_s["E"]), host(ref_s["phi"])
    # AUTO takes the CUDA-core kernel at p <= 6
    for a, b in zip(out["auto"], out["ffma"]):
        assert np.array_equal(a, b)
    # FP32 arithmetic throughout: within FP32 round-off of FP64
    assert oracle.rel_rms(out["ffma"][0], ref) < 5e-6
    assert oracle.rel_rms(out["ffma"][1], ref_e) < 5e-6
    assert oracle.rel_rms(out["ffma"][2], ref_phi) < 5e-6
    assert oracle.rel_rms(out["ffma"][0], out["simt"][0]) < 5e-6
    assert max_site_err(out["ffma"][0], ref) < 1e-4
    assert max_site_err(out["ffma"][1], ref_e) < 1e-4


def test_ffma_m2l_forces_within_gate(w2):
    outs = {}
    for mode, impl in (("fp64", "simt"), ("mixed", "ffma")):
        with PolFMM(dev(w2.pos), dev(w2.q), dev(w2.alpha), p=w2.p, depth=w2.depth, mode=mode, m2l=impl) as f:
            f.solve(1e-8 if mode == "fp64" else 1e-7)
            outs[mode] = host(f.energy_forces()["F"])
    assert oracle.rel_rms(outs["mixed"], outs["fp64"]) < MIXED_FORCE_TOL
    assert max_site_err(outs["mixed"], outs["fp64"]) < MIXED_SITE_TOL


def test_tensor_core_m2l_forces_within_gate(w2):
    outs = {}
    for mode, impl in (("fp64", "simt"), ("mixed", "tensor")):
        with PolFMM(dev(w2.pos), dev(w2.q), dev(w2.alpha), p=w2.p, depth=w2.depth, mode=mode, m2l=impl) as f:
            f.solve(1e-8 if mode == "fp64" else 1e-7)
            outs[mode] = host(f.energy_forces()["F"])
    assert oracle.rel_rms(outs["mixed"], outs["fp64"]) < MIXED_FORCE_TOL
    assert max_site_err(outs["mixed"], outs["fp64"]) < MIXED_SITE_TOL


def test_programmatic_launch_matches_stream_order(w2):
    """The solver iteration's kernels with programmatic dependent launch (each
    waits for its predecessor's completion before reading its output) give
    bit-for-bit the same dipoles, energy and forces as plain stream order."""
    res = {}
    for pdl in (True, False):
        with PolFMM(dev(w2.pos), dev(w2.q), dev(w2.alpha), p=w2.p, depth=w2.depth, mode="mixed", pdl=pdl) as f:
            info = f.solve(1e-6)
            out = f.energy_forces()
            res[pdl] = (info["iterations"], host(f.dipoles()), float(out["U"]), host(out["F"]))
    assert res[True][0] == res[False][0]
    assert np.array_equal(res[True][1], res[False][1])
    assert res[True][2] == res[False][2]
    assert np.array_equal(res[True][3], res[False][3])


def test_graph_replay_matches_direct_launches(w1):
    res = {}
    for graphs in (True, False):
        with PolFMM(dev(w1.pos), dev(w1.q), dev(w1.alpha), p=4, depth=3, mode="mixed", graphs=graphs) as f:
            info = f.solve(1e-7)
            res[graphs] = (info["iterations"], host(f.dipoles()), host(f.energy_forces()["F"]))
            # a new tree re-captures (or updates) the graph
            f.update_positions(dev(w1.pos * 1.01))
            f.reset_dipoles()
            f.solve(1e-7)
            res[graphs] += (host(f.dipoles()),)
    assert res[True][0] == res[False][0]
    for k in (1, 2, 3):
        np.testing.assert_array_equal(res[True][k], res[False][k])
