"""Dynamics on the polarizable FMM forces (the differentiation / MD
configuration): the library's wall against a brute-force pair sum and its own
finite differences, the kick / drift / kinetic kernels, velocity Verlet's
energy conservation, the multiple-time-step integrator with the FMM as the
slow force (Sec. IV.B: one inner step reproduces velocity Verlet bit for bit;
five inner steps per FMM evaluation), and the autograd gradients against
central finite differences, at a small size and at the 100k-site globule."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1408_6527_gb300 import md  # noqa: E402


def _system(n=3000, seed=7):
    w = synth.workload(4, n=n, depth=3)
    rng = np.random.default_rng(seed)
    masses = rng.uniform(1.0, 16.0, w.n)
    return w, masses, md.maxwell_velocities(masses, 300.0, seed + 1)


def _brute_wall(x, eps, sigma):
    """U = sum_{i<j, r < 2^(1/6) sigma} 4 eps [(s/r)^12 - (s/r)^6] + eps and F = -grad U."""
    rc = 2.0 ** (1.0 / 6.0) * sigma
    n = x.shape[0]
    U, F = 0.0, np.zeros_like(x)
    for i in range(n):
        r = x[i] - x[i + 1:]
        d = np.linalg.norm(r, axis=1)
        m = d < rc
        t6 = (sigma / d[m]) ** 6
        U += np.sum(4 * eps * (t6 * t6 - t6) + eps)
        f = (4 * eps * (12 * t6 * t6 - 6 * t6) / d[m] ** 2)[:, None] * r[m]
        F[i] += f.sum(0)
        F[i + 1:][m] -= f
    return U, F


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("which", ["lattice", "globule"])
def test_wall_matches_the_brute_force_pair_sum(which):
    # jittered lattice: nearest pairs from 1.9 A, inside the 2.3 A wall; the
    # globule's random sites give the long tail of close pairs
    x = synth.workload(1).pos if which == "lattice" else synth.workload(4, n=6000, depth=3).pos
    rep = md.Repulsion()
    U, F = rep(_dev(x))
    Ub, Fb = _brute_wall(x, rep.eps, rep.sigma)
    assert Ub > 0
    assert abs(float(U) - Ub) <= 1e-12 * Ub
    assert np.abs(F.cpu().numpy() - Fb).max() <= 1e-10 * np.abs(Fb).max()
    # bitwise reproducible
    U2, F2 = rep(_dev(x))
    assert float(U2) == float(U) and torch.equal(F2, F)


def test_wall_edge_cases():
    rep = md.Repulsion(capacity=8)
    U, F = rep(torch.zeros(0, 3, dtype=torch.float64, device="cuda"))
    assert float(U) == 0.0 and F.shape == (0, 3)
    U, F = rep(_dev([[0.3, -7.0, 2.0]]))
    assert float(U) == 0.0 and torch.all(F == 0)
    # one pair inside the wall: the pair formula; one just outside r_c: nothing
    r = 2.0
    U, F = rep(_dev([[0.0, 0.0, 0.0], [r, 0.0, 0.0], [40.0, 0.0, 0.0], [40.0 + 1.0001 * rep.rc, 0.0, 0.0]]))
    t6 = (rep.sigma / r) ** 6
    assert abs(float(U) - (4 * rep.eps * (t6 * t6 - t6) + rep.eps)) < 1e-12
    f = 4 * rep.eps * (12 * t6 * t6 - 6 * t6) / r
    Fh = F.cpu().numpy()
    assert abs(Fh[0, 0] + f) < 1e-12 * f and abs(Fh[1, 0] - f) < 1e-12 * f and np.all(Fh[2:] == 0)
    # more sites than the scratch was made for: it grows
    x = synth.workload(1).pos[:100]
    U, _ = rep(_dev(x))
    assert abs(float(U) - _brute_wall(x, rep.eps, rep.sigma)[0]) <= 1e-12 * max(1.0, float(U))
    # negative coordinates and cells far from the origin hash like any other
    U, _ = rep(_dev(x - 1.0e4))
    assert abs(float(U) - _brute_wall(x, rep.eps, rep.sigma)[0]) <= 1e-9 * max(1.0, float(U))


def test_wall_force_is_minus_gradient():
    rng = np.random.default_rng(1)
    x = synth.workload(1).pos
    rep = md.Repulsion()
    F = rep(_dev(x))[1].cpu().numpy()
    h = 1e-6
    for i in rng.choice(x.shape[0], 8, replace=False):
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, d] += h
            xm[i, d] -= h
            fd = -(float(rep(_dev(xp))[0]) - float(rep(_dev(xm))[0])) / (2 * h)
            assert abs(fd - F[i, d]) <= 1e-6 * max(1.0, abs(F[i, d])), (i, d, fd, F[i, d])


def test_kick_drift_and_kinetic_kernels():
    rng = np.random.default_rng(4)
    n = 5003
    x, v, F = (rng.standard_normal((n, 3)) for _ in range(3))
    m = rng.uniform(1.0, 16.0, n)
    ops = md.Repulsion(capacity=n)
    xd, vd, Fd, md_ = _dev(x), _dev(v), _dev(F), _dev(m)
    ops.kick(vd, Fd, md_, 0.37)
    v1 = v + 0.37 * F / m[:, None]
    assert np.abs(vd.cpu().numpy() - v1).max() <= 1e-15 * np.abs(v1).max()
    ops.drift(xd, vd, 0.5)
    x1 = x + 0.5 * v1
    assert np.abs(xd.cpu().numpy() - x1).max() <= 1e-15 * np.abs(x1).max()
    ke = float(ops.kinetic(vd, md_, 2.0))
    assert abs(ke - 2.0 * 0.5 * (m[:, None] * v1 * v1).sum()) <= 1e-13 * ke
    assert float(ops.kinetic(vd, md_, 2.0)) == ke  # fixed summation order


def test_velocity_verlet_conserves_energy_and_mixed_follows_fp64():
    w, masses, v0 = _system()
    H = {}
    ke0 = float(0.5 * (masses[:, None] * v0 * v0).sum() / md.ACC)
    for mode, tol in (("fp64", 1e-10), ("mixed", 1e-7)):
        # polarizabilities halved: undamped point dipoles at the full values reach
        # the polarization catastrophe within a few fs of motion
        dyn = md.Dynamics(w.pos, w.q, 0.5 * w.alpha, masses, p=w.p, depth=w.depth, mode=mode, tol=tol)
        Hm, _ = dyn.run(_dev(v0), 40, dt=0.5)
        dyn.close()
        assert np.all(np.isfinite(Hm))
        H[mode] = Hm
    # velocity Verlet at 0.5 fs: the total energy fluctuates by a small fraction
    # of the kinetic energy and does not run away
    assert np.abs(H["fp64"] - H["fp64"][0]).max() / ke0 < 1e-2
    # the MIXED trajectory stays on the FP64 one over the short run
    assert np.abs(H["mixed"] - H["fp64"]).max() / ke0 < 1e-4


@pytest.mark.parametrize("mode,tol", [("fp64", 1e-10), ("mixed", 1e-7)])
def test_one_inner_step_with_the_fmm_as_slow_force_is_velocity_verlet_bit_for_bit(mode, tol):
    w, masses, v0 = _system()
    out = []
    for multistep in (False, True):
        dyn = md.Dynamics(w.pos, w.q, 0.5 * w.alpha, masses, p=w.p, depth=w.depth, mode=mode, tol=tol)
        H, v = dyn.run(_dev(v0), 12, dt=0.5, inner=1, multistep=multistep)
        out.append((H, v.clone(), dyn.x.clone(), list(dyn.iterations)))
        dyn.close()
    (Ha, va, xa, ia), (Hb, vb, xb, ib) = out
    assert ia == ib
    assert np.array_equal(Ha, Hb) and torch.equal(va, vb) and torch.equal(xa, xb)


def test_five_inner_steps_per_fmm_evaluation():
    """Sec. IV.B's scheme: the long-range (FMM) forces every 5 inner steps.
    Over the same 25 fs, five inner steps of 0.5 fs per FMM evaluation keep the
    total energy as well as velocity Verlet at 0.5 fs does, with a fifth of the
    FMM evaluations."""
    w, masses, v0 = _system()
    ke0 = float(0.5 * (masses[:, None] * v0 * v0).sum() / md.ACC)
    res = {}
    for inner, steps in ((1, 50), (5, 10)):
        dyn = md.Dynamics(w.pos, w.q, 0.5 * w.alpha, masses, p=w.p, depth=w.depth, mode="fp64", tol=1e-10)
        H, _ = dyn.run(_dev(v0), steps, dt=0.5, inner=inner)
        res[inner] = (np.abs(H - H[0]).max() / ke0, (H[-1] - H[0]) / ke0, len(dyn.iterations))
        dyn.close()
        assert np.all(np.isfinite(H))
    print("max |H - H0| / KE0 and end drift / KE0: inner 1", res[1][:2], "inner 5", res[5][:2])
    assert res[5][2] == 1 + 10 and res[1][2] == 1 + 50
    assert res[1][0] < 1e-2
    assert res[5][0] < 2e-2


def test_autograd_matches_finite_differences_on_random_sites():
    w = synth.workload(4, n=2000, depth=3)
    worst = md.fd_check(w.pos, w.q, w.alpha, w.p, w.depth, sites=3, h=1e-5, tol=1e-12)
    assert worst["x"] < 1e-5, worst
    assert worst["q"] < 1e-5, worst
    assert worst["alpha"] < 1e-5, worst


def test_autograd_matches_finite_differences_at_the_100k_globule():
    """The differentiation configuration at its own size: 100,000 sites, p = 6,
    depth 5, 64 random sites (3 position, 1 charge and 1 polarizability
    derivative each, every one from two FP64 energy evaluations)."""
    w = synth.workload(4, n=100000)
    assert (w.n, w.p, w.depth) == (100000, 6, 5)
    worst = md.fd_check(w.pos, w.q, w.alpha, w.p, w.depth, sites=64, h=1e-5, tol=1e-11)
    print("100k FD check, max relative difference:", worst)
    assert worst["x"] < 1e-5, worst
    assert worst["q"] < 1e-5, worst
    assert worst["alpha"] < 1e-5, worst


def test_momentum_kernel():
    rng = np.random.default_rng(8)
    n = 3001
    v, m = rng.standard_normal((n, 3)), rng.uniform(1.0, 16.0, n)
    ops = md.Repulsion(capacity=n)
    P = ops.momentum(_dev(v), _dev(m)).cpu().numpy()
    ref = (m[:, None] * v).sum(0)
    assert np.abs(P - ref).max() <= 1e-12 * np.abs(m[:, None] * v).sum()


def test_linear_dipole_predictor_starts_from_the_extrapolation():
    w, masses, v0 = _system()
    from paper_1408_6527_gb300 import PolFMM

    x = _dev(w.pos)
    with PolFMM(x, _dev(w.q), _dev(0.5 * w.alpha), p=w.p, depth=w.depth, coulomb_k=md.COULOMB) as f:
        f.set_dipole_predictor(1)
        f.solve(1e-10)
        mus = [f.dipoles().cpu().numpy()]
        for k in range(2):
            x = x + 0.01 * _dev(v0)
            f.update_positions(x)
            start = f.dipoles().cpu().numpy()
            if k == 0:  # one update seen: the last dipoles
                np.testing.assert_array_equal(start, mus[-1])
            else:       # two: 2 mu(t) - mu(t - dt), bit for bit
                np.testing.assert_array_equal(start, 2.0 * mus[-1] - mus[-2])
            f.solve(1e-10)
            mus.append(f.dipoles().cpu().numpy())


def test_predictor_saves_iterations_and_momentum_is_conserved():
    w, masses, v0 = _system()
    res = {}
    for pred in (0, 1):
        dyn = md.Dynamics(w.pos, w.q, 0.5 * w.alpha, masses, p=w.p, depth=w.depth, mode="fp64", tol=1e-8,
                          predictor=pred)
        H, _ = dyn.run(_dev(v0), 30, dt=0.5, track_momentum=True)
        P = np.array(dyn.momenta)
        scale = (masses * np.linalg.norm(v0, axis=1)).sum()
        res[pred] = (float(np.mean(dyn.iterations[3:])), float(np.abs(P - P[0]).max() / scale),
                     float(np.abs(H - H[0]).max()))
        dyn.close()
    print("mean iterations (no predictor, linear predictor), momentum drift, energy excursion:", res)
    assert res[1][0] < res[0][0]
    assert res[0][1] < 1e-3 and res[1][1] < 1e-3
