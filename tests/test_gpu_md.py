"""Dynamics on the polarizable FMM forces (the differentiation / MD
configuration, small sizes): the repulsive wall's forces are its energy's
gradient, velocity Verlet conserves the total energy, MIXED follows FP64, and
the autograd gradients match central finite differences."""
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


def test_repulsion_force_is_minus_gradient():
    rng = np.random.default_rng(1)
    x = synth.workload(1).pos  # lattice sites, pairs from 1.9 A up
    rep = md.Repulsion()
    xt = torch.as_tensor(x, device="cuda")
    U0, F = rep(xt)
    assert U0 > 0
    F = F.cpu().numpy()
    h = 1e-6
    for i in rng.choice(x.shape[0], 8, replace=False):
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, d] += h
            xm[i, d] -= h
            fd = -(rep(torch.as_tensor(xp, device="cuda"))[0] - rep(torch.as_tensor(xm, device="cuda"))[0]) / (2 * h)
            assert abs(fd - F[i, d]) <= 1e-6 * max(1.0, abs(F[i, d])), (i, d, fd, F[i, d])


def test_velocity_verlet_conserves_energy_and_mixed_follows_fp64():
    w, masses, v0 = _system()
    H = {}
    ke0 = float(0.5 * (masses[:, None] * v0 * v0).sum() / md.ACC)
    for mode, tol in (("fp64", 1e-10), ("mixed", 1e-7)):
        # polarizabilities halved: undamped point dipoles at the full values reach
        # the polarization catastrophe within a few fs of motion
        dyn = md.Dynamics(w.pos, w.q, 0.5 * w.alpha, masses, p=w.p, depth=w.depth, mode=mode, tol=tol)
        Hm, _ = dyn.run(torch.as_tensor(v0, device="cuda"), 40, dt=0.5)
        dyn.close()
        assert np.all(np.isfinite(Hm))
        H[mode] = Hm
    # velocity Verlet at 0.5 fs: the total energy fluctuates by a small fraction
    # of the kinetic energy and does not run away
    assert np.abs(H["fp64"] - H["fp64"][0]).max() / ke0 < 1e-2
    # the MIXED trajectory stays on the FP64 one over the short run
    assert np.abs(H["mixed"] - H["fp64"]).max() / ke0 < 1e-4


def test_autograd_matches_finite_differences_on_random_sites():
    w = synth.workload(4, n=2000, depth=3)
    worst = md.fd_check(w.pos, w.q, w.alpha, w.p, w.depth, sites=3, h=1e-5, tol=1e-12)
    assert worst["x"] < 1e-5, worst
    assert worst["q"] < 1e-5, worst
    assert worst["alpha"] < 1e-5, worst
