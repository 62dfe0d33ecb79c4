"""Host-side pieces of the dynamics driver on the CPU: the repulsive wall
against a brute-force pair sum and its own finite differences (torch on the
CPU), and the initial velocities' momentum and temperature."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
from paper_1408_6527_gb300 import md  # noqa: E402


def _brute(x, eps, sigma):
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


def test_repulsion_matches_the_brute_force_pair_sum():
    x = synth.workload(1).pos  # jittered lattice: nearest pairs from 1.9 A, inside the 2.3 A wall
    rep = md.Repulsion()
    U, F = rep(torch.as_tensor(x))
    Ub, Fb = _brute(x, rep.eps, rep.sigma)
    assert Ub > 0
    assert abs(U - Ub) <= 1e-12 * Ub
    assert np.abs(F.numpy() - Fb).max() <= 1e-10 * np.abs(Fb).max()


def test_repulsion_force_is_minus_its_gradient_on_cpu():
    x = synth.workload(1).pos
    rep = md.Repulsion()
    _, F = rep(torch.as_tensor(x))
    F = F.numpy()
    rng = np.random.default_rng(2)
    h = 1e-6
    for i in rng.choice(x.shape[0], 6, replace=False):
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, d] += h
            xm[i, d] -= h
            fd = -(rep(torch.as_tensor(xp))[0] - rep(torch.as_tensor(xm))[0]) / (2 * h)
            assert abs(fd - F[i, d]) <= 1e-6 * max(1.0, abs(F[i, d]))


def test_maxwell_velocities_have_no_net_momentum_and_the_target_temperature():
    masses = np.random.default_rng(5).uniform(1.0, 16.0, 20000)
    v = md.maxwell_velocities(masses, 300.0, seed=6)
    p = (masses[:, None] * v).sum(0)
    assert np.abs(p).max() < 1e-10 * np.abs(masses[:, None] * v).sum()
    ke = 0.5 * (masses[:, None] * v * v).sum() / md.ACC  # kcal/mol
    T = 2 * ke / (3 * masses.shape[0] * md.KB)
    assert abs(T - 300.0) < 6.0  # 3 N = 60,000 degrees of freedom: sd ~ 300 sqrt(2 / 3N) = 1.7 K
