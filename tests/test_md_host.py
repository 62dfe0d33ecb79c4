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


def _chain(n=16, seed=0):
    """Stiff springs along a chain (fast) in a weak harmonic trap (slow), unit masses."""
    g = torch.Generator().manual_seed(seed)
    x0 = torch.randn(n, 3, dtype=torch.float64, generator=g) * 3
    v0 = torch.randn(n, 3, dtype=torch.float64, generator=g) * 0.3
    L0 = torch.linalg.norm(x0[1:] - x0[:-1], dim=1)

    def fast_u(x):
        d = torch.linalg.norm(x[1:] - x[:-1], dim=1)
        return 0.5 * ((d - L0) ** 2).sum()

    def slow_u(x):
        return 0.5 * 0.0025 * (x * x).sum()

    def acc(u):
        def f(x):
            x = x.clone().requires_grad_(True)
            (g_,) = torch.autograd.grad(u(x), x)
            return -g_.detach()
        return f

    return x0, v0, acc(slow_u), acc(fast_u), lambda x, v: float(0.5 * (v * v).sum() + fast_u(x) + slow_u(x))


def test_respa_with_one_inner_step_is_velocity_verlet():
    x0, v0, slow, fast, _ = _chain()
    x, v, a_s, a_f = x0, v0, slow(x0), fast(x0)
    xv, vv = x0, v0
    a = slow(xv) + fast(xv)
    for _ in range(50):
        x, v, a_s, a_f = md.respa(x, v, a_s, a_f, slow, fast, 0.05, 1)
        vv = vv + 0.025 * a
        xv = xv + 0.05 * vv
        a = slow(xv) + fast(xv)
        vv = vv + 0.025 * a
    assert torch.abs(x - xv).max() < 1e-12 and torch.abs(v - vv).max() < 1e-12


def test_respa_is_time_reversible():
    x0, v0, slow, fast, _ = _chain()
    x, v, a_s, a_f = x0, v0, slow(x0), fast(x0)
    for _ in range(100):
        x, v, a_s, a_f = md.respa(x, v, a_s, a_f, slow, fast, 0.05, 10)
    v = -v
    for _ in range(100):
        x, v, a_s, a_f = md.respa(x, v, a_s, a_f, slow, fast, 0.05, 10)
    assert torch.abs(x - x0).max() < 1e-9 and torch.abs(v + v0).max() < 1e-9


def test_respa_is_stable_where_verlet_at_the_outer_step_is_not():
    """The point of multiple time steps: the slow force at a step (1.5) past
    the stability limit of the fast springs, which are integrated at 0.05."""
    x0, v0, slow, fast, energy = _chain()
    H0 = energy(x0, v0)
    x, v, a_s, a_f = x0, v0, slow(x0), fast(x0)
    dev = 0.0
    for _ in range(400):
        x, v, a_s, a_f = md.respa(x, v, a_s, a_f, slow, fast, 0.05, 30)
        dev = max(dev, abs(energy(x, v) - H0))
    assert dev < 1e-2 * H0
    xv, vv = x0, v0
    a = slow(xv) + fast(xv)
    for _ in range(400):
        vv = vv + 0.75 * a
        xv = xv + 1.5 * vv
        a = slow(xv) + fast(xv)
        vv = vv + 0.75 * a
    Hv = energy(xv, vv)
    assert not np.isfinite(Hv) or abs(Hv - H0) > 1.0 * H0


class _TrapFMM:
    """Stands in for the FMM context: an analytic slow force (a harmonic trap)
    with the context's update / solve / energy_forces calls."""

    def __init__(self, k=0.3):
        self.k, self.x = k, None

    def update_positions(self, x):
        self.x = x

    def solve(self, tol):
        return {"iterations": 1}

    def energy_forces(self, forces=True, dq=False, dalpha=False):
        return {"U": float(0.5 * self.k * (self.x * self.x).sum()), "F": -self.k * self.x}


def test_dynamics_multiple_time_steps_drive_the_slow_and_fast_forces():
    x0 = torch.as_tensor(synth.workload(1).pos)
    x0 = x0 - x0.mean(0)
    n = x0.shape[0]
    m = torch.full((n,), 12.0, dtype=torch.float64)
    v0 = torch.as_tensor(md.maxwell_velocities(m.numpy(), 300.0, 3))
    dyn = md.Dynamics.__new__(md.Dynamics)
    dyn.x, dyn.m, dyn.tol, dyn.iterations = x0.clone(), m, 1e-8, []
    dyn.rep, dyn.fmm = md.Repulsion(), _TrapFMM()
    dyn.fmm.update_positions(dyn.x)
    u_s = dyn.fmm.energy_forces()
    u_r, f_r = dyn.rep(dyn.x)
    dyn.U, dyn.F = u_s["U"] + u_r, u_s["F"] + f_r
    H, v = dyn.run(v0.clone(), 20, dt=0.5, inner=4)
    # the same steps through the integrator itself
    inv_m = md.ACC / m[:, None]
    slow = lambda x: -0.3 * x * inv_m
    fast = lambda x: md.Repulsion()(x)[1] * inv_m
    x, vv, a_s, a_f = x0.clone(), v0.clone(), slow(x0), fast(x0)
    for _ in range(20):
        x, vv, a_s, a_f = md.respa(x, vv, a_s, a_f, slow, fast, 0.5, 4)
    assert torch.abs(dyn.x - x).max() < 1e-12 and torch.abs(v - vv).max() < 1e-12
    assert len(dyn.iterations) == 20  # one slow solve per outer step
    ke = 0.5 * (m[:, None] * v * v).sum() / md.ACC
    assert abs(H[-1] - (float(ke) + 0.5 * 0.3 * float((x * x).sum()) + md.Repulsion()(x)[0])) < 1e-9 * abs(H[-1])
    assert np.abs(H - H[0]).max() < 1e-2 * float(0.5 * (m[:, None] * v0 * v0).sum() / md.ACC)
