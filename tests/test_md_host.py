"""Host-side logic of the dynamics driver on the CPU: the step sequencing of
velocity Verlet and of the multiple-time-step integrator (Sec. IV.B), driven
through Dynamics with torch stand-ins for the library's kicks, drifts and
wall and an analytic stand-in for the FMM context; and the initial
velocities' momentum and temperature."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
from paper_1408_6527_gb300 import md  # noqa: E402


class _TorchOps:
    """Kick, drift and kinetic energy written out in torch, with the fast force
    of a given potential (the wall's role in Dynamics)."""

    def __init__(self, fast_u):
        self.fast_u, self.wall_calls = fast_u, 0

    def wall(self, x):
        self.wall_calls += 1
        xr = x.clone().requires_grad_(True)
        u = self.fast_u(xr)
        (g,) = torch.autograd.grad(u, xr)
        return u.detach(), -g

    def kick(self, v, F, m, coef):
        v.add_(coef * F / m[:, None])

    def drift(self, x, v, dt):
        x.add_(dt * v)

    def kinetic(self, v, m, scale):
        return scale * 0.5 * (m[:, None] * v * v).sum()


class _TrapFMM:
    """Stands in for the FMM context: the slow force of a harmonic trap, with
    the context's update / solve / energy_forces calls."""

    def __init__(self, k):
        self.k, self.x, self.updates = k, None, 0

    def update_positions(self, x):
        self.x = x.clone()
        self.updates += 1

    def solve(self, tol):
        return {"iterations": 1}

    def energy_forces(self, forces=True, dq=False, dalpha=False):
        return {"U": float(0.5 * self.k * (self.x * self.x).sum()), "F": -self.k * self.x}


def _chain(n=16, seed=0):
    """Stiff springs along a chain (fast) in a weak harmonic trap (slow)."""
    g = torch.Generator().manual_seed(seed)
    x0 = torch.randn(n, 3, dtype=torch.float64, generator=g) * 3
    v0 = torch.randn(n, 3, dtype=torch.float64, generator=g) * 0.3
    L0 = torch.linalg.norm(x0[1:] - x0[:-1], dim=1)

    def fast_u(x):
        d = torch.linalg.norm(x[1:] - x[:-1], dim=1)
        return 0.5 * ((d - L0) ** 2).sum()

    return x0, v0, fast_u, 0.0025


def _dynamics(x0, m, fast_u, k):
    """Dynamics without a GPU: masses in units where a force over a mass of ACC
    is an acceleration of 1 (the chain's own units)."""
    dyn = md.Dynamics.__new__(md.Dynamics)
    dyn.x, dyn.m, dyn.tol, dyn.iterations = x0.clone(), m, 1e-8, []
    dyn.ops, dyn.fmm = _TorchOps(fast_u), _TrapFMM(k)
    dyn.fmm.update_positions(dyn.x)
    dyn.start()
    return dyn


def _plain_verlet(x0, v0, fast_u, k, dt, steps):
    """Velocity Verlet on the summed force, written out."""
    def acc(x):
        xr = x.clone().requires_grad_(True)
        (g,) = torch.autograd.grad(fast_u(xr), xr)
        return -g - k * x
    x, v = x0.clone(), v0.clone()
    a = acc(x)
    for _ in range(steps):
        v = v + 0.5 * dt * a
        x = x + dt * v
        a = acc(x)
        v = v + 0.5 * dt * a
    return x, v


def test_one_inner_step_gives_velocity_verlet_bit_for_bit():
    x0, v0, fast_u, k = _chain()
    m = torch.full((x0.shape[0],), md.ACC, dtype=torch.float64)
    a = _dynamics(x0, m, fast_u, k)
    Ha, va = a.run(v0, 50, dt=0.05, inner=1)
    b = _dynamics(x0, m, fast_u, k)
    Hb, vb = b.run(v0, 50, dt=0.05, inner=1, multistep=True)
    assert torch.equal(a.x, b.x) and torch.equal(va, vb) and np.array_equal(Ha, Hb)
    # and it is velocity Verlet on the summed force (up to the rounding of the split kicks)
    xv, vv = _plain_verlet(x0, v0, fast_u, k, 0.05, 50)
    assert torch.abs(a.x - xv).max() < 1e-11 and torch.abs(va - vv).max() < 1e-11


def test_multiple_time_steps_are_time_reversible():
    x0, v0, fast_u, k = _chain()
    m = torch.full((x0.shape[0],), md.ACC, dtype=torch.float64)
    d = _dynamics(x0, m, fast_u, k)
    _, v = d.run(v0, 100, dt=0.05, inner=10)
    _, v = d.run(-v, 100, dt=0.05, inner=10)
    assert torch.abs(d.x - x0).max() < 1e-9 and torch.abs(v + v0).max() < 1e-9


def test_multiple_time_steps_are_stable_where_verlet_at_the_outer_step_is_not():
    """The point of multiple time steps: the slow force at a step (1.5) past
    the stability limit of the fast springs, which are integrated at 0.05."""
    x0, v0, fast_u, k = _chain()
    m = torch.full((x0.shape[0],), md.ACC, dtype=torch.float64)
    d = _dynamics(x0, m, fast_u, k)
    H, _ = d.run(v0, 400, dt=0.05, inner=30)
    assert np.abs(H - H[0]).max() < 1e-2 * H[0]
    xv, vv = _plain_verlet(x0, v0, fast_u, k, 1.5, 400)
    Hv = float(0.5 * (vv * vv).sum() + fast_u(xv) + 0.5 * k * (xv * xv).sum())
    assert not np.isfinite(Hv) or abs(Hv - H[0]) > 1.0 * H[0]


def test_each_outer_step_evaluates_the_slow_force_once_and_the_wall_every_inner_step():
    x0, v0, fast_u, k = _chain()
    m = torch.full((x0.shape[0],), md.ACC, dtype=torch.float64)
    d = _dynamics(x0, m, fast_u, k)
    d.run(v0, 7, dt=0.05, inner=4)
    assert d.fmm.updates == 1 + 7      # the set-up, then one per outer step
    assert len(d.iterations) == 1 + 7  # one dipole solve per slow force
    assert d.ops.wall_calls == 1 + 7 * 4


def test_maxwell_velocities_have_no_net_momentum_and_the_target_temperature():
    masses = np.random.default_rng(5).uniform(1.0, 16.0, 20000)
    v = md.maxwell_velocities(masses, 300.0, seed=6)
    p = (masses[:, None] * v).sum(0)
    assert np.abs(p).max() < 1e-10 * np.abs(masses[:, None] * v).sum()
    ke = 0.5 * (masses[:, None] * v * v).sum() / md.ACC  # kcal/mol
    T = 2 * ke / (3 * masses.shape[0] * md.KB)
    assert abs(T - 300.0) < 6.0  # 3 N = 60,000 degrees of freedom: sd ~ 300 sqrt(2 / 3N) = 1.7 K


def test_the_wall_and_the_integrator_have_no_cpu_path():
    """The wall, kicks and drifts run in the library's kernels only."""
    if torch.cuda.is_available():  # pragma: no cover
        pytest.skip("a GPU is present")
    with pytest.raises(Exception):
        md.Repulsion(capacity=16)(torch.zeros(16, 3, dtype=torch.float64))
