"""Velocity-Verlet and multiple-time-step dynamics on the polarizable FMM
forces, and the finite-difference check of the gradients (the differentiation / MD configuration).

Units: positions in Angstrom, charges in e, polarizabilities in Angstrom^3,
masses in amu, time in fs, energies in kcal/mol (Coulomb constant
332.0637 kcal Angstrom / (mol e^2)).  One step (Sec. III, stages 1-3 per step):
tree rebuild and static pass at the new positions, the dipole solve started
from the previous step's dipoles (a warm start), the force pass.

Point dipoles without Thole damping collapse onto each other (the
polarization catastrophe, r below (4 alpha_i alpha_j)^(1/6), 1.7 A at the
largest polarizabilities), and a pure Coulomb system of light opposite charges
collapses within some tens of fs.  The paper's force field has short-range
repulsion that is out of scope here, so the dynamics adds a purely repulsive
wall (the repulsive part of a Lennard-Jones pair, shifted to zero at its
minimum): U = 4 eps [(sigma/r)^12 - (sigma/r)^6] + eps for r < 2^(1/6) sigma,
eps = 5 kcal/mol, sigma = 2.05 A (zero beyond 2.30 A), evaluated in FP64 by
the library's own kernels from a spatial hash of cells (it is not part of the
FMM path); kicks, drifts and the kinetic energy are library kernels too.
Even so, undamped point dipoles with alpha up to 2.5 A^3 at 0.1 sites/A^3 are
collectively near the catastrophe (largest eigenvalue of alpha^1/2 T alpha^1/2
0.84 on the lattice) and a few fs of motion push them over it; the dynamics
therefore runs with the polarizabilities scaled by --alpha-scale (default 0.5),
while the finite-difference check uses them as they are.

    python -m paper_1408_6527_gb300.md --sites 100000 --steps 1000
"""
from __future__ import annotations

import argparse
import ctypes
import json
import time

import numpy as np

COULOMB = 332.0637          # kcal Angstrom / (mol e^2)
ACC = 4.184e-4              # Angstrom / fs^2 per (kcal / mol / Angstrom / amu)
KB = 0.0019872              # kcal / (mol K)


class Repulsion:
    """The purely repulsive wall between pairs closer than 2^(1/6) sigma, and
    the kicks, drifts and kinetic energy of the integrators, in the library's
    CUDA kernels (FP64; fmm_wall_forces, fmm_md_kick, fmm_md_drift,
    fmm_md_kinetic).  Scratch for up to `capacity` sites, grown on demand; the
    kernels run on the stream current at creation."""

    def __init__(self, eps=5.0, sigma=2.05, capacity=0, stream=None):
        import torch

        from . import _lib

        self.lib = _lib.load()
        self.eps, self.sigma = float(eps), float(sigma)
        self.rc = 2.0 ** (1.0 / 6.0) * self.sigma
        self.stream = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        self.h, self.cap = None, 0
        if capacity > 0:
            self._reserve(capacity)

    def _reserve(self, n):
        from . import _lib

        if self.h is not None and n <= self.cap:
            return
        self.close()
        h = ctypes.c_void_p()
        _lib.check(self.lib.fmm_wall_create(ctypes.byref(h), max(int(n), 1), ctypes.c_void_p(self.stream)),
                   "fmm_wall_create")
        self.h, self.cap = h, max(int(n), 1)

    @staticmethod
    def _ptr(t):
        return ctypes.c_void_p(t.data_ptr())

    @staticmethod
    def _check_f8(*ts):
        import torch

        for t in ts:
            if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
                raise ValueError("dynamics arrays must be contiguous float64 CUDA tensors")

    def __call__(self, x):
        """(U, F): U a 0-d device tensor (kcal/mol), F = -dU/dx (n x 3)."""
        import torch

        from . import _lib

        x = torch.as_tensor(x, dtype=torch.float64, device="cuda").contiguous()
        n = int(x.shape[0])
        self._reserve(n)
        U = torch.empty((), dtype=torch.float64, device="cuda")
        F = torch.empty_like(x)
        _lib.check(self.lib.fmm_wall_forces(self.h, self._ptr(x), n, self.eps, self.sigma, self._ptr(U),
                                            self._ptr(F)), "fmm_wall_forces")
        return U, F

    wall = __call__

    def kick(self, v, F, m, coef):
        """v += coef * F / m, in place."""
        from . import _lib

        self._check_f8(v, F, m)
        _lib.check(self.lib.fmm_md_kick(self._ptr(v), self._ptr(F), self._ptr(m), float(coef), int(v.shape[0]),
                                        ctypes.c_void_p(self.stream)), "fmm_md_kick")

    def drift(self, x, v, dt):
        """x += dt * v, in place."""
        from . import _lib

        self._check_f8(x, v)
        _lib.check(self.lib.fmm_md_drift(self._ptr(x), self._ptr(v), float(dt), int(x.shape[0]),
                                         ctypes.c_void_p(self.stream)), "fmm_md_drift")

    def kinetic(self, v, m, scale):
        """scale * sum 1/2 m |v|^2 as a 0-d device tensor."""
        import torch

        from . import _lib

        self._check_f8(v, m)
        self._reserve(int(v.shape[0]))
        out = torch.empty((), dtype=torch.float64, device="cuda")
        _lib.check(self.lib.fmm_md_kinetic(self.h, self._ptr(v), self._ptr(m), int(v.shape[0]), float(scale),
                                           self._ptr(out)), "fmm_md_kinetic")
        return out

    def momentum(self, v, m):
        """Total momentum sum m v as a device tensor of three."""
        import torch

        from . import _lib

        self._check_f8(v, m)
        self._reserve(int(v.shape[0]))
        out = torch.empty(3, dtype=torch.float64, device="cuda")
        _lib.check(self.lib.fmm_md_momentum(self.h, self._ptr(v), self._ptr(m), int(v.shape[0]), self._ptr(out)),
                   "fmm_md_momentum")
        return out

    def close(self):
        if self.h is not None:
            self.lib.fmm_wall_destroy(self.h)
            self.h, self.cap = None, 0

    def __del__(self):
        try:
            self.close()
        except Exception:  # pragma: no cover
            pass


class Dynamics:
    """Molecular dynamics on FMM electrostatics + polarization (the slow force)
    and the wall (the fast force).  A step is velocity Verlet (inner = 1), or
    one outer step of the reversible multiple-time-step integrator (r-RESPA,
    Sec. IV.B runs the long-range forces on a longer step): a half kick of the
    FMM force over the outer step inner * dt, `inner` velocity-Verlet steps of
    dt under the wall, and the closing FMM half kick.  Velocity Verlet applies
    its kicks force by force in the order the multiple-time-step form does
    (opening: FMM then wall; closing: wall then FMM), so that one inner step
    gives the same bits as velocity Verlet.  `ops` provides wall(x),
    kick(v, F, m, coef), drift(x, v, dt) and kinetic(v, m, scale): by default
    the library's CUDA kernels (Repulsion)."""

    def __init__(self, pos, q, alpha, masses, p=6, depth=5, mode="fp64", tol=1e-8, ops=None, predictor=0):
        import torch

        from . import PolFMM

        self.x = torch.as_tensor(pos, dtype=torch.float64, device="cuda").clone().contiguous()
        self.q = torch.as_tensor(q, dtype=torch.float64, device="cuda")
        self.alpha = torch.as_tensor(alpha, dtype=torch.float64, device="cuda")
        self.m = torch.as_tensor(masses, dtype=torch.float64, device="cuda").contiguous()
        self.tol = tol
        self.ops = ops or Repulsion(capacity=self.x.shape[0])
        self.fmm = PolFMM(self.x, self.q, self.alpha, p=p, depth=depth, mode=mode, coulomb_k=COULOMB,
                          max_iter=500)
        if predictor:
            self.fmm.set_dipole_predictor(predictor)
        self.iterations = []
        self.momenta = []
        self.start()

    def start(self):
        """Forces at the current positions (the first step's opening kicks use them)."""
        self.Us, self.Fs = self._slow(update=False)
        self.Uw, self.Fw = self.ops.wall(self.x)

    def _slow(self, update=True):
        """FMM electrostatics and polarization at self.x: (U, F); the solve starts
        from the previous dipoles."""
        if update:
            self.fmm.update_positions(self.x)
        info = self.fmm.solve(self.tol)
        self.iterations.append(info["iterations"])
        out = self.fmm.energy_forces(forces=True, dq=False, dalpha=False)
        return out["U"], out["F"]

    def kinetic(self, v):
        return float(self.ops.kinetic(v, self.m, 1.0 / ACC))

    def total(self, v):
        """Kinetic + FMM + wall energy (kcal/mol)."""
        return self.kinetic(v) + float(self.Us) + float(self.Uw)

    def _verlet_step(self, v, dt):
        c = 0.5 * dt * ACC
        self.ops.kick(v, self.Fs, self.m, c)
        self.ops.kick(v, self.Fw, self.m, c)
        self.ops.drift(self.x, v, dt)
        self.Uw, self.Fw = self.ops.wall(self.x)
        self.Us, self.Fs = self._slow()
        self.ops.kick(v, self.Fw, self.m, c)
        self.ops.kick(v, self.Fs, self.m, c)

    def _respa_step(self, v, dt, inner):
        c_out = 0.5 * inner * dt * ACC
        c = 0.5 * dt * ACC
        self.ops.kick(v, self.Fs, self.m, c_out)
        for _ in range(inner):
            self.ops.kick(v, self.Fw, self.m, c)
            self.ops.drift(self.x, v, dt)
            self.Uw, self.Fw = self.ops.wall(self.x)
            self.ops.kick(v, self.Fw, self.m, c)
        self.Us, self.Fs = self._slow()
        self.ops.kick(v, self.Fs, self.m, c_out)

    def run(self, v, steps, dt=1.0, inner=1, multistep=None, track_momentum=False):
        """Returns the total energy before and after each step (kcal/mol) and the
        final velocities (a new tensor; v itself is not changed).  A step is
        velocity Verlet at dt when inner == 1 (unless multistep=True), else one
        multiple-time-step outer step of inner * dt.  track_momentum: the total
        momentum after each step goes to self.momenta."""
        import torch

        multistep = inner > 1 if multistep is None else bool(multistep)
        v = torch.as_tensor(v, dtype=torch.float64, device=self.x.device).clone().contiguous()
        H = [self.total(v)]
        if track_momentum:
            self.momenta.append(self.ops.momentum(v, self.m).cpu().numpy())
        for _ in range(steps):
            if multistep:
                self._respa_step(v, dt, inner)
            else:
                self._verlet_step(v, dt)
            H.append(self.total(v))
            if track_momentum:
                self.momenta.append(self.ops.momentum(v, self.m).cpu().numpy())
        return np.array(H), v

    def close(self):
        self.fmm.close()
        if hasattr(self.ops, "close"):
            self.ops.close()


def maxwell_velocities(masses, temperature, seed):
    """Velocities of a Maxwell distribution at the temperature, centre-of-mass
    motion removed (Angstrom / fs)."""
    rng = np.random.default_rng(seed)
    sd = np.sqrt(KB * temperature * ACC / masses)
    v = rng.standard_normal((masses.shape[0], 3)) * sd[:, None]
    v -= (masses[:, None] * v).sum(0) / masses.sum()
    return v


def fd_check(pos, q, alpha, p, depth, sites, h=1e-5, tol=1e-11, seed=3):
    """Autograd forces and dU/dq, dU/dalpha against central finite differences
    (FP64, fixed root box) on `sites` random sites: max relative difference."""
    import torch

    from .autograd import polarizable_energy

    xs = np.asarray(pos, dtype=np.float64)
    lo = xs.min(0) - 1.0
    side = float((xs.max(0) - xs.min(0)).max() + 2.0)
    root = (lo, side)
    dev = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
    x = dev(xs).requires_grad_(True)
    qq = dev(q).requires_grad_(True)
    aa = dev(alpha).requires_grad_(True)
    U = polarizable_energy(x, qq, aa, p=p, depth=depth, tol=tol, root_box=root)
    gx, gq, ga = torch.autograd.grad(U, (x, qq, aa))
    gx, gq, ga = gx.cpu().numpy(), gq.cpu().numpy(), ga.cpu().numpy()
    rng = np.random.default_rng(seed)
    pick = rng.choice(xs.shape[0], size=sites, replace=False)

    def energy(xv, qv, av):
        return float(polarizable_energy(dev(xv), dev(qv), dev(av), p=p, depth=depth, tol=tol, root_box=root))

    worst = {"x": 0.0, "q": 0.0, "alpha": 0.0}
    scale_x = np.abs(gx).max()
    for i in pick:
        for d in range(3):
            xp, xm = xs.copy(), xs.copy()
            xp[i, d] += h
            xm[i, d] -= h
            fd = (energy(xp, q, alpha) - energy(xm, q, alpha)) / (2 * h)
            worst["x"] = max(worst["x"], abs(fd - gx[i, d]) / scale_x)
        qp, qm = np.array(q, dtype=np.float64), np.array(q, dtype=np.float64)
        qp[i] += h
        qm[i] -= h
        fd = (energy(xs, qp, alpha) - energy(xs, qm, alpha)) / (2 * h)
        worst["q"] = max(worst["q"], abs(fd - gq[i]) / np.abs(gq).max())
        ap, am = np.array(alpha, dtype=np.float64), np.array(alpha, dtype=np.float64)
        ap[i] += h
        am[i] -= h
        fd = (energy(xs, q, ap) - energy(xs, q, am)) / (2 * h)
        worst["alpha"] = max(worst["alpha"], abs(fd - ga[i]) / np.abs(ga).max())
    return worst


def main(argv=None):
    import torch

    import synth

    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--sites", type=int, default=100000)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--dt", type=float, default=1.0)
    ap.add_argument("--inner", type=int, default=1,
                    help="wall steps per FMM force evaluation (multiple time steps; 1 = velocity Verlet)")
    ap.add_argument("--temperature", type=float, default=300.0)
    ap.add_argument("--fd-sites", type=int, default=64)
    ap.add_argument("--alpha-scale", type=float, default=0.5)
    ap.add_argument("--predictor", type=int, default=0, choices=[0, 1],
                    help="start of each solve: 0 = last dipoles, 1 = linear extrapolation from the last two")
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--modes", default="fp64,mixed", help="comma-separated precision modes to run (fp64, mixed)")
    args = ap.parse_args(argv)
    modes = [m.strip() for m in args.modes.split(",") if m.strip()]
    if not modes or any(m not in ("fp64", "mixed") for m in modes):
        ap.error("--modes takes fp64 and/or mixed")
    w = synth.workload(4, n=args.sites)
    rng = np.random.default_rng(args.seed)
    masses = rng.uniform(1.0, 16.0, w.n)
    v0 = maxwell_velocities(masses, args.temperature, args.seed + 1)
    result = {"config": {"workload": f"globule {w.n} sites p={w.p} depth={w.depth}", "steps": args.steps,
                         "dt_fs": args.dt, "inner_steps": args.inner, "temperature_K": args.temperature,
                         "masses_amu": "U(1, 16)",
                         "repulsion": "repulsive Lennard-Jones wall, eps 5 kcal/mol, sigma 2.05 A, zero beyond 2.30 A",
                         "alpha_scale_dynamics": args.alpha_scale, "dipole_predictor": args.predictor}}
    if args.fd_sites > 0:
        t0 = time.perf_counter()
        result["fd_check"] = {"sites": args.fd_sites, "h": 1e-5,
                              "max_rel_diff": fd_check(w.pos, w.q, w.alpha, w.p, w.depth, args.fd_sites),
                              "seconds": round(time.perf_counter() - t0, 1)}
    for mode, tol in (("fp64", 1e-8), ("mixed", 1e-6)):
        if mode not in modes:
            continue
        dyn = Dynamics(w.pos, w.q, args.alpha_scale * w.alpha, masses, p=w.p, depth=w.depth, mode=mode, tol=tol,
                       predictor=args.predictor)
        v = torch.as_tensor(v0, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        H, v = dyn.run(v, args.steps, args.dt, args.inner, track_momentum=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        ke0 = float(0.5 * (masses[:, None] * v0 * v0).sum() / ACC)
        # drift as a fraction of the initial kinetic energy (the paper's measure)
        result[mode] = {"H0_kcal_mol": float(H[0]), "KE0_kcal_mol": ke0, "drift_of_ke0": float((H[-1] - H[0]) / ke0),
                        "drift_of_ke0_per_step": float(np.polyfit(np.arange(H.size), H, 1)[0] / ke0),
                        "max_dev_of_ke0": float(np.abs(H - H[0]).max() / ke0),
                        "mean_iterations": float(np.mean(dyn.iterations[1:])) if len(dyn.iterations) > 1 else None,
                        "ms_per_step": round(1e3 * dt / max(1, args.steps), 2),
                        # centre-of-mass momentum: largest |P(t) - P(0)| over sum m |v(0)|
                        "momentum_drift": float(np.abs(np.array(dyn.momenta) - dyn.momenta[0]).max()
                                                / (masses * np.linalg.norm(v0, axis=1)).sum()),
                        "finite": bool(np.all(np.isfinite(H)))}
        dyn.close()
    print(json.dumps(result))


if __name__ == "__main__":
    main()
