"""Velocity-Verlet dynamics on the polarizable FMM forces, and the finite-
difference check of the gradients (the differentiation / MD configuration).

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
eps = 5 kcal/mol, sigma = 2.05 A (zero beyond 2.30 A), evaluated in FP64 with
a cell list (torch operations on the GPU; it is not part of the FMM path).
Even so, undamped point dipoles with alpha up to 2.5 A^3 at 0.1 sites/A^3 are
collectively near the catastrophe (largest eigenvalue of alpha^1/2 T alpha^1/2
0.84 on the lattice) and a few fs of motion push them over it; the dynamics
therefore runs with the polarizabilities scaled by --alpha-scale (default 0.5),
while the finite-difference check uses them as they are.

    python -m paper_1408_6527_gb300.md --sites 100000 --steps 1000
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

COULOMB = 332.0637          # kcal Angstrom / (mol e^2)
ACC = 4.184e-4              # Angstrom / fs^2 per (kcal / mol / Angstrom / amu)
KB = 0.0019872              # kcal / (mol K)


class Repulsion:
    """Purely repulsive wall between pairs closer than 2^(1/6) sigma (FP64)."""

    def __init__(self, eps=5.0, sigma=2.05):
        self.eps, self.sigma = float(eps), float(sigma)
        self.rc = 2.0 ** (1.0 / 6.0) * self.sigma

    def __call__(self, x):
        import torch

        n = x.shape[0]
        rc = self.rc
        lo = x.min(0).values - 1e-6
        cell = torch.floor((x - lo) / rc).long()
        dims = cell.max(0).values + 3  # one empty layer of cells on each side
        cell = cell + 1
        key = cell[:, 0] + dims[0] * (cell[:, 1] + dims[1] * cell[:, 2])
        order = torch.argsort(key)
        skey = key[order]
        ncell = int(dims[0] * dims[1] * dims[2])
        count = torch.bincount(skey, minlength=ncell)
        start = torch.cumsum(count, 0) - count
        kmax = int(count.max())
        # table[c, k] = k-th site of cell c, -1 past its count
        table = torch.full((ncell, kmax), -1, dtype=torch.long, device=x.device)
        rank = torch.arange(n, device=x.device) - start[skey]
        table[skey, rank] = order
        U = torch.zeros((), dtype=torch.float64, device=x.device)
        F = torch.zeros_like(x)
        s6 = self.sigma ** 6
        me = torch.arange(n, device=x.device)[:, None]
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    nk = key + dx + dims[0] * (dy + dims[1] * dz)
                    js = table[nk]                                   # [n, kmax]
                    jj = js.clamp(min=0)
                    r = x[:, None, :] - x[jj]                        # [n, kmax, 3]
                    r2 = (r * r).sum(-1)
                    valid = (js >= 0) & (jj != me) & (r2 < rc * rc)
                    r2 = torch.where(valid, r2, torch.ones_like(r2))
                    t6 = s6 * r2 ** -3                               # (sigma / r)^6
                    e = torch.where(valid, 4.0 * self.eps * (t6 * t6 - t6) + self.eps, torch.zeros_like(r2))
                    U = U + 0.5 * e.sum()
                    fmag = torch.where(valid, 4.0 * self.eps * (12.0 * t6 * t6 - 6.0 * t6) / r2, torch.zeros_like(r2))
                    F = F + (fmag[..., None] * r).sum(1)
        return float(U), F


def respa(x, v, acc_slow, acc_fast, slow, fast, dt, inner):
    """One outer step of the reversible multiple-time-step integrator (r-RESPA):
    a half kick of the slow acceleration over the outer step inner * dt,
    `inner` velocity-Verlet steps of dt under the fast acceleration, and the
    closing slow half kick. slow(x) and fast(x) return accelerations; the
    accelerations at the current x are passed in and the new ones returned:
    (x, v, acc_slow, acc_fast). With inner = 1 this is velocity Verlet under
    the sum of the two."""
    h = 0.5 * inner * dt
    v = v + h * acc_slow
    for _ in range(inner):
        v = v + 0.5 * dt * acc_fast
        x = x + dt * v
        acc_fast = fast(x)
        v = v + 0.5 * dt * acc_fast
    acc_slow = slow(x)
    v = v + h * acc_slow
    return x, v, acc_slow, acc_fast


class Dynamics:
    """Velocity Verlet with FMM electrostatics + polarization and the wall;
    with inner > 1 the multiple-time-step form (the FMM forces every inner
    steps, the wall every step)."""

    def __init__(self, pos, q, alpha, masses, p=6, depth=5, mode="fp64", tol=1e-8, repulsion=None):
        import torch

        from . import PolFMM

        self.x = torch.as_tensor(pos, dtype=torch.float64, device="cuda").clone()
        self.q = torch.as_tensor(q, dtype=torch.float64, device="cuda")
        self.alpha = torch.as_tensor(alpha, dtype=torch.float64, device="cuda")
        self.m = torch.as_tensor(masses, dtype=torch.float64, device="cuda")
        self.tol = tol
        self.rep = repulsion or Repulsion()
        self.fmm = PolFMM(self.x, self.q, self.alpha, p=p, depth=depth, mode=mode, coulomb_k=COULOMB,
                          max_iter=500)
        self.iterations = []
        self.U, self.F = self._forces(first=True)

    def _forces(self, first=False):
        if not first:
            self.fmm.update_positions(self.x)  # keeps the dipoles as the start of the next solve
        info = self.fmm.solve(self.tol)
        self.iterations.append(info["iterations"])
        out = self.fmm.energy_forces(forces=True, dq=False, dalpha=False)
        ur, fr = self.rep(self.x)
        return out["U"] + ur, out["F"] + fr

    def kinetic(self, v):
        return float(0.5 * (self.m[:, None] * v * v).sum() / ACC)

    def _slow(self):
        """FMM electrostatics and polarization at self.x: (U, F)."""
        self.fmm.update_positions(self.x)
        info = self.fmm.solve(self.tol)
        self.iterations.append(info["iterations"])
        out = self.fmm.energy_forces(forces=True, dq=False, dalpha=False)
        return out["U"], out["F"]

    def run(self, v, steps, dt=1.0, inner=1):
        """Returns the total energy before and after each step (kcal/mol) and the
        final velocities. With inner > 1 a step is one outer step of inner * dt:
        the wall is integrated at dt and the FMM forces at inner * dt (r-RESPA)."""
        if inner > 1:
            return self._run_respa(v, steps, dt, inner)
        H = [self.kinetic(v) + self.U]
        a = self.F / self.m[:, None] * ACC
        for _ in range(steps):
            v = v + 0.5 * dt * a
            self.x = self.x + dt * v
            self.U, self.F = self._forces()
            a = self.F / self.m[:, None] * ACC
            v = v + 0.5 * dt * a
            H.append(self.kinetic(v) + self.U)
        return np.array(H), v

    def _run_respa(self, v, steps, dt, inner):
        inv_m = ACC / self.m[:, None]
        ur, fr = self.rep(self.x)
        us, fs = self.U - ur, self.F - fr  # the first forces hold both parts
        state = {"ur": ur, "us": us}

        def fast(x):
            state["ur"], f = self.rep(x)
            return f * inv_m

        def slow(x):
            self.x = x
            state["us"], f = self._slow()
            return f * inv_m

        H = [self.kinetic(v) + us + ur]
        a_s, a_f = fs * inv_m, fr * inv_m
        for _ in range(steps):
            self.x, v, a_s, a_f = respa(self.x, v, a_s, a_f, slow, fast, dt, inner)
            H.append(self.kinetic(v) + state["us"] + state["ur"])
        self.U = state["us"] + state["ur"]
        self.F = (a_s + a_f) / inv_m
        return np.array(H), v

    def close(self):
        self.fmm.close()


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
    ap.add_argument("--seed", type=int, default=7)
    args = ap.parse_args(argv)
    w = synth.workload(4, n=args.sites)
    rng = np.random.default_rng(args.seed)
    masses = rng.uniform(1.0, 16.0, w.n)
    v0 = maxwell_velocities(masses, args.temperature, args.seed + 1)
    result = {"config": {"workload": f"globule {w.n} sites p={w.p} depth={w.depth}", "steps": args.steps,
                         "dt_fs": args.dt, "inner_steps": args.inner, "temperature_K": args.temperature,
                         "masses_amu": "U(1, 16)",
                         "repulsion": "repulsive Lennard-Jones wall, eps 5 kcal/mol, sigma 2.05 A, zero beyond 2.30 A",
                         "alpha_scale_dynamics": args.alpha_scale}}
    if args.fd_sites > 0:
        t0 = time.perf_counter()
        result["fd_check"] = {"sites": args.fd_sites, "h": 1e-5,
                              "max_rel_diff": fd_check(w.pos, w.q, w.alpha, w.p, w.depth, args.fd_sites),
                              "seconds": round(time.perf_counter() - t0, 1)}
    for mode, tol in (("fp64", 1e-8), ("mixed", 1e-6)):
        dyn = Dynamics(w.pos, w.q, args.alpha_scale * w.alpha, masses, p=w.p, depth=w.depth, mode=mode, tol=tol)
        v = torch.as_tensor(v0, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        H, v = dyn.run(v, args.steps, args.dt, args.inner)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        ke0 = float(0.5 * (masses[:, None] * v0 * v0).sum() / ACC)
        # drift as a fraction of the initial kinetic energy (the paper's measure)
        result[mode] = {"H0_kcal_mol": float(H[0]), "KE0_kcal_mol": ke0, "drift_of_ke0": float((H[-1] - H[0]) / ke0),
                        "drift_of_ke0_per_step": float(np.polyfit(np.arange(H.size), H, 1)[0] / ke0),
                        "max_dev_of_ke0": float(np.abs(H - H[0]).max() / ke0),
                        "mean_iterations": float(np.mean(dyn.iterations[1:])) if len(dyn.iterations) > 1 else None,
                        "ms_per_step": round(1e3 * dt / max(1, args.steps), 2),
                        "finite": bool(np.all(np.isfinite(H)))}
        dyn.close()
    print(json.dumps(result))


if __name__ == "__main__":
    main()
