"""Seeded synthetic inputs for the polarizable FMM workloads.

This module only draws random site sets (positions, charges, polarizabilities)
with the densities and value distributions of the paper's molecular systems
(protein-like density of about 0.1 atoms per cubic Angstrom, a minimum pair
distance as in the sphere test of Sec. IV.A).  It holds none of the method's
arithmetic: no potentials, fields, expansions or solves.  Both the CPU oracle
and the CUDA path receive the arrays it returns.

Readings taken where the workload descriptions are under-specified:

* Thole-free point dipoles at protein density are close to the
  polarization catastrophe: random sequential addition with a 1.75-1.8 A hard
  core leaves the largest eigenvalue of alpha^1/2 T alpha^1/2 above 1 (1.14 for
  the cube, 1.15 in the globule core), i.e. an indefinite dipole matrix.  The
  five workloads therefore place their sites on a randomly rotated and
  shifted face-centred-cubic lattice of the target density (nearest neighbour
  2.42 A at 0.1 A^-3), displace each site uniformly within 0.2 A, and select
  the sites by the density profile (lowest key u / p(x), u uniform).  Largest
  eigenvalue then 0.84 (globule core) and 0.86 (cube): positive definite.
  The paper's sphere test (Sec. IV.A, 2 A minimum separation at low density)
  keeps random sequential addition.
* The Gaussian globule is a capped Gaussian rho(r) = min(0.1, A exp(-r^2/2s^2))
  with s = 15 A; the flat-core radius is solved so that the integral is N.
* The six-lobe ring uses the union density min(0.1, sum_g rho_g) with one
  shared core radius solved so that the integral is N.
* The hollow shell keeps a 40 A thickness at 0.1 A^-3 and solves the inner
  radius from N.
* Charges: +-U(0.1, 0.8) e for the cube, N(0, 0.35) e otherwise, shifted to
  net zero.  Seeds: PCG64(20140827 + workload index).
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20140827
RHO0 = 0.1  # sites per cubic Angstrom


@dataclass
class Workload:
    name: str
    pos: np.ndarray  # (n, 3) float64, Angstrom
    q: np.ndarray  # (n,) float64, e
    alpha: np.ndarray  # (n,) float64, Angstrom^3
    p: int
    depth: int
    tol: float
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


# --------------------------------------------------------------------------
# hard-core random sequential addition on a cell grid
# --------------------------------------------------------------------------

def _neighbour_offsets(cell: float, d_min: float, reach: int):
    offs = []
    for a in range(-reach, reach + 1):
        for b in range(-reach, reach + 1):
            for c in range(-reach, reach + 1):
                gap = [max(abs(t) - 1, 0) * cell for t in (a, b, c)]
                if math.sqrt(sum(g * g for g in gap)) < d_min:
                    offs.append((a, b, c))
    return np.array(offs, dtype=np.int64)


def hardcore_sample(rng, n, d_min, lo, hi, propose, max_rounds=20000):
    """Draw n points with pairwise distance >= d_min.

    `propose(rng, m)` returns up to m candidate points (already thinned to the
    target density).  Candidates are accepted in order; a candidate is rejected
    if it lies within d_min of an accepted point or of an earlier candidate of
    the same batch.
    """
    lo = np.asarray(lo, dtype=np.float64) - 1e-9
    hi = np.asarray(hi, dtype=np.float64) + 1e-9
    cell = d_min / math.sqrt(3.0) * 0.999  # one point per cell at most
    pad = 3
    dims = np.ceil((hi - lo) / cell).astype(np.int64) + 2 * pad
    ncell = int(np.prod(dims))
    strides = np.array([1, dims[0], dims[0] * dims[1]], dtype=np.int64)
    offs = _neighbour_offsets(cell, d_min, 2)
    off_lin = offs @ strides
    grid = np.full(ncell, -1, dtype=np.int64)
    pts = np.empty((n, 3), dtype=np.float64)
    cnt = 0
    d2min = d_min * d_min
    batch = max(1024, n // 8)
    stalled = 0
    for _ in range(max_rounds):
        if cnt >= n:
            break
        if stalled >= 40:
            break
        cand = propose(rng, batch)
        if cand.shape[0] == 0:
            continue
        ijk = np.floor((cand - lo) / cell).astype(np.int64) + pad
        ci = ijk @ strides
        ok = grid[ci] < 0
        cand, ci = cand[ok], ci[ok]
        # conflicts with accepted points
        ok = np.ones(cand.shape[0], dtype=bool)
        for ol in off_lin:
            nb = grid[ci + ol]
            has = nb >= 0
            if not has.any():
                continue
            d = cand[has] - pts[nb[has]]
            bad = np.einsum("ij,ij->i", d, d) < d2min
            idx = np.nonzero(has)[0][bad]
            ok[idx] = False
        cand, ci = cand[ok], ci[ok]
        if cand.shape[0] == 0:
            stalled += 1
            batch = min(batch * 2, 1 << 22)
            continue
        # conflicts inside the batch: keep the earliest candidate per cell,
        # then reject any candidate near an earlier surviving one
        order = np.arange(cand.shape[0])
        first = {}
        tmp_cells, first_idx = np.unique(ci, return_index=True)
        keep = np.zeros(cand.shape[0], dtype=bool)
        keep[first_idx] = True
        cand, ci, order = cand[keep], ci[keep], order[keep]
        tmp = {}
        # dense temp grid restricted to touched cells via a sorted lookup
        sorter = np.argsort(ci)
        sci = ci[sorter]
        ok = np.ones(cand.shape[0], dtype=bool)
        for ol in off_lin:
            if ol == 0:
                continue
            tgt = ci + ol
            pos_ = np.searchsorted(sci, tgt)
            pos_c = np.minimum(pos_, sci.shape[0] - 1)
            found = sci[pos_c] == tgt
            if not found.any():
                continue
            other = sorter[pos_c[found]]
            me = np.nonzero(found)[0]
            earlier = order[other] < order[me]
            if not earlier.any():
                continue
            me, other = me[earlier], other[earlier]
            d = cand[me] - cand[other]
            bad = np.einsum("ij,ij->i", d, d) < d2min
            ok[me[bad]] = False
        del first, tmp
        cand, ci = cand[ok], ci[ok]
        take = min(cand.shape[0], n - cnt)
        stalled = stalled + 1 if take * 1000 < batch else 0
        cand, ci = cand[:take], ci[:take]
        pts[cnt:cnt + take] = cand
        grid[ci] = np.arange(cnt, cnt + take)
        cnt += take
        rate = take / max(batch, 1)
        if rate < 0.05:
            batch = min(batch * 2, 1 << 22)
    if cnt < n:
        raise RuntimeError(f"hard-core sampler placed only {cnt} of {n} points")
    return pts


# --------------------------------------------------------------------------
# density profiles (sampling only)
# --------------------------------------------------------------------------

def _capped_gaussian_count(rc, sigma, rho0=RHO0):
    """Number of sites in min(rho0, A exp(-r^2/2s^2)) with the cap ending at rc."""
    r = np.linspace(rc, rc + 12 * sigma, 20001)
    f = 4 * math.pi * r * r * rho0 * np.exp(-(r * r - rc * rc) / (2 * sigma * sigma))
    tail = np.trapezoid(f, r)
    return rho0 * 4.0 / 3.0 * math.pi * rc ** 3 + tail


def _solve_monotone(fun, target, lo, hi, iters=200):
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if fun(mid) < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def globule_core_radius(n, sigma=15.0):
    return _solve_monotone(lambda rc: _capped_gaussian_count(rc, sigma), n, 0.0, 1e4)


def _ball_proposer(center, radius, accept_prob):
    center = np.asarray(center, dtype=np.float64)

    def propose(rng, m):
        u = rng.random((m, 3)) * 2 - 1
        u = u[np.einsum("ij,ij->i", u, u) <= 1.0]
        x = center + radius * u
        keep = rng.random(x.shape[0]) < accept_prob(x)
        return x[keep]

    return propose


LATTICE_JITTER = 0.2  # Angstrom


def fcc_points(rng, rho, lo, hi, jitter=LATTICE_JITTER):
    """Face-centred-cubic lattice points of density rho covering the box
    [lo, hi], randomly rotated and shifted, each displaced uniformly within a
    ball of radius `jitter`."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    a = (4.0 / rho) ** (1.0 / 3.0)
    centre = 0.5 * (lo + hi)
    half = 0.5 * np.linalg.norm(hi - lo) + a
    m = int(np.ceil(half / a)) + 1
    g = np.arange(-m, m + 1, dtype=np.float64)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    shift = rng.random(3) * a
    out = []
    for z in g:  # slab by slab to bound memory
        X, Y = np.meshgrid(g, g, indexing="ij")
        base = np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], 1)
        pts = (base[:, None, :] + basis[None]).reshape(-1, 3) * a
        pts = (pts + shift - 0.5 * a) @ Q.T + centre
        keep = np.all((pts >= lo - jitter) & (pts <= hi + jitter), axis=1)
        out.append(pts[keep])
    pts = np.concatenate(out)
    u = rng.normal(size=pts.shape)
    u /= np.linalg.norm(u, axis=1)[:, None]
    return pts + jitter * u * rng.random((pts.shape[0], 1)) ** (1.0 / 3.0)


def _select(rng, pts, n, prob, outside_dist=None):
    """Keep the n points with the lowest key u / p(x) (p > 0) or 2 + distance
    outside the region (p = 0), u uniform: thinning to exactly n points."""
    p = prob(pts)
    u = rng.random(pts.shape[0])
    key = np.where(p > 0, u / np.maximum(p, 1e-300), np.inf)
    if outside_dist is not None:
        key = np.where(p > 0, key, 2.0 + outside_dist(pts))
    idx = np.argsort(key, kind="stable")[:n]
    if not np.all(np.isfinite(key[idx])):
        raise RuntimeError("lattice region too small for the requested site count")
    sel = pts[idx]
    return sel[rng.permutation(n)]


def sites_globule(rng, n, sigma=15.0):
    rc = globule_core_radius(n, sigma)
    rs = rc + 60.0

    def prob(x):
        r2 = np.einsum("ij,ij->i", x, x)
        return np.where(r2 <= rs * rs, np.minimum(1.0, np.exp(-(r2 - rc * rc) / (2 * sigma * sigma))), 0.0)

    pts = _select(rng, fcc_points(rng, RHO0, [-rs] * 3, [rs] * 3), n, prob)
    return pts, {"core_radius": rc, "sigma": sigma, "lattice": "fcc", "jitter": LATTICE_JITTER}


def _ring_centres(n_lobes, ring_radius):
    ang = 2 * math.pi * np.arange(n_lobes) / n_lobes
    return np.stack([ring_radius * np.cos(ang), ring_radius * np.sin(ang), np.zeros(n_lobes)], 1)


def _ring_prob(x, centres, rc, sigma):
    s = np.zeros(x.shape[0])
    for c in centres:
        d = x - c
        r2 = np.einsum("ij,ij->i", d, d)
        s += np.exp(-(r2 - rc * rc) / (2 * sigma * sigma))
    return np.minimum(1.0, s)


def ring_core_radius(n, n_lobes=6, ring_radius=60.0, sigma=15.0, h=1.5):
    centres = _ring_centres(n_lobes, ring_radius)

    def count(rc):
        ext = ring_radius + rc + 8 * sigma
        zext = rc + 8 * sigma
        xs = np.arange(-ext, ext + h, h)
        zs = np.arange(-zext, zext + h, h)
        tot = 0.0
        X, Y = np.meshgrid(xs, xs, indexing="ij")
        for z in zs:
            pts = np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], 1)
            tot += _ring_prob(pts, centres, rc, sigma).sum()
        return tot * RHO0 * h ** 3

    return _solve_monotone(count, n, 0.0, 200.0, iters=40)


def sites_ring(rng, n, n_lobes=6, ring_radius=60.0, sigma=15.0):
    rc = ring_core_radius(n, n_lobes, ring_radius, sigma)
    centres = _ring_centres(n_lobes, ring_radius)
    ext = ring_radius + rc + 60.0
    zext = rc + 60.0
    lo = np.array([-ext, -ext, -zext])
    hi = np.array([ext, ext, zext])
    pts = _select(rng, fcc_points(rng, RHO0, lo, hi), n, lambda x: _ring_prob(x, centres, rc, sigma))
    return pts, {"core_radius": rc, "sigma": sigma, "ring_radius": ring_radius, "lobes": n_lobes,
                 "lattice": "fcc", "jitter": LATTICE_JITTER}


def shell_inner_radius(n, thickness=40.0):
    f = lambda r: RHO0 * 4.0 / 3.0 * math.pi * ((r + thickness) ** 3 - r ** 3)
    return _solve_monotone(f, n, 0.0, 1e5)


def sites_shell(rng, n, thickness=40.0):
    r_in = shell_inner_radius(n, thickness)
    r_out = r_in + thickness

    def rad(x):
        return np.sqrt(np.einsum("ij,ij->i", x, x))

    pts = _select(rng, fcc_points(rng, RHO0, [-r_out - 3] * 3, [r_out + 3] * 3), n,
                  lambda x: ((rad(x) >= r_in) & (rad(x) <= r_out)).astype(np.float64),
                  lambda x: np.maximum(r_in - rad(x), rad(x) - r_out))
    return pts, {"inner_radius": r_in, "thickness": thickness, "lattice": "fcc", "jitter": LATTICE_JITTER}


def sites_cube(rng, n, side=20.0):
    def inside(x):
        return np.all((x >= 0) & (x <= side), axis=1).astype(np.float64)

    def dist(x):
        return np.max(np.maximum(-x, x - side), axis=1)

    pts = _select(rng, fcc_points(rng, n / side**3, [0, 0, 0], [side] * 3), n, inside, dist)
    return pts, {"side": side, "lattice": "fcc", "jitter": LATTICE_JITTER}


def sites_sphere(rng, n, radius, d_min):
    """Uniform points in a ball with a minimum separation (sphere test, Sec. IV.A)."""
    prop = _ball_proposer([0, 0, 0], radius, lambda x: np.ones(x.shape[0]))
    return hardcore_sample(rng, n, d_min, [-radius] * 3, [radius] * 3, prop)


# --------------------------------------------------------------------------
# charges and polarizabilities
# --------------------------------------------------------------------------

def charges_uniform_pm(rng, n, lo=0.1, hi=0.8):
    s = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    q = s * rng.uniform(lo, hi, n)
    return q - q.mean()


def charges_normal(rng, n, sd=0.35):
    q = rng.normal(0.0, sd, n)
    return q - q.mean()


def charges_pm_equal(rng, n):
    q = np.ones(n)
    q[: n // 2] = -1.0
    rng.shuffle(q)
    return q


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

_CACHE = os.environ.get("POLFMM_SYNTH_CACHE", os.path.join(os.path.dirname(os.path.abspath(__file__)), "_cache"))


def _cached_positions(key, make):
    path = os.path.join(_CACHE, key + ".npy")
    if os.path.exists(path):
        try:
            return np.load(path)
        except Exception:
            pass
    pts = make()
    try:
        os.makedirs(_CACHE, exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp.npy"
        np.save(tmp, pts)
        os.replace(tmp, path)
    except OSError:
        pass
    return pts


def workload(index: int, n: int | None = None, depth: int | None = None) -> Workload:
    """Workloads 1..5: cube 1k, globule 30k, six-lobe ring 300k, globule 100k, shell sweep."""
    seed = SEED_BASE + index
    rng = np.random.Generator(np.random.PCG64(seed))
    meta = {"seed": seed}
    if index == 1:
        n = n or 1000
        pos, m = sites_cube(rng, n)
        q = charges_uniform_pm(rng, n)
        alpha = rng.uniform(0.5, 2.0, n)
        return Workload("cube", pos, q, alpha, 4, depth or 3, 1e-8, {**meta, **m})
    if index in (2, 4):
        n = n or (30000 if index == 2 else 100000)
        pts = _cached_positions(f"globule_fcc_{n}_{seed}", lambda: sites_globule(rng, n)[0])
        rng2 = np.random.Generator(np.random.PCG64(seed + 1000))
        q = charges_normal(rng2, n)
        alpha = rng2.uniform(0.3, 2.5, n)
        rc = globule_core_radius(n)
        return Workload("globule", pts, q, alpha, 6, depth or (4 if index == 2 else 5), 1e-8,
                        {**meta, "core_radius": rc, "sigma": 15.0, "lattice": "fcc", "jitter": LATTICE_JITTER})
    if index == 3:
        n = n or 300000
        pts = _cached_positions(f"ring_fcc_{n}_{seed}", lambda: sites_ring(rng, n)[0])
        rng2 = np.random.Generator(np.random.PCG64(seed + 1000))
        q = charges_normal(rng2, n)
        alpha = rng2.uniform(0.3, 2.5, n)
        return Workload("ring6", pts, q, alpha, 6, depth or 5, 1e-6, {**meta, "lobes": 6, "ring_radius": 60.0})
    if index == 5:
        n = n or 250000
        # depth minimising the measured cost of one FMM pass at p = 8 (near-field
        # pairs x 1.6 ps + M2L box pairs x 0.64 ns): 4 / 5 / 6 at 250k / 1M / 4M
        d = depth or max(3, int(round(math.log(n / 40.0, 8))))
        pts = _cached_positions(f"shell_fcc_{n}_{seed}", lambda: sites_shell(rng, n)[0])
        rng2 = np.random.Generator(np.random.PCG64(seed + 1000))
        q = charges_normal(rng2, n)
        alpha = rng2.uniform(0.3, 2.5, n)
        return Workload("shell", pts, q, alpha, 8, d, 1e-6, {**meta, "inner_radius": shell_inner_radius(n)})
    raise ValueError(f"unknown workload {index}")


def small_random(seed, n, box=12.0, d_min=1.8, alpha_range=(0.3, 2.0), q_sd=0.35):
    """Small random cluster for unit tests (not one of the five workloads)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = hardcore_sample(rng, n, d_min, [0, 0, 0], [box] * 3, lambda r, m: box * r.random((m, 3)))
    q = charges_normal(rng, n, q_sd)
    alpha = rng.uniform(alpha_range[0], alpha_range[1], n)
    return pos, q, alpha
