"""Polarizable energy with exclusion lists and a separate field-charge set, on
the CPU in FP64 (the Polaris specifics of Sec. II.A and Sec. III).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``; pinned by
``tests/test_oracle_polaris.py``.

What the paper fixes:
- The starred sums skip a set of excluded pairs: the Coulomb energy
  (Eq. equ:Uqq), the static field E^q and the dipole field E^mu (Sec. II.A).
- Only the atoms with a field charge q^E, which may differ from the Coulomb
  charge q, generate E^q. The field acts on the polarizable atoms (Sec. III).

Energy, with mu solving mu_i = alpha_i (E^q_i + E^mu_i) at the polarizable
sites:
    U = 1/2 sum_i q_i sum*_j q_j / r_ij
      + sum_i |mu_i|^2 / (2 alpha_i) - sum_i mu_i.E^q_i - 1/2 sum_i mu_i.E^mu_i.

At that stationary point the first-order change of mu drops out (Eq.
upol_derivatives), so the derivatives are those of the explicit dependence:
    F_k        = q_k E^coul_k + q^E_k E^mu_k + (grad E^qE_k + grad E^mu_k) mu_k
    dU/dq_k    = Phi^coul_k (potential of the Coulomb charges)
    dU/dq^E_k  = Phi^mu_k   (potential of the dipoles)
    dU/dalpha  = -|mu|^2 / (2 alpha^2), and its alpha -> 0 limit -|E|^2 / 2 at
                 sites without polarizability (E = E^qE + E^mu there)
Here E^coul and Phi^coul come from the charges q, E^qE from the q^E, and
E^mu and Phi^mu from the dipoles, all over the non-excluded pairs; E^mu is
needed at every site that carries a q^E.

Readings:
- The exclusion set is an input list of site pairs. The paper's example (atoms
  "separated by less than two chemical bonds") names a common choice, not a
  rule.
- A pair that is excluded is excluded from all three sums.

``dense`` evaluates the pair sums directly. ``fmm`` takes the CPU octree FMM's
fields over all pairs and subtracts the excluded pairs' direct terms, which
is how an FMM handles exclusions.
"""
from __future__ import annotations

import numpy as np

from . import OracleError, fmm_fields, pcg_dipole_solve


def _pairs(pos):
    r = pos[:, None, :] - pos[None, :, :]  # r_ij = x_i - x_j
    r2 = np.einsum("ijk,ijk->ij", r, r)
    np.fill_diagonal(r2, 1.0)
    return r, 1.0 / np.sqrt(r2)


def _mask(n, exclusions):
    m = ~np.eye(n, dtype=bool)
    for i, j in exclusions:
        m[i, j] = m[j, i] = False
    return m


def _charge_fields(r, ri, w):
    """Phi, E, G at every site from charges w over the weighted pairs (w already
    carries the mask): Phi = sum w/r, E = sum w r/r^3, G = sum w (1/r^3 - 3 r r / r^5)."""
    ri3 = ri ** 3
    phi = (w * ri).sum(1)
    E = np.einsum("ij,ijk->ik", w * ri3, r)
    ri5 = ri3 * ri * ri
    G = np.zeros((r.shape[0], 6))
    for c, (a, b) in enumerate(((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))):
        G[:, c] = (w * (ri3 * (a == b) - 3.0 * r[:, :, a] * r[:, :, b] * ri5)).sum(1)
    return phi, E, G


def _dipole_fields(r, ri, mask, mu):
    """Phi, E, G at every site from point dipoles mu over the non-excluded pairs:
    Phi = mu.r/r^3, E = 3 (mu.r) r / r^5 - mu / r^3,
    G_ab = 3 (mu_a r_b + mu_b r_a + (mu.r) delta_ab) / r^5 - 15 (mu.r) r_a r_b / r^7."""
    ri3 = ri ** 3 * mask
    ri5 = ri3 * ri * ri
    ri7 = ri5 * ri * ri
    mr = np.einsum("ijk,jk->ij", r, mu)
    phi = (mr * ri3).sum(1)
    E = 3.0 * np.einsum("ij,ijk->ik", mr * ri5, r) - ri3 @ mu
    G = np.zeros((r.shape[0], 6))
    for c, (a, b) in enumerate(((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))):
        G[:, c] = (3.0 * ri5 * (mu[None, :, a] * r[:, :, b] + mu[None, :, b] * r[:, :, a] + mr * (a == b))
                   - 15.0 * mr * r[:, :, a] * r[:, :, b] * ri7).sum(1)
    return phi, E, G


def _excluded_correction(pos, exclusions, w, mu=None):
    """Direct terms of the excluded pairs (both directions): Phi, E, G of charges
    w, or of dipoles mu when given, at every site; what an FMM over all pairs
    must subtract."""
    n = pos.shape[0]
    phi, E, G = np.zeros(n), np.zeros((n, 3)), np.zeros((n, 6))
    for i, j in exclusions:
        for t, s in ((i, j), (j, i)):
            sub = pos[[s, t]]
            r, ri = _pairs(sub)
            m = np.array([[False, False], [True, False]])  # target row 1 sees source 0
            if mu is None:
                ww = np.array([[0.0, 0.0], [w[s], 0.0]])
                ph, e, g = _charge_fields(r, ri, ww)
            else:
                ph, e, g = _dipole_fields(r, ri, m, np.array([mu[s], np.zeros(3)]))
            phi[t] += ph[1]
            E[t] += e[1]
            G[t] += g[1]
    return phi, E, G


def polaris_energy(pos, q, qE, alpha, exclusions=(), method="dense", p=8, depth=3, root=None, solve="dense",
                   tol=1e-13, max_iter=500):
    """U, its gradients and the dipoles for charges q, field charges qE,
    polarizabilities alpha and the excluded pairs. method: "dense" (pair sums)
    or "fmm" (CPU octree FMM at order p over all pairs, minus the excluded
    pairs' direct terms). solve: "dense" (Cholesky of diag(1/alpha) - T, T
    built column by column from the method's dipole field and symmetrised) or
    "pcg" (the preconditioned conjugate gradients of ``oracle.pcg_dipole_solve``
    on the method's dipole field as it is, to the relative residual tol)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    q, qE, alpha = (np.asarray(v, dtype=np.float64) for v in (q, qE, alpha))
    n = pos.shape[0]
    exclusions = [(int(i), int(j)) for i, j in exclusions]
    mask = _mask(n, exclusions)
    r, ri = _pairs(pos)
    act = alpha > 0

    if method == "dense":
        def charges(w):
            return _charge_fields(r, ri, mask * w[None, :])

        def dipoles(mu):
            return _dipole_fields(r, ri, mask, mu)
    elif method == "fmm":
        def charges(w):
            f = fmm_fields(pos, w, None, p=p, depth=depth, root=root)
            c = _excluded_correction(pos, exclusions, w)
            return f["phi"] - c[0], f["E"] - c[1], f["G"] - c[2]

        def dipoles(mu):
            f = fmm_fields(pos, None, mu, p=p, depth=depth, root=root)
            c = _excluded_correction(pos, exclusions, None, mu)
            return f["phi"] - c[0], f["E"] - c[1], f["G"] - c[2]
    else:
        raise ValueError(method)

    phi_c, E_c, _ = charges(q)
    _, E_qE, G_qE = charges(qE)
    # mu = alpha (E^qE + T mu) on the polarizable sites: dense Cholesky of
    # diag(1/alpha) - T over the active sites, T applied through `dipoles`,
    # or PCG with that operator
    idx = np.nonzero(act)[0]
    mu = np.zeros((n, 3))
    if solve == "pcg":
        mu, _, _, _ = pcg_dipole_solve(alpha, E_qE, lambda v: dipoles(v)[1], tol=tol, max_iter=max_iter)
    elif solve != "dense":
        raise ValueError(solve)
    elif idx.size:
        k = idx.size
        T = np.zeros((3 * k, 3 * k))
        for c in range(3 * k):
            e = np.zeros((n, 3))
            e[idx[c // 3], c % 3] = 1.0
            T[:, c] = dipoles(e)[1][idx].ravel()
        T = 0.5 * (T + T.T)
        A = np.diag(np.repeat(1.0 / alpha[idx], 3)) - T
        try:
            L = np.linalg.cholesky(A)
        except np.linalg.LinAlgError as err:
            raise OracleError(f"dipole matrix not positive definite: {err}")
        y = np.linalg.solve(L, E_qE[idx].ravel())
        mu[idx] = np.linalg.solve(L.T, y).reshape(-1, 3)
    phi_m, E_m, G_m = dipoles(mu)

    m2 = (mu * mu).sum(1)
    safe = np.where(act, alpha, 1.0)
    Uqq = 0.5 * float((q * phi_c).sum())
    Upol = float(0.5 * np.where(act, m2 / safe, 0.0).sum() - (mu * E_qE).sum() - 0.5 * (mu * E_m).sum())
    G = G_qE + G_m
    Gm = np.stack([G[:, 0] * mu[:, 0] + G[:, 1] * mu[:, 1] + G[:, 2] * mu[:, 2],
                   G[:, 1] * mu[:, 0] + G[:, 3] * mu[:, 1] + G[:, 4] * mu[:, 2],
                   G[:, 2] * mu[:, 0] + G[:, 4] * mu[:, 1] + G[:, 5] * mu[:, 2]], 1)
    F = q[:, None] * E_c + qE[:, None] * E_m + Gm
    return {"U": Uqq + Upol, "Uqq": Uqq, "Upol": Upol, "Upol_stationary": -0.5 * float((mu * E_qE).sum()),
            "F": F, "dUdq": phi_c, "dUdqE": phi_m,
            "dUdalpha": np.where(act, -m2 / (2.0 * safe * safe), -0.5 * ((E_qE + E_m) ** 2).sum(1)),
            "mu": mu}
