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
- Thole damping of the dipole tensor (Sec. II.A cites Thole's model without
  printing it): the exponential model of B. T. Thole, Chem. Phys. 59, 341
  (1981), in the form of P. Ren and J. W. Ponder, J. Phys. Chem. B 107, 5933
  (2003). Between two dipoles the field 3 (mu.r) r / r^5 - mu / r^3 becomes
  lambda5 3 (mu.r) r / r^5 - lambda3 mu / r^3, with u = r / (alpha_i alpha_j)^(1/6),
  lambda3 = 1 - exp(-a u^3), lambda5 = 1 - (1 + a u^3) exp(-a u^3); a pair with
  a non-polarizable site is not damped. Charge-dipole terms stay undamped.
  The dipole-dipole part of the forces and of dU/dalpha then carries the
  derivatives of lambda3 and lambda5:
      F_i  += sum_j grad_i (mu_i . T^d_ij mu_j),
      dU/dalpha_i += -sum_j mu_i . (d T^d_ij / d alpha_i) mu_j.

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


def thole_factors(r, ri, alpha, a, mask):
    """lambda3, lambda5 of every pair and their derivatives with respect to r
    and to u (the damping is 1 where alpha_i alpha_j = 0 or the pair is masked)."""
    rr = 1.0 / ri
    s = np.cbrt(np.sqrt(np.outer(alpha, alpha)))  # (alpha_i alpha_j)^(1/6)
    on = mask & (s > 0)
    u = np.where(on, rr / np.where(on, s, 1.0), np.inf)
    au3 = a * u ** 3
    ex = np.where(on, np.exp(-np.where(on, au3, 0.0)), 0.0)
    au3 = np.where(on, au3, 0.0)
    l3 = 1.0 - ex
    l5 = 1.0 - (1.0 + au3) * ex
    uf = np.where(on, u, 0.0)
    d3u = 3.0 * a * uf ** 2 * ex
    d5u = 3.0 * a * a * uf ** 5 * ex
    sf = np.where(on, s, 1.0)
    return {"l3": l3, "l5": l5, "d3r": d3u / sf, "d5r": d5u / sf, "d3u": d3u, "d5u": d5u, "u": uf}


def _dipole_field_damped(r, ri, mask, mu, th):
    """E_i = sum_j lambda5 3 (mu_j.r) r / r^5 - lambda3 mu_j / r^3 (Thole)."""
    ri3 = ri ** 3 * mask
    ri5 = ri3 * ri * ri
    mr = np.einsum("ijk,jk->ij", r, mu)
    return 3.0 * np.einsum("ij,ijk->ik", th["l5"] * mr * ri5, r) - (th["l3"] * ri3) @ mu


def _dipole_pair_gradients(r, ri, mask, mu, alpha, th):
    """sum_j grad_i (mu_i . T^d_ij mu_j) and sum_j mu_i . (d T^d_ij / d alpha_i) mu_j
    with T^d_ij mu_j the damped field of dipole j at i."""
    ri1 = ri * mask
    ri3 = ri1 ** 3
    ri5 = ri3 * ri1 * ri1
    ri7 = ri5 * ri1 * ri1
    A = mu @ mu.T                                   # mu_i . mu_j
    Bi = np.einsum("ijk,ik->ij", r, mu)             # mu_i . r_ij
    Bj = np.einsum("ijk,jk->ij", r, mu)             # mu_j . r_ij
    l3, l5, d3r, d5r = th["l3"], th["l5"], th["d3r"], th["d5r"]
    # coefficient of r_ij, and of mu_i / mu_j
    cr = 3.0 * Bi * Bj * (d5r * ri1 * ri5 - 5.0 * l5 * ri7) - A * (d3r * ri1 * ri3 - 3.0 * l3 * ri5)
    F = (np.einsum("ij,ijk->ik", cr, r) + 3.0 * np.einsum("ij,ik->ik", l5 * ri5 * Bj, mu)
         + 3.0 * (l5 * ri5 * Bi) @ mu)
    act = alpha > 0
    dadu = np.where(act[:, None], -th["u"] / (6.0 * np.where(act, alpha, 1.0))[:, None], 0.0)
    dA = ((3.0 * Bi * Bj * ri5 * th["d5u"] - A * ri3 * th["d3u"]) * dadu).sum(1)
    return F, dA


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
                   tol=1e-13, max_iter=500, thole=0.0):
    """U, its gradients and the dipoles for charges q, field charges qE,
    polarizabilities alpha and the excluded pairs. method: "dense" (pair sums)
    or "fmm" (CPU octree FMM at order p over all pairs, minus the excluded
    pairs' direct terms). solve: "dense" (Cholesky of diag(1/alpha) - T, T
    built column by column from the method's dipole field and symmetrised) or
    "pcg" (the preconditioned conjugate gradients of ``oracle.pcg_dipole_solve``
    on the method's dipole field as it is, to the relative residual tol).
    thole > 0: Thole damping of the dipole-dipole tensor with that a (the
    damped minus undamped terms as pair sums over the non-excluded pairs)."""
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
    th = thole_factors(r, ri, alpha, float(thole), mask) if thole > 0 else None

    def dipole_field_dd(mu):
        """the field of the dipoles as the dipoles feel it (damped when thole > 0)"""
        E = dipoles(mu)[1]
        if th is not None:
            E = E + _dipole_field_damped(r, ri, mask, mu, th) - _dipoles_undamped_E(mu)
        return E

    def _dipoles_undamped_E(mu):
        return _dipole_fields(r, ri, mask, mu)[1]

    phi_c, E_c, _ = charges(q)
    _, E_qE, G_qE = charges(qE)
    # mu = alpha (E^qE + T mu) on the polarizable sites: dense Cholesky of
    # diag(1/alpha) - T over the active sites, T applied through `dipoles`,
    # or PCG with that operator
    idx = np.nonzero(act)[0]
    mu = np.zeros((n, 3))
    if solve == "pcg":
        mu, _, _, _ = pcg_dipole_solve(alpha, E_qE, dipole_field_dd, tol=tol, max_iter=max_iter)
    elif solve != "dense":
        raise ValueError(solve)
    elif idx.size:
        k = idx.size
        T = np.zeros((3 * k, 3 * k))
        for c in range(3 * k):
            e = np.zeros((n, 3))
            e[idx[c // 3], c % 3] = 1.0
            T[:, c] = dipole_field_dd(e)[idx].ravel()
        T = 0.5 * (T + T.T)
        A = np.diag(np.repeat(1.0 / alpha[idx], 3)) - T
        try:
            L = np.linalg.cholesky(A)
        except np.linalg.LinAlgError as err:
            raise OracleError(f"dipole matrix not positive definite: {err}")
        y = np.linalg.solve(L, E_qE[idx].ravel())
        mu[idx] = np.linalg.solve(L.T, y).reshape(-1, 3)
    phi_m, E_m, G_m = dipoles(mu)
    E_dd = dipole_field_dd(mu)

    m2 = (mu * mu).sum(1)
    safe = np.where(act, alpha, 1.0)
    Uqq = 0.5 * float((q * phi_c).sum())
    Upol = float(0.5 * np.where(act, m2 / safe, 0.0).sum() - (mu * E_qE).sum() - 0.5 * (mu * E_dd).sum())

    def gmu(G):
        return np.stack([G[:, 0] * mu[:, 0] + G[:, 1] * mu[:, 1] + G[:, 2] * mu[:, 2],
                         G[:, 1] * mu[:, 0] + G[:, 3] * mu[:, 1] + G[:, 4] * mu[:, 2],
                         G[:, 2] * mu[:, 0] + G[:, 4] * mu[:, 1] + G[:, 5] * mu[:, 2]], 1)

    F = q[:, None] * E_c + qE[:, None] * E_m + gmu(G_qE) + gmu(G_m)
    dUda = np.where(act, -m2 / (2.0 * safe * safe), -0.5 * ((E_qE + E_m) ** 2).sum(1))
    if th is not None:
        # dipole-dipole terms with the damping and its derivatives, in place of
        # the undamped (grad E^mu) mu
        th0 = {k: (np.ones_like(v) if k in ("l3", "l5") else np.zeros_like(v)) for k, v in th.items()}
        Fd, dAd = _dipole_pair_gradients(r, ri, mask, mu, alpha, th)
        Fu, _ = _dipole_pair_gradients(r, ri, mask, mu, alpha, th0)
        F = F + Fd - Fu
        dUda = dUda - dAd
    return {"U": Uqq + Upol, "Uqq": Uqq, "Upol": Upol, "Upol_stationary": -0.5 * float((mu * E_qE).sum()),
            "F": F, "dUdq": phi_c, "dUdqE": phi_m, "dUdalpha": dUda, "mu": mu}
