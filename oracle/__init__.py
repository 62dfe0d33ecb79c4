"""CPU FP64 oracle for the polarizable FMM (Coles & Masella, arXiv:1408.6527).

TEST INFRASTRUCTURE ONLY: the plain, slow reference that the CUDA path is
checked against.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import it; the product path never does.  It
shares no code with the CUDA library.

Heavy loops live in ``polfmm_oracle.c`` (compiled with gcc on first use);
this module adds the dense and iterative dipole solves and the energy and
gradient assembly, each citing the passage it follows.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, symbolic derivatives, exactness of the shift operators,
Newton's third law, stationarity checked by finite differences, error decay
with the expansion order).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "polfmm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

G_ORDER = ("xx", "xy", "xz", "yy", "yz", "zz")


def build(force: bool = False) -> str:
    """Compile the C oracle (plain gcc, OpenMP, strict IEEE semantics)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            ci = ctypes.c_int
            cd = ctypes.c_double
            lib.orc_direct.argtypes = [i64, P, P, P, i64, P, P, P, P]
            lib.orc_fmm.argtypes = [i64, P, P, P, ci, ci, P, cd, P, P, P]
            lib.orc_fmm_ex.argtypes = [i64, P, P, P, ci, ci, P, cd, P, P, P, ci, cd]
            lib.orc_derivatives.argtypes = [ci, P, P]
            lib.orc_multi_indices.argtypes = [ci, P]
            lib.orc_p2m.argtypes = [ci, P, i64, P, P, P, P]
            lib.orc_m2m.argtypes = [ci, P, P, P]
            lib.orc_m2l.argtypes = [ci, P, P, P]
            lib.orc_l2l.argtypes = [ci, P, P, P]
            lib.orc_l2p.argtypes = [ci, P, P, P, P, P]
            lib.orc_root_box.argtypes = [i64, P, P, P]
            lib.orc_leaf_cells.argtypes = [i64, P, ci, P, cd, P]
            lib.orc_set_num_threads.argtypes = [ci]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(k: int) -> None:
    _load().orc_set_num_threads(int(k))


class OracleError(RuntimeError):
    pass


def _check(st):
    if st == 2:
        raise OracleError("coincident sites")
    if st != 0:
        raise OracleError(f"oracle status {st}")


def ncoef(p: int) -> int:
    return (p + 1) * (p + 2) * (p + 3) // 6


def multi_indices(p: int) -> np.ndarray:
    out = np.zeros((ncoef(p), 3), dtype=np.int32)
    _check(_load().orc_multi_indices(p, _ptr(out)))
    return out


# ---------------------------------------------------------------------------
# direct sums (Sec. II.A)
# ---------------------------------------------------------------------------

def direct_fields(pos, q=None, mu=None, targets=None):
    """Phi, E and G = grad E at the sites from charges q and point dipoles mu,
    summed over all j != i (Sec. II.A; dipole field with the physical sign)."""
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    q = _f64(q)
    mu = _f64(mu, (-1, 3)) if mu is not None else None
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if tg is None else tg.shape[0]
    phi = np.zeros(nt)
    E = np.zeros((nt, 3))
    G = np.zeros((nt, 6))
    _check(_load().orc_direct(n, _ptr(pos), _ptr(q), _ptr(mu), nt, _ptr(tg), _ptr(phi), _ptr(E), _ptr(G)))
    return {"phi": phi, "E": E, "G": G}


# ---------------------------------------------------------------------------
# CPU FMM (Sec. II.B, Sec. III) on a uniform octree
# ---------------------------------------------------------------------------

def root_box(pos):
    pos = _f64(pos, (-1, 3))
    lo = np.zeros(3)
    side = np.zeros(1)
    _check(_load().orc_root_box(pos.shape[0], _ptr(pos), _ptr(lo), _ptr(side)))
    return lo, float(side[0])


def leaf_cells(pos, depth, lo, side):
    pos = _f64(pos, (-1, 3))
    lo = _f64(lo)
    cells = np.zeros((pos.shape[0], 3), dtype=np.int32)
    _check(_load().orc_leaf_cells(pos.shape[0], _ptr(pos), int(depth), _ptr(lo), float(side), _ptr(cells)))
    return cells


def fmm_fields(pos, q=None, mu=None, p=4, depth=3, root=None, fp32_top=-1, dipole_dl=0.0):
    """Phi, E, G at every site by the CPU FMM at order p on a uniform octree of
    the given depth; root = (lo, side) or None for the default root cube.
    fp32_top >= 2: the multipole shifts into levels 2..fp32_top and the local
    shifts out of them in single precision (a measurement of what single
    precision at the top of the tree costs); -1: all FP64.  dipole_dl > 0: the
    dipoles enter the multipoles as the +-q^mu pairs of Sec. II.C at that
    separation (the near field keeps the explicit dipoles); 0: analytically."""
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    q = _f64(q)
    mu = _f64(mu, (-1, 3)) if mu is not None else None
    phi = np.zeros(n)
    E = np.zeros((n, 3))
    G = np.zeros((n, 6))
    lo = None if root is None else _f64(root[0])
    side = 0.0 if root is None else float(root[1])
    _check(_load().orc_fmm_ex(n, _ptr(pos), _ptr(q), _ptr(mu), int(p), int(depth), _ptr(lo), side,
                              _ptr(phi), _ptr(E), _ptr(G), int(fp32_top), float(dipole_dl)))
    return {"phi": phi, "E": E, "G": G}


# ---------------------------------------------------------------------------
# single-box operators, exposed for the pins
# ---------------------------------------------------------------------------

def derivatives(R, p):
    out = np.zeros(ncoef(p))
    _check(_load().orc_derivatives(int(p), _ptr(_f64(R)), _ptr(out)))
    return out


def p2m(p, z, x, q=None, mu=None):
    x = _f64(x, (-1, 3))
    M = np.zeros(ncoef(p))
    _check(_load().orc_p2m(int(p), _ptr(_f64(z)), x.shape[0], _ptr(x), _ptr(_f64(q)),
                           _ptr(_f64(mu, (-1, 3)) if mu is not None else None), _ptr(M)))
    return M


def m2m(p, s, M):
    out = np.zeros(ncoef(p))
    _check(_load().orc_m2m(int(p), _ptr(_f64(s)), _ptr(_f64(M)), _ptr(out)))
    return out


def m2l(p, R, M):
    out = np.zeros(ncoef(p))
    _check(_load().orc_m2l(int(p), _ptr(_f64(R)), _ptr(_f64(M)), _ptr(out)))
    return out


def l2l(p, s, F):
    out = np.zeros(ncoef(p))
    _check(_load().orc_l2l(int(p), _ptr(_f64(s)), _ptr(_f64(F)), _ptr(out)))
    return out


def l2p(p, r, F):
    phi = np.zeros(1)
    dphi = np.zeros(3)
    ddphi = np.zeros(6)
    _check(_load().orc_l2p(int(p), _ptr(_f64(r)), _ptr(_f64(F)), _ptr(phi), _ptr(dphi), _ptr(ddphi)))
    return float(phi[0]), dphi, ddphi


# ---------------------------------------------------------------------------
# induced dipoles (Eq. dipole moment, Sec. II.A) and energies
# ---------------------------------------------------------------------------

def dipole_matrix(pos):
    """Dense 3N x 3N T with blocks T_ij = (3 r r^T / r^2 - 1) / r^3 (i != j), so
    that E^mu = T mu is the physical dipole field; zero diagonal blocks."""
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    r = pos[:, None, :] - pos[None, :, :]
    r2 = np.einsum("ijk,ijk->ij", r, r)
    np.fill_diagonal(r2, 1.0)
    ri = 1.0 / np.sqrt(r2)
    ri3 = ri ** 3
    ri5 = ri3 * ri * ri
    T = 3.0 * r[:, :, :, None] * r[:, :, None, :] * ri5[:, :, None, None] - np.eye(3)[None, None] * ri3[:, :, None, None]
    idx = np.arange(n)
    T[idx, idx] = 0.0
    return T.transpose(0, 2, 1, 3).reshape(3 * n, 3 * n)


def dense_dipole_solve(pos, alpha, Eq):
    """Solve mu = alpha (E^q + T mu), i.e. (diag(1/alpha) - T) mu = E^q, by a
    dense Cholesky factorisation (sites with alpha = 0 carry no dipole).
    Raises OracleError if the matrix is not positive definite (the
    polarization catastrophe)."""
    import scipy.linalg as sla

    alpha = _f64(alpha)
    Eq = _f64(Eq, (-1, 3))
    act = np.nonzero(alpha > 0)[0]
    mu = np.zeros_like(Eq)
    if act.size == 0:
        return mu
    T = dipole_matrix(_f64(pos, (-1, 3))[act])
    A = np.diag(np.repeat(1.0 / alpha[act], 3)) - T
    try:
        c = sla.cho_factor(A, lower=True, check_finite=True)
    except np.linalg.LinAlgError as e:
        raise OracleError(f"dipole matrix not positive definite: {e}")
    mu[act] = sla.cho_solve(c, Eq[act].ravel()).reshape(-1, 3)
    return mu


def pcg_dipole_solve(alpha, Eq, apply_T, tol=1e-8, max_iter=100, mu0=None):
    """Preconditioned conjugate gradients on (diag(1/alpha) - T) mu = E^q with
    the Jacobi preconditioner diag(alpha), started from mu0 = alpha E^q
    (the first step of the fixed point of Eq. dipole moment).

    apply_T(v) returns the dipole field T v at all sites.  Stops when
    ||r|| / ||E^q|| <= tol (checked before each iteration) or after max_iter
    iterations.  Returns (mu, iterations, relative residual, history)."""
    alpha = _f64(alpha)
    Eq = _f64(Eq, (-1, 3))
    act = (alpha > 0)[:, None]
    a3 = np.where(act, alpha[:, None], 0.0)
    inv_a3 = np.where(act, 1.0 / np.where(act, alpha[:, None], 1.0), 0.0)
    mu = a3 * Eq if mu0 is None else np.where(act, _f64(mu0, (-1, 3)), 0.0)
    bnorm = np.sqrt(np.sum(np.where(act, Eq, 0.0) ** 2))
    if bnorm == 0.0:
        return np.zeros_like(Eq), 0, 0.0, [0.0]
    r = np.where(act, Eq - (inv_a3 * mu - apply_T(mu)), 0.0)
    z = a3 * r
    d = z.copy()
    rz = np.sum(r * z)
    hist = [float(np.sqrt(np.sum(r * r)) / bnorm)]
    it = 0
    while it < max_iter and hist[-1] > tol:
        Ad = np.where(act, inv_a3 * d - apply_T(d), 0.0)
        dAd = np.sum(d * Ad)
        a = rz / dAd
        mu = mu + a * d
        r = r - a * Ad
        z = a3 * r
        rz_new = np.sum(r * z)
        beta = rz_new / rz
        rz = rz_new
        d = z + beta * d
        it += 1
        hist.append(float(np.sqrt(np.sum(r * r)) / bnorm))
    return mu, it, hist[-1], hist


def energy_terms(q, alpha, mu, phi_q, Eq, Emu):
    """U^qq' = 1/2 sum q_i Phi^q_i (Eq. equ:Uqq) and
    U^pol = A(mu) - sum mu.E^q - 1/2 sum mu.E^mu with A = 1/2 sum |mu|^2/alpha
    (Sec. II.A); sites with alpha = 0 carry no dipole and no A term."""
    q = _f64(q)
    alpha = _f64(alpha)
    mu = _f64(mu, (-1, 3))
    m2 = np.sum(mu * mu, axis=1)
    A = 0.5 * np.sum(np.where(alpha > 0, m2 / np.where(alpha > 0, alpha, 1.0), 0.0))
    Uqq = 0.5 * np.sum(q * phi_q)
    Upol = A - np.sum(mu * Eq) - 0.5 * np.sum(mu * Emu)
    return Uqq, Upol


def gradients(q, alpha, mu, tot):
    """Forces and parameter gradients at a stationary point (Eq.
    upol_derivatives): F_i = q_i E_i + (grad E_i) mu_i with E the total field of
    charges and dipoles; dU/dq_i = Phi_i (total potential);
    dU/dalpha_i = -|mu_i|^2 / (2 alpha_i^2) (= -|E_i|^2/2 at convergence,
    which is used where alpha_i = 0)."""
    q = _f64(q)
    alpha = _f64(alpha)
    mu = _f64(mu, (-1, 3))
    E, G, phi = tot["E"], tot["G"], tot["phi"]
    Gm = np.stack([
        G[:, 0] * mu[:, 0] + G[:, 1] * mu[:, 1] + G[:, 2] * mu[:, 2],
        G[:, 1] * mu[:, 0] + G[:, 3] * mu[:, 1] + G[:, 4] * mu[:, 2],
        G[:, 2] * mu[:, 0] + G[:, 4] * mu[:, 1] + G[:, 5] * mu[:, 2],
    ], 1)
    F = q[:, None] * E + Gm
    m2 = np.sum(mu * mu, axis=1)
    safe = np.where(alpha > 0, alpha, 1.0)
    dUda = np.where(alpha > 0, -m2 / (2.0 * safe * safe), -0.5 * np.sum(E * E, axis=1))
    return F, phi.copy(), dUda


def polarizable_energy(pos, q, alpha, method="direct", p=4, depth=3, root=None, tol=1e-12,
                       max_iter=500, solve="pcg", mu0=None, coulomb_k=1.0, dipole_dl=0.0):
    """Whole path on the CPU: static field, induced dipoles, energy and gradients.

    method: "direct" (O(N^2) sums) or "fmm" (CPU FMM at order p and depth).
    solve: "pcg" (PCG as in pcg_dipole_solve), "dense" (Cholesky; direct only).
    dipole_dl (fmm): the dipoles' multipoles from +-q pairs (Sec. II.C)."""
    pos = _f64(pos, (-1, 3))
    q = _f64(q)
    alpha = _f64(alpha)

    if method == "direct":
        field = lambda qq, mm: direct_fields(pos, qq, mm)
    elif method == "fmm":
        field = lambda qq, mm: fmm_fields(pos, qq, mm, p=p, depth=depth, root=root, dipole_dl=dipole_dl)
    else:
        raise ValueError(method)
    st = field(q, None)
    Eq, phi_q = st["E"], st["phi"]
    info = {}
    if solve == "dense":
        mu = dense_dipole_solve(pos, alpha, Eq)
        info.update(iterations=0, residual=0.0)
    else:
        mu, it, res, hist = pcg_dipole_solve(alpha, Eq, lambda v: field(None, v)["E"], tol=tol,
                                             max_iter=max_iter, mu0=mu0)
        info.update(iterations=it, residual=res, history=hist)
    tot = field(q, mu)
    Emu = tot["E"] - Eq
    Uqq, Upol = energy_terms(q, alpha, mu, phi_q, Eq, Emu)
    F, dUdq, dUda = gradients(q, alpha, mu, tot)
    k = float(coulomb_k)
    return {
        "U": k * (Uqq + Upol), "Uqq": k * Uqq, "Upol": k * Upol,
        "Upol_stationary": -0.5 * k * float(np.sum(mu * Eq)),
        "F": k * F, "dUdq": k * dUdq, "dUdalpha": k * dUda,
        "mu": mu, "Eq": Eq, "phi_q": phi_q, "Emu": Emu, "tot": tot, **info,
    }


def rel_rms(a, b):
    """sqrt(sum |a - b|^2 / sum |b|^2): the relative RMS error used for forces."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.sum(b * b)
    return float(np.sqrt(np.sum((a - b) ** 2) / den)) if den > 0 else float(np.sqrt(np.sum((a - b) ** 2)))


def per_site_rel_err(a, b):
    """f_err_i = |a_i - b_i| / |b_i| (Eq. error, Sec. IV)."""
    a = np.asarray(a).reshape(len(a), -1)
    b = np.asarray(b).reshape(len(b), -1)
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)
