"""Polarizable fast multipole method on one GB300 GPU.

Python binding of the C ABI in include/polfmm.h (Coles & Masella,
arXiv:1408.6527): FMM potential, field and field gradient of point charges and
induced point dipoles (Sec. II.B, II.C), the self-consistent dipole solve
(Sec. II.A, Eq. dipole moment) and the energy and forces (Sec. III).  Every step
runs in the CUDA library; this module only marshals arguments.  Tensors on a
CUDA device are passed as device pointers on the current torch stream; numpy
arrays are passed as host buffers (copies then happen inside the library).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (FP64, M2L_AUTO, M2L_FFMA, M2L_SIMT, M2L_TENSOR, MIXED, SOLVER_JACOBI, SOLVER_PCG, Options,
                   PolFMMError)

__all__ = ["PolFMM", "PolFMMError", "build", "polarizable_energy", "FP64", "MIXED"]

_MODES = {"fp64": FP64, "mixed": MIXED, FP64: FP64, MIXED: MIXED}
_SOLVERS = {"pcg": SOLVER_PCG, "jacobi": SOLVER_JACOBI}
_M2L = {"auto": M2L_AUTO, "simt": M2L_SIMT, "tensor": M2L_TENSOR, "ffma": M2L_FFMA}


def build(force: bool = False) -> str:
    """Compile libpolfmm.so for sm_103a (nvcc) in the package directory."""
    from . import _build

    return _build.build(force=force)


def _is_torch(x):
    try:
        import torch
    except ImportError:  # pragma: no cover
        return False
    return isinstance(x, torch.Tensor)


class _Buf:
    """A float64 / int32 buffer given to the C ABI (device tensor or host array)."""

    def __init__(self, x, device, dtype="f8", shape=None):
        if device:
            import torch

            tdt = torch.float64 if dtype == "f8" else torch.int32
            t = torch.as_tensor(x, dtype=tdt, device="cuda") if not _is_torch(x) else x
            if t.dtype != tdt or not t.is_cuda:
                t = t.to(device="cuda", dtype=tdt)
            t = t.contiguous()
            if shape is not None:
                t = t.reshape(shape)
            self.obj = t
            self.ptr = ctypes.c_void_p(t.data_ptr())
        else:
            a = np.ascontiguousarray(x.detach().cpu().numpy() if _is_torch(x) else x,
                                     dtype=np.float64 if dtype == "f8" else np.int32)
            if shape is not None:
                a = a.reshape(shape)
            self.obj = a
            self.ptr = a.ctypes.data_as(ctypes.c_void_p)


class PolFMM:
    """One octree, its static pass and the induced dipoles (an opaque C context)."""

    def __init__(self, pos, q, alpha, p=6, depth=4, mode="fp64", solver="pcg", max_iter=100, coulomb_k=1.0,
                 root_box=None, m2l="auto", profile=False, stream=None, graphs=True, dipole_dl=0.0,
                 pdl=True, dipole_tree=False):
        self.lib = _lib.load()
        self.device = _is_torch(pos) and pos.is_cuda
        self.n = int(pos.shape[0])
        opt = Options()
        self.lib.fmm_default_options(ctypes.byref(opt))
        opt.mode = _MODES[mode]
        opt.solver = _SOLVERS[solver]
        opt.max_iter = int(max_iter)
        opt.coulomb_k = float(coulomb_k)
        opt.m2l_impl = _M2L[m2l]
        opt.profile = int(bool(profile))
        opt.no_graphs = int(not graphs)
        opt.dipole_dl = float(dipole_dl)
        opt.no_pdl = int(not pdl)
        opt.dipole_tree = int(bool(dipole_tree))
        if root_box is not None:
            opt.use_root_box = 1
            for d in range(3):
                opt.root_lo[d] = float(root_box[0][d])
            opt.root_side = float(root_box[1])
        if stream is None and self.device:
            import torch

            stream = torch.cuda.current_stream().cuda_stream
        opt.cuda_stream = ctypes.c_void_p(stream or 0)
        self.opt = opt
        self.mode = mode
        self.p, self.depth = int(p), int(depth)
        bx = _Buf(pos, self.device, shape=(self.n, 3))
        bq = _Buf(q, self.device, shape=(self.n,))
        ba = _Buf(alpha, self.device, shape=(self.n,))
        h = ctypes.c_void_p()
        st = self.lib.fmm_build(ctypes.byref(h), self.n, bx.ptr, bq.ptr, ba.ptr, self.p, self.depth,
                                ctypes.byref(opt), int(self.device))
        _lib.check(st, "fmm_build")
        self.h = h

    # -- helpers ---------------------------------------------------------------
    def _out(self, *shape, dtype="f8"):
        if self.device:
            import torch

            t = torch.empty(shape, dtype=torch.float64 if dtype == "f8" else torch.int32, device="cuda")
            return t, ctypes.c_void_p(t.data_ptr())
        a = np.empty(shape, dtype=np.float64 if dtype == "f8" else np.int32)
        return a, a.ctypes.data_as(ctypes.c_void_p)

    def _in(self, x, shape):
        return _Buf(x, self.device, shape=shape)

    def close(self):
        if getattr(self, "h", None):
            self.lib.fmm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- the three stages --------------------------------------------------------
    def solve(self, tol=1e-8, raise_on_nonconvergence=False):
        it = ctypes.c_int()
        res = ctypes.c_double()
        st = self.lib.fmm_solve_induced_dipoles(self.h, float(tol), ctypes.byref(it), ctypes.byref(res))
        _lib.check(st, "fmm_solve_induced_dipoles", allow=() if raise_on_nonconvergence else (_lib.ERR_NOT_CONVERGED,))
        return {"iterations": it.value, "residual": res.value, "converged": st == _lib.OK, "status": st}

    def energy_forces(self, forces=True, dq=True, dalpha=True):
        e = np.zeros(3)
        F, pF = self._out(self.n, 3) if forces else (None, None)
        Q, pQ = self._out(self.n) if dq else (None, None)
        A, pA = self._out(self.n) if dalpha else (None, None)
        st = self.lib.fmm_energy_forces(self.h, e.ctypes.data_as(ctypes.c_void_p), pF, pQ, pA, int(self.device))
        _lib.check(st, "fmm_energy_forces")
        return {"U": float(e[0]), "Uqq": float(e[1]), "Upol": float(e[2]), "F": F, "dUdq": Q, "dUdalpha": A}

    def energy(self):
        """Stationary energy [U, U^qq', U^pol] at the current (converged) dipoles,
        reduced in the library (no force pass)."""
        e = np.zeros(3)
        _lib.check(self.lib.fmm_energy(self.h, e.ctypes.data_as(ctypes.c_void_p)), "fmm_energy")
        return {"U": float(e[0]), "Uqq": float(e[1]), "Upol": float(e[2])}

    # -- accessors ----------------------------------------------------------------
    def dipoles(self):
        out, p = self._out(self.n, 3)
        _lib.check(self.lib.fmm_get_dipoles(self.h, p, int(self.device)), "fmm_get_dipoles")
        return out

    def set_dipoles(self, mu):
        b = self._in(mu, (self.n, 3))
        _lib.check(self.lib.fmm_set_dipoles(self.h, b.ptr, int(self.device)), "fmm_set_dipoles")

    def reset_dipoles(self):
        _lib.check(self.lib.fmm_reset_dipoles(self.h), "fmm_reset_dipoles")

    def update_positions(self, pos):
        b = self._in(pos, (self.n, 3))
        _lib.check(self.lib.fmm_update_positions(self.h, b.ptr, int(self.device)), "fmm_update_positions")

    def set_field_charges(self, qE):
        """Field charges q^E (Sec. III): the charges whose field polarizes the sites."""
        b = self._in(qE, (self.n,))
        _lib.check(self.lib.fmm_set_field_charges(self.h, b.ptr, int(self.device)), "fmm_set_field_charges")

    def set_exclusions(self, pairs):
        """Excluded site pairs (Sec. II.A starred sums), an (m, 2) integer array of caller indices."""
        arr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        _lib.check(self.lib.fmm_set_exclusions(self.h, int(arr.shape[0]), arr.ctypes.data_as(ctypes.c_void_p), 0),
                   "fmm_set_exclusions")

    def set_dipole_predictor(self, order):
        """Start of the next solve after update_positions: 0 = last dipoles,
        1 = linear extrapolation from the last two."""
        _lib.check(self.lib.fmm_set_dipole_predictor(self.h, int(order)), "fmm_set_dipole_predictor")

    def set_thole(self, a):
        """Thole damping of the dipole-dipole interaction with parameter a (0 = off)."""
        _lib.check(self.lib.fmm_set_thole(self.h, float(a)), "fmm_set_thole")

    def field_charge_gradient(self):
        """dU/dq^E of the last energy_forces() with field charges set."""
        out, p = self._out(self.n)
        _lib.check(self.lib.fmm_field_charge_gradient(self.h, p, int(self.device)), "fmm_field_charge_gradient")
        return out

    def static_field(self):
        phi, pp = self._out(self.n)
        E, pe = self._out(self.n, 3)
        _lib.check(self.lib.fmm_static_field(self.h, pp, pe, int(self.device)), "fmm_static_field")
        return {"phi": phi, "E": E}

    def dipole_field(self, mu):
        b = self._in(mu, (self.n, 3))
        E, pe = self._out(self.n, 3)
        _lib.check(self.lib.fmm_dipole_field(self.h, b.ptr, pe, int(self.device)), "fmm_dipole_field")
        return E

    def total_field(self, mu=None):
        b = self._in(mu, (self.n, 3)) if mu is not None else None
        phi, pp = self._out(self.n)
        E, pe = self._out(self.n, 3)
        G, pg = self._out(self.n, 6)
        _lib.check(self.lib.fmm_total_field(self.h, b.ptr if b else None, pp, pe, pg, int(self.device)),
                   "fmm_total_field")
        return {"phi": phi, "E": E, "G": G}

    def leaf_cells(self):
        out, p = self._out(self.n, 3, dtype="i4")
        _lib.check(self.lib.fmm_leaf_cells(self.h, p, int(self.device)), "fmm_leaf_cells")
        return out

    def tree_info(self):
        info = np.zeros(11, dtype=np.int64)
        _lib.check(self.lib.fmm_tree_info(self.h, info.ctypes.data_as(ctypes.c_void_p)), "fmm_tree_info")
        d = int(info[0])
        return {"depth": d, "p": int(info[1]), "boxes": [int(v) for v in info[2:3 + d]]}

    def root_box(self):
        lo = np.zeros(3)
        side = np.zeros(1)
        _lib.check(self.lib.fmm_root_box(self.h, lo.ctypes.data_as(ctypes.c_void_p),
                                         side.ctypes.data_as(ctypes.c_void_p)), "fmm_root_box")
        return lo, float(side[0])

    def profile(self, family):
        ms = ctypes.c_double()
        k = ctypes.c_int64()
        _lib.check(self.lib.fmm_profile_get(self.h, family.encode(), ctypes.byref(ms), ctypes.byref(k)),
                   "fmm_profile_get")
        return ms.value, k.value

    def profile_reset(self):
        _lib.check(self.lib.fmm_profile_reset(self.h), "fmm_profile_reset")

    def launch_count(self) -> int:
        return int(self.lib.fmm_launch_count(self.h))


def kdtree_fields(pos, q=None, mu=None, p=5, theta=0.5, n_bucket=8, n_direct=64, pad=1e-3, dipole_dl=0.0,
                  stream=None):
    """Phi, E, G at every site by the adaptive kd-tree FMM of Sec. III on the
    GPU (FP64, fmm_kdtree_fields), and the walk's counts."""
    lib = _lib.load()
    device = _is_torch(pos) and pos.is_cuda
    n = int(pos.shape[0])
    if stream is None and device:
        import torch

        stream = torch.cuda.current_stream().cuda_stream
    bx = _Buf(pos, device, shape=(n, 3))
    bq = _Buf(q, device, shape=(n,)) if q is not None else None
    bm = _Buf(mu, device, shape=(n, 3)) if mu is not None else None
    if device:
        import torch

        outs = [torch.empty(s, dtype=torch.float64, device="cuda") for s in ((n,), (n, 3), (n, 6))]
        ptrs = [ctypes.c_void_p(t.data_ptr()) for t in outs]
    else:
        outs = [np.empty(s) for s in ((n,), (n, 3), (n, 6))]
        ptrs = [a.ctypes.data_as(ctypes.c_void_p) for a in outs]
    stats = np.zeros(5, dtype=np.int64)
    _lib.check(lib.fmm_kdtree_fields(n, bx.ptr, bq.ptr if bq else None, bm.ptr if bm else None, int(p), float(theta),
                                     int(n_bucket), int(n_direct), float(pad), float(dipole_dl), *ptrs,
                                     stats.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(stream or 0),
                                     int(device)), "fmm_kdtree_fields")
    return {"phi": outs[0], "E": outs[1], "G": outs[2],
            "stats": dict(zip(("cells", "leaves", "levels", "multipole_pairs", "direct_pairs"), stats.tolist()))}


def measure_peak(kind: str, stream=None) -> float:
    """Measured FP32 ("fp32") or FP64 ("fp64") fused multiply-add peak of the
    current device in TFLOP/s (for roofline fractions)."""
    lib = _lib.load()
    v = ctypes.c_double()
    _lib.check(lib.fmm_measure_peak({"fp32": 0, "fp64": 1}[kind], ctypes.c_void_p(stream or 0), ctypes.byref(v)),
               "fmm_measure_peak")
    return v.value


from .autograd import polarizable_energy  # noqa: E402
