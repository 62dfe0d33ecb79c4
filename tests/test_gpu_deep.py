"""Parity at the tree depths the large workloads run at (depth 6 for the 4M
shell) and at the library's limit (depth 8): dense key -> slot maps of 8^l
entries, mostly empty boxes, every leaf holding one or two sites, and
tensor-core tiles whose rows mix levels 2 .. depth.

FP64 against the CPU oracle's FMM on the same tree (per site and in norm);
MIXED (FP32 + 3xTF32 tensor-core M2L) against the oracle directly and against
the FP64 path, and the precision gate (1e-5 relative RMS force error) on the
4M-site shell at its bench depth 6, with the energy and dipole errors.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1408_6527_gb300 import PolFMM  # noqa: E402
from siteerr import max_site_err  # noqa: E402


def dev(a):
    return torch.as_tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


# (workload index, sites, depth, p): hollow shells of 20k sites, whose deep
# leaves hold about one site each, and the 100k globule at depth 6
DEEP = [(5, 20000, 6, 5), (5, 20000, 7, 4), (5, 20000, 8, 3), (4, None, 6, 4)]


@pytest.mark.parametrize("index,n,depth,p", DEEP)
def test_deep_static_and_dipole_field_fp64(index, n, depth, p):
    w = synth.workload(index, n=n, depth=depth)
    mu = 0.2 * np.random.default_rng(depth).normal(size=(w.n, 3))
    with PolFMM(dev(w.pos), dev(w.q), dev(w.alpha), p=p, depth=depth) as f:
        st = f.static_field()
        Emu = host(f.dipole_field(dev(mu)))
        lo, side = f.root_box()
        info = f.tree_info()
    cells = oracle.leaf_cells(w.pos, depth, lo, side)
    for l in range(depth + 1):
        c = cells >> (depth - l)
        assert info["boxes"][l] == len(np.unique(c[:, 0] + (1 << l) * (c[:, 1] + (1 << l) * c[:, 2])))
    ref = oracle.fmm_fields(w.pos, w.q, None, p=p, depth=depth, root=(lo, side))
    refm = oracle.fmm_fields(w.pos, None, mu, p=p, depth=depth, root=(lo, side))
    for a, b in ((host(st["E"]), ref["E"]), (host(st["phi"]), ref["phi"]), (Emu, refm["E"])):
        assert oracle.rel_rms(a, b) < 1e-10
        assert max_site_err(a, b) < 1e-8


@pytest.mark.parametrize("index,n,depth,p", DEEP + [(2, None, 4, 6)])
def test_deep_mixed_against_oracle_and_fp64(index, n, depth, p):
    """MIXED straight against the oracle: the FP32 expansions and the 3xTF32
    tensor-core M2L carry FP32-level error (a few 1e-7 relative RMS)."""
    w = synth.workload(index, n=n, depth=depth)
    mu = 0.2 * np.random.default_rng(depth).normal(size=(w.n, 3))
    out = {}
    for mode in ("mixed", "fp64"):
        with PolFMM(dev(w.pos), dev(w.q), dev(w.alpha), p=p, depth=depth, mode=mode) as f:
            out[mode] = (host(f.static_field()["E"]), host(f.dipole_field(dev(mu))))
            lo, side = f.root_box()
    ref = oracle.fmm_fields(w.pos, w.q, None, p=p, depth=depth, root=(lo, side))["E"]
    refm = oracle.fmm_fields(w.pos, None, mu, p=p, depth=depth, root=(lo, side))["E"]
    for got, want in ((out["mixed"][0], ref), (out["mixed"][1], refm)):
        assert oracle.rel_rms(got, want) < 2e-6
        assert max_site_err(got, want) < 1e-4
    assert oracle.rel_rms(out["fp64"][0], ref) < 1e-10


def test_shell_4m_mixed_gate_at_depth_6():
    """The headline precision gate on the largest workload at its bench depth:
    MIXED against FP64 on the same tree, both solved to the bench tolerances;
    the energy and dipole errors are reported beside the force error."""
    from bench import tol_for

    w = synth.workload(5, n=4000000)
    assert w.depth == 6 and w.p == 8
    res = {}
    for mode in ("fp64", "mixed"):
        with PolFMM(dev(w.pos), dev(w.q), dev(w.alpha), p=w.p, depth=w.depth, mode=mode, max_iter=500) as f:
            info = f.solve(tol_for(mode, w.n))
            assert info["converged"], (mode, info)
            out = f.energy_forces(dq=False, dalpha=False)
            res[mode] = (host(out["F"]), host(f.dipoles()), out["U"])
    F64, mu64, U64 = res["fp64"]
    Fmx, mumx, Umx = res["mixed"]
    err_F = oracle.rel_rms(Fmx, F64)
    err_mu = oracle.rel_rms(mumx, mu64)
    err_U = abs(Umx - U64) / abs(U64)
    print(f"4M shell depth 6: force {err_F:.2e}, dipoles {err_mu:.2e}, energy {err_U:.2e}, "
          f"worst site force {max_site_err(Fmx, F64):.2e}")
    assert err_F < 1e-5
    assert err_mu < 1e-5
    assert err_U < 1e-6
