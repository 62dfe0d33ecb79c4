"""Full-size workloads on the GPU against the CPU oracle (same order, same
tree): the six-lobe ring (300k sites, p = 6, depth 5), the hollow shell
(250k sites, p = 8; depth 5 against the oracle, the bench depth 4 for the
precision gate) and the 30k globule solved exactly as bench.py times it."""
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


@pytest.mark.parametrize("index,n,depth", [(3, None, None), (5, 250000, 5)])
def test_large_static_field_fp64_matches_oracle(index, n, depth):
    w = synth.workload(index, n=n, depth=depth)
    with PolFMM(dev(w.pos), dev(w.q), dev(w.alpha), p=w.p, depth=w.depth) as f:
        st = f.static_field()
        lo, side = f.root_box()
    ref = oracle.fmm_fields(w.pos, w.q, None, p=w.p, depth=w.depth, root=(lo, side))
    assert oracle.rel_rms(host(st["E"]), ref["E"]) < 1e-10
    assert oracle.rel_rms(host(st["phi"]), ref["phi"]) < 1e-10
    assert max_site_err(host(st["E"]), ref["E"]) < 1e-8
    assert max_site_err(host(st["phi"]), ref["phi"]) < 1e-8


@pytest.mark.parametrize("index,n", [(2, None), (3, None), (5, 250000)])
def test_large_mixed_forces_within_gate(index, n):
    """Relative RMS force error of MIXED (FP32 FMM, 3xTF32 tensor-core M2L,
    FP64 solver) against FP64, both solved to the bench tolerances."""
    from bench import tol_for

    w = synth.workload(index, n=n)
    F = {}
    for mode in ("fp64", "mixed"):
        tol = tol_for(mode, w.n)
        with PolFMM(dev(w.pos), dev(w.q), dev(w.alpha), p=w.p, depth=w.depth, mode=mode, max_iter=500) as f:
            info = f.solve(tol)
            assert info["converged"], (mode, info)
            F[mode] = host(f.energy_forces()["F"])
    assert oracle.rel_rms(F["mixed"], F["fp64"]) < 1e-5
    assert max_site_err(F["mixed"], F["fp64"]) < 1e-3


def test_globule_fp64_solve_matches_oracle_at_bench_size():
    """The bench workload end to end in FP64: the same PCG on the same FMM
    operator, so dipoles, energy and forces agree to round-off."""
    w = synth.workload(2)
    with PolFMM(dev(w.pos), dev(w.q), dev(w.alpha), p=w.p, depth=w.depth, max_iter=500) as f:
        info = f.solve(1e-8)
        out = f.energy_forces()
        mu = host(f.dipoles())
        lo, side = f.root_box()
    ref = oracle.polarizable_energy(w.pos, w.q, w.alpha, method="fmm", p=w.p, depth=w.depth, root=(lo, side),
                                    tol=1e-8, max_iter=500)
    assert info["iterations"] == ref["iterations"]
    assert oracle.rel_rms(mu, ref["mu"]) < 1e-9
    assert out["U"] == pytest.approx(ref["U"], rel=1e-10)
    assert oracle.rel_rms(host(out["F"]), ref["F"]) < 1e-9
    assert max_site_err(mu, ref["mu"]) < 1e-7
    assert max_site_err(host(out["F"]), ref["F"]) < 1e-7
