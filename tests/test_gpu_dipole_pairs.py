"""The +-q pair form of the point dipoles on the GPU (Sec. II.C, mu = 2 |q^mu| dl;
NEXT-4): FP64 parity with the oracle's pair form, the options it refuses, and
the paper's dl sweep on its sphere test (Fig. pol-radius: no difference in the
force errors from 1e-5 to 1e-1 A)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1408_6527_gb300 import PolFMM, PolFMMError  # noqa: E402
from paper_1408_6527_gb300 import _lib  # noqa: E402
from siteerr import max_site_err  # noqa: E402


def dev(a):
    return torch.as_tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("dl", [1e-4, 1e-2])
def test_pair_dipole_field_matches_the_oracle(dl):
    w = synth.workload(1)
    mu = 0.3 * np.random.default_rng(3).normal(size=(w.n, 3))
    with PolFMM(dev(w.pos), dev(w.q), dev(w.alpha), p=6, depth=3, dipole_dl=dl) as f:
        out = f.total_field(dev(mu))
        lo, side = f.root_box()
    ref = oracle.fmm_fields(w.pos, w.q, mu, p=6, depth=3, root=(lo, side), dipole_dl=dl)
    for k in ("phi", "E", "G"):
        assert oracle.rel_rms(host(out[k]), ref[k]) < 1e-10, k
        assert max_site_err(host(out[k]), ref[k]) < 1e-8, k


def test_pair_dipoles_converged_solve_and_forces_match_the_oracle():
    w = synth.workload(1)
    with PolFMM(dev(w.pos), dev(w.q), dev(w.alpha), p=5, depth=3, dipole_dl=1e-3) as f:
        assert f.solve(1e-12)["converged"]
        out = f.energy_forces()
        mu = host(f.dipoles())
        lo, side = f.root_box()
    ref = oracle.polarizable_energy(w.pos, w.q, w.alpha, method="fmm", p=5, depth=3, root=(lo, side), tol=1e-13,
                                    dipole_dl=1e-3)
    assert oracle.rel_rms(mu, ref["mu"]) < 1e-9
    assert out["U"] == pytest.approx(ref["U"], rel=1e-10)
    for k in ("F", "dUdq", "dUdalpha"):
        assert oracle.rel_rms(host(out[k]), ref[k]) < 1e-9, k


def test_pair_form_options_that_are_refused():
    w = synth.workload(1)
    # FP32 arithmetic would cancel the pair's multipole catastrophically
    with pytest.raises(PolFMMError) as e:
        PolFMM(dev(w.pos), dev(w.q), dev(w.alpha), p=4, depth=3, mode="mixed", dipole_dl=1e-4)
    assert e.value.status == _lib.ERR_INVALID_ARG
    for dl in (-1e-4, float("nan"), 5.0):  # 5 A is more than a quarter of the leaf side
        with pytest.raises(PolFMMError) as e:
            PolFMM(dev(w.pos), dev(w.q), dev(w.alpha), p=4, depth=3, dipole_dl=dl)
        assert e.value.status == _lib.ERR_INVALID_ARG


def test_dl_sweep_on_the_sphere_test():
    """Sec. IV.A's sphere (4,096 sites, r = 45 A, 2 A apart, charges +-[0.1, 0.8])
    with dipoles mu = E^q (alpha = 1, one induction step, the paper's
    'without polarization' case of Fig. pol-radius). The per-atom relative
    force error against the direct sum does not depend on dl over five orders
    of magnitude."""
    rng = np.random.default_rng(11)
    pos = synth.sites_sphere(rng, 4096, 45.0, 2.0)
    q = synth.charges_uniform_pm(rng, 4096)
    alpha = np.ones(4096)
    Eq = oracle.direct_fields(pos, q)["E"]
    mu = Eq.copy()
    d = oracle.direct_fields(pos, q, mu)
    Fd = q[:, None] * d["E"] + np.einsum("nij,nj->ni", _sym(d["G"]), mu)
    p80 = {}
    for dl in (0.0, 1e-5, 1e-4, 1e-3, 1e-2, 1e-1):
        with PolFMM(dev(pos), dev(q), dev(alpha), p=5, depth=4, dipole_dl=dl) as f:
            out = f.total_field(dev(mu))
        F = q[:, None] * host(out["E"]) + np.einsum("nij,nj->ni", _sym(host(out["G"])), mu)
        err = np.linalg.norm(F - Fd, axis=1) / np.linalg.norm(Fd, axis=1)
        p80[dl] = float(np.percentile(err, 80))
    print("80th percentile of the per-atom relative force error by dl:", p80)
    for dl in (1e-5, 1e-4, 1e-3, 1e-2, 1e-1):
        assert abs(p80[dl] - p80[0.0]) <= 0.02 * p80[0.0], (dl, p80)


def _sym(G):
    """(n, 6) xx xy xz yy yz zz -> (n, 3, 3)."""
    xx, xy, xz, yy, yz, zz = G.T
    return np.stack([np.stack([xx, xy, xz], -1), np.stack([xy, yy, yz], -1), np.stack([xz, yz, zz], -1)], -2)
