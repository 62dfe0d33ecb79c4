"""Gradients of the energy through the autograd Function (Sec. III, third
stage; Eq. upol_derivatives): the backward FMM pass against central finite
differences of the GPU energy with the dipoles re-solved, and against the
oracle's analytic gradients.  The root cube is fixed so that no site changes
leaf under the perturbation."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1408_6527_gb300 import polarizable_energy  # noqa: E402


def _setup(n=400, seed=61):
    pos, q, alpha = synth.small_random(seed, n, box=16.0)
    lo, side = oracle.root_box(pos)
    return pos, q, alpha, (lo - 0.5, side + 1.0)


@pytest.mark.parametrize("keep_context", [True, False])
def test_autograd_gradients_match_oracle(keep_context):
    pos, q, alpha, root = _setup()
    x = torch.tensor(pos, device="cuda", requires_grad=True)
    qq = torch.tensor(q, device="cuda", requires_grad=True)
    aa = torch.tensor(alpha, device="cuda", requires_grad=True)
    U = polarizable_energy(x, qq, aa, p=6, depth=3, tol=1e-12, root_box=root, keep_context=keep_context)
    U.backward()
    ref = oracle.polarizable_energy(pos, q, alpha, method="fmm", p=6, depth=3, root=root, tol=1e-13)
    assert U.item() == pytest.approx(ref["U"], rel=1e-10)
    assert oracle.rel_rms(-x.grad.cpu().numpy(), ref["F"]) < 1e-8
    assert oracle.rel_rms(qq.grad.cpu().numpy(), ref["dUdq"]) < 1e-8
    assert oracle.rel_rms(aa.grad.cpu().numpy(), ref["dUdalpha"]) < 1e-8


def test_autograd_gradients_match_finite_differences():
    pos, q, alpha, root = _setup()
    x = torch.tensor(pos, device="cuda", requires_grad=True)
    qq = torch.tensor(q, device="cuda", requires_grad=True)
    aa = torch.tensor(alpha, device="cuda", requires_grad=True)
    U = polarizable_energy(x, qq, aa, p=6, depth=3, tol=1e-13, root_box=root)
    U.backward()
    gx, gq, ga = x.grad.cpu().numpy(), qq.grad.cpu().numpy(), aa.grad.cpu().numpy()

    def energy(p_, q_, a_):
        with torch.no_grad():
            return polarizable_energy(torch.tensor(p_, device="cuda"), torch.tensor(q_, device="cuda"),
                                      torch.tensor(a_, device="cuda"), p=6, depth=3, tol=1e-13,
                                      root_box=root).item()

    h = 1e-5
    hcell = root[1] / 8
    rng = np.random.default_rng(7)
    checked = 0
    for i in rng.permutation(len(q)):
        u = (pos[i] - root[0]) / hcell
        if np.min(np.abs(u - np.round(u))) < 1e-3:
            continue
        for d in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, d] += h
            pm[i, d] -= h
            fd = (energy(pp, q, alpha) - energy(pm, q, alpha)) / (2 * h)
            assert gx[i, d] == pytest.approx(fd, rel=1e-5, abs=1e-7)
        qp, qm = q.copy(), q.copy()
        qp[i] += h
        qm[i] -= h
        assert gq[i] == pytest.approx((energy(pos, qp, alpha) - energy(pos, qm, alpha)) / (2 * h), rel=1e-5, abs=1e-7)
        ap, am = alpha.copy(), alpha.copy()
        ap[i] += h
        am[i] -= h
        assert ga[i] == pytest.approx((energy(pos, q, ap) - energy(pos, q, am)) / (2 * h), rel=1e-5, abs=1e-7)
        checked += 1
        if checked == 6:
            break
    assert checked == 6


def test_second_backward_reuses_the_gradients():
    """retain_graph=True: a second backward gives the same gradients (the force
    pass runs once; its results are kept)."""
    pos, q, alpha, root = _setup(n=200, seed=62)
    x = torch.tensor(pos, device="cuda", requires_grad=True)
    U = polarizable_energy(x, torch.tensor(q, device="cuda"), torch.tensor(alpha, device="cuda"), p=4, depth=3,
                           tol=1e-12, root_box=root)
    U.backward(retain_graph=True)
    g1 = x.grad.clone()
    x.grad = None
    (2.0 * U).backward()
    torch.testing.assert_close(x.grad, 2.0 * g1, rtol=0, atol=0)
