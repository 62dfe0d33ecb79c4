"""The adaptive kd-tree FMM of Sec. III on the GPU (NEXT-1: the paper's own
tree, Eq. mac and the mutual dual-tree walk), in FP64, against the kd-tree
oracle: the same cells, the same walk counts, the same fields to round-off,
with charges, dipoles and the +-q pair form; the sphere test's accuracy; edge
cases; and the cost against the octree on the 30k globule."""
import json
import os
import time

import numpy as np
import pytest

import oracle
import synth
from oracle import kdtree

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1408_6527_gb300 import PolFMM, PolFMMError, _lib, kdtree_fields  # noqa: E402
from siteerr import max_site_err  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sphere(seed, n, radius):
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = synth.sites_sphere(rng, n, radius, 2.0)
    return pos, synth.charges_pm_equal(rng, pos.shape[0])


def _oracle_counts(pos, theta, n_bucket, n_direct):
    root = kdtree.build_tree(pos, n_bucket)
    cells = kdtree.cells(root)
    direct, multi = kdtree.walk(root, theta, n_direct)
    return {"cells": len(cells), "leaves": sum(c.leaf for c in cells), "multipole_pairs": len(multi),
            "direct_pairs": len(direct)}


@pytest.mark.parametrize("theta,n_direct,p", [(0.5, 64, 5), (0.8, 8, 4), (0.0, 64, 3)])
def test_kdtree_fields_match_the_oracle(theta, n_direct, p):
    pos, q = _sphere(4, 1500, 33.0)
    mu = np.random.default_rng(5).normal(0.0, 0.1, pos.shape)
    g = kdtree_fields(pos, q, mu, p=p, theta=theta, n_direct=n_direct)
    ref = kdtree.kdtree_fields(pos, q, mu, p=p, theta=theta, n_direct=n_direct)
    for k in ("phi", "E", "G"):
        assert oracle.rel_rms(g[k], ref[k]) < 1e-10, k
        assert max_site_err(g[k], ref[k]) < 1e-8, k
    counts = _oracle_counts(pos, theta, 8, n_direct)
    for k, v in counts.items():
        assert g["stats"][k] == v, (k, g["stats"], counts)


def test_kdtree_dipole_pairs_and_device_buffers():
    pos, q = _sphere(6, 900, 28.0)
    mu = np.random.default_rng(7).normal(0.0, 0.2, pos.shape)
    dev = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
    g = kdtree_fields(dev(pos), dev(q), dev(mu), p=5, theta=0.5, dipole_dl=1e-2)
    ref = kdtree.kdtree_fields(pos, q, mu, p=5, theta=0.5, dipole_dl=1e-2)
    for k in ("phi", "E", "G"):
        assert oracle.rel_rms(g[k].cpu().numpy(), ref[k]) < 1e-10, k
    # charges only, dipoles only
    for qq, mm in ((q, None), (None, mu)):
        g = kdtree_fields(pos, qq, mm, p=4, theta=0.6)
        ref = kdtree.kdtree_fields(pos, qq, mm, p=4, theta=0.6)
        assert oracle.rel_rms(g["E"], ref["E"]) < 1e-10


def test_kdtree_sphere_test_accuracy_and_momentum():
    """Sec. IV.A's sphere (4096 sites of +-e, r = 45 A, 2 A apart), theta = 0.5,
    p = 5: the paper's error distribution, and the mutual walk's momentum."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_sphere_test.json")))
    pos, q = _sphere(16, gold["n_sites"], gold["radius_A"])
    f = kdtree_fields(pos, q, p=gold["order_p"], theta=gold["theta"])
    d = oracle.direct_fields(pos, q)
    e = oracle.per_site_rel_err(q[:, None] * f["E"], q[:, None] * d["E"])
    assert (e < 1e-4).mean() >= gold["fraction_below_1e-4"]
    assert e.max() < gold["max_rel_force_error"]
    F = q[:, None] * f["E"]
    assert np.linalg.norm(F.sum(axis=0)) / np.abs(F).sum() < 1e-13


def test_kdtree_edge_cases():
    # one site; fewer sites than a bucket (one leaf, all direct); coincident sites
    for pos in (np.zeros((1, 3)), np.random.default_rng(1).normal(size=(5, 3)) * 3.0):
        q = np.linspace(-0.5, 0.5, pos.shape[0])
        g = kdtree_fields(pos, q, p=3, theta=0.5)
        d = oracle.direct_fields(pos, q)
        assert oracle.rel_rms(g["phi"], d["phi"]) < 1e-13 if pos.shape[0] > 1 else g["phi"][0] == 0.0
    pos = np.repeat(np.random.default_rng(2).normal(size=(3, 3)) * 5.0, 20, axis=0)  # 20 sites at each of 3 points
    pos += np.random.default_rng(3).normal(size=pos.shape) * 1e-3
    q = np.random.default_rng(4).normal(size=pos.shape[0])
    g = kdtree_fields(pos, q, p=3, theta=0.5, n_direct=4)
    ref = kdtree.kdtree_fields(pos, q, p=3, theta=0.5, n_direct=4)
    assert oracle.rel_rms(g["E"], ref["E"]) < 1e-10
    for bad in (dict(theta=1.0), dict(theta=-0.1), dict(p=0), dict(n_bucket=0)):
        kw = dict(p=3, theta=0.5, n_bucket=8)
        kw.update(bad)
        with pytest.raises(PolFMMError) as e:
            kdtree_fields(pos, q, **kw)
        assert e.value.status == _lib.ERR_INVALID_ARG


def test_kdtree_against_the_octree_on_the_globule():
    """The 30k globule with charges and dipoles: the error against the direct
    sum (on 300 sampled sites) and the time of the kd-tree (p = 6,
    theta = 0.7, the paper's n_bucket and n_direct) and of the octree pass
    (p = 6, depth 4), both FP64."""
    w = synth.workload(2)
    mu = np.random.default_rng(3).normal(0.0, 0.1, (w.n, 3))
    dev = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
    x, qd, md = dev(w.pos), dev(w.q), dev(mu)
    kdtree_fields(x, qd, md, p=6, theta=0.7)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = kdtree_fields(x, qd, md, p=6, theta=0.7)
    torch.cuda.synchronize()
    t_kd = time.perf_counter() - t0
    with PolFMM(x, qd, dev(w.alpha), p=6, depth=4) as f:
        f.total_field(md)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        o = f.total_field(md)
        torch.cuda.synchronize()
        t_oct = time.perf_counter() - t0
    sel = np.random.default_rng(9).choice(w.n, 300, replace=False)
    d = oracle.direct_fields(w.pos, w.q, mu, targets=sel)
    e_kd = oracle.rel_rms(g["E"].cpu().numpy()[sel], d["E"])
    e_oct = oracle.rel_rms(o["E"].cpu().numpy()[sel], d["E"])
    print(f"30k globule, FP64: kd-tree {1e3 * t_kd:.1f} ms (E error {e_kd:.2e}, {g['stats']}), "
          f"octree {1e3 * t_oct:.1f} ms (E error {e_oct:.2e})")
    assert e_kd < 1e-2 and e_oct < 1e-2
