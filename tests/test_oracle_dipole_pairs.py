"""The +-q pair form of the point dipoles in the oracle's multipoles (Sec. II.C,
mu = 2 |q^mu| dl, NEXT-4), pinned by what the mathematics fixes: the pair's
multipole differs from the point dipole's by even powers of dl only, so the
field converges to the analytic one as dl^2; charges alone are untouched; and
dl = 0 is the analytic form itself."""
import numpy as np

import oracle
import synth


def _rel(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


def test_pair_dipoles_converge_to_the_point_dipole_as_dl_squared():
    w = synth.workload(1)
    mu = np.random.default_rng(1).standard_normal((w.n, 3)) * 0.3
    ref = oracle.fmm_fields(w.pos, w.q, mu, p=6, depth=3)
    d = {dl: _rel(oracle.fmm_fields(w.pos, w.q, mu, p=6, depth=3, dipole_dl=dl)["E"], ref["E"])
         for dl in (1e-3, 1e-2, 2e-2, 4e-2)}
    # the first omitted term is O(dl^2): doubling dl quadruples the difference
    assert 3.9 < d[2e-2] / d[1e-2] < 4.1
    assert 3.9 < d[4e-2] / d[2e-2] < 4.1
    assert 95 < d[1e-2] / d[1e-3] < 105
    # at the paper's recommended 1e-4 A the two forms agree to ~1e-10
    assert _rel(oracle.fmm_fields(w.pos, w.q, mu, p=6, depth=3, dipole_dl=1e-4)["E"], ref["E"]) < 1e-9


def test_pair_form_leaves_charges_and_the_near_field_alone():
    w = synth.workload(1)
    a = oracle.fmm_fields(w.pos, w.q, None, p=5, depth=3)
    b = oracle.fmm_fields(w.pos, w.q, None, p=5, depth=3, dipole_dl=1e-2)
    np.testing.assert_array_equal(a["E"], b["E"])
    # one leaf (depth 1: every pair is a near pair): the dipoles act through
    # the explicit near field, identical for any dl
    mu = np.random.default_rng(2).standard_normal((w.n, 3))
    a = oracle.fmm_fields(w.pos, None, mu, p=5, depth=1)
    b = oracle.fmm_fields(w.pos, None, mu, p=5, depth=1, dipole_dl=1e-2)
    np.testing.assert_array_equal(a["E"], b["E"])
