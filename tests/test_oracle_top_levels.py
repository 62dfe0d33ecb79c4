"""What single precision at the top of the tree costs (CPU oracle only).

The MIXED mode keeps the multipole shifts into the top levels and the local
shifts out of them in FP32.  The oracle's measurement knob runs exactly those
shifts (levels 2..T, arithmetic and stored results) in single precision and
everything else in FP64; the difference to the all-FP64 oracle at depths 5
and 6 is the whole cost of that choice, to be compared with the MIXED error
budget (1e-5 relative RMS in the forces)."""
import numpy as np
import pytest

import oracle
import synth


def _rel_rms(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


@pytest.mark.parametrize("n,depth", [(12000, 5), (12000, 6)])
def test_single_precision_top_levels_cost_round_off_only(n, depth):
    w = synth.workload(5, n=n, depth=depth)
    mu = np.random.default_rng(3).standard_normal((w.n, 3)) * 0.1
    ref = oracle.fmm_fields(w.pos, w.q, mu, p=6, depth=depth)
    err = {}
    for top in (2, 3):
        f = oracle.fmm_fields(w.pos, w.q, mu, p=6, depth=depth, fp32_top=top)
        err[top] = (_rel_rms(f["E"], ref["E"]), _rel_rms(f["phi"], ref["phi"]))
    print(f"depth {depth}: single-precision shifts at levels 2..T, relative RMS vs FP64 (E, phi): {err}")
    # the knob acts, and what it changes stays at FP32 round-off: two orders of
    # magnitude under the 1e-5 force budget of the mixed mode
    assert 0 < err[2][0] <= err[3][0] < 1e-7
    assert err[3][1] < 1e-6
