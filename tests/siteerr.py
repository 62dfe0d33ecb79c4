"""Per-site error of a per-site field against its reference (test helper).

The relative error of site i is |a_i - b_i| / max(|b_i|, floor * rms(b)), with
|.| the Euclidean norm of the site's components (Sec. IV, Eq. error: the
per-atom relative force error).  The floor keeps sites whose reference value
is nearly zero (a near-cancelling field) from dominating the maximum: the error
is then measured against 1 % of the typical magnitude instead.
"""
import numpy as np

FLOOR = 1e-2


def per_site(a, b, floor=FLOOR):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    a = a.reshape(len(a), -1)
    b = b.reshape(len(b), -1)
    nb = np.linalg.norm(b, axis=1)
    rms = np.sqrt(np.mean(nb ** 2))
    den = np.maximum(nb, floor * rms) if rms > 0 else np.ones_like(nb)
    return np.linalg.norm(a - b, axis=1) / den


def max_site_err(a, b, floor=FLOOR):
    return float(per_site(a, b, floor).max())
