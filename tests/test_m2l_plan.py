"""The schedule the FP32 CUDA-core M2L is compiled with (read from the library,
no device work): for every p it is exactly the contraction
L_n += sum_{|m| <= p - |n|} D_{n+m} M_m (Sec. II.B), split between the two
warps of a pair by output degree, each D value loaded before its first use."""
import ctypes
import os
import shutil

import numpy as np
import pytest

from paper_1408_6527_gb300 import _lib


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_lib.LIB_PATH):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available to build the library")
        import paper_1408_6527_gb300

        paper_1408_6527_gb300.build()
    return ctypes.CDLL(_lib.LIB_PATH)


def multi_indices(p):
    """The coefficient order written out: degree ascending, then x descending,
    then z ascending."""
    out = []
    for o in range(p + 1):
        for x in range(o, -1, -1):
            for z in range(o - x + 1):
                out.append((x, o - x - z, z))
    return out


def plan(lib, p, part):
    f = lib.fmm_testing_m2l_plan
    f.restype = ctypes.c_int
    split = ctypes.c_int(-1)
    nt = f(p, part, 0, None, None, None, None, ctypes.byref(split))
    arrs = [np.zeros(nt, dtype=np.int32) for _ in range(4)]
    ptrs = [a.ctypes.data_as(ctypes.c_void_p) for a in arrs]
    assert f(p, part, nt, *ptrs, ctypes.byref(split)) == nt
    return split.value, arrs


@pytest.mark.parametrize("p", range(1, 7))
def test_plan_is_the_contraction(lib, p):
    mi = multi_indices(p)
    index = {t: i for i, t in enumerate(mi)}
    deg = [sum(t) for t in mi]
    nc = len(mi)
    # every (n, m) with |n| + |m| <= p exactly once, k = index of n + m
    want = {(n, m, index[tuple(a + b for a, b in zip(mi[n], mi[m]))])
            for n in range(nc) for m in range(nc) if deg[n] + deg[m] <= p}
    got = set()
    split = None
    for part in (0, 1):
        split, (n, m, k, load) = plan(lib, p, part)
        na = sum(1 for d in deg if d <= split)
        n_abs = n + (0 if part == 0 else na)
        # the part's outputs are the degrees on its side of the split
        assert all((deg[i] <= split) == (part == 0) for i in n_abs)
        # the second warp reads only the inputs of degree <= p - split - 1
        if part == 1:
            assert all(deg[j] <= p - split - 1 for j in m)
        # ordered by k; a float4 of D is loaded at the first term that needs it
        assert np.all(np.diff(k) >= 0)
        cur = -1
        for kk, ld in zip(k, load):
            if ld:
                cur = kk // 4
            assert cur == kk // 4
        triples = set(zip(n_abs.tolist(), m.tolist(), k.tolist()))
        assert len(triples) == len(n)  # no term twice
        got |= triples
    assert got == want
    # 924 terms at p = 6: the sum over k = n + m of prod_d (k_d + 1)
    assert len(want) == sum(int(np.prod([c + 1 for c in t])) for t in mi)
    # the split balances the two warps' term counts as well as the degrees allow
    per_degree = [sum(1 for d in deg if d == s) * sum(1 for d in deg if d <= p - s) for s in range(p + 1)]
    imbalance = lambda c: abs(sum(per_degree[:c + 1]) - sum(per_degree[c + 1:]))
    assert imbalance(split) == min(imbalance(c) for c in range(p))


def test_plan_rejects_other_orders(lib):
    f = lib.fmm_testing_m2l_plan
    f.restype = ctypes.c_int
    for p, part in ((0, 0), (7, 0), (6, 2), (6, -1)):
        assert f(p, part, 0, None, None, None, None, None) == -1
