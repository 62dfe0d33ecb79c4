"""The allocation-free tree set-up (fmm_sort_sites_noalloc) against the
allocating path of fmm_build, through the C ABI.

Callers that cannot allocate device memory (a host framework that owns the
device's memory pool, a time-critical loop that cannot afford the
synchronisation of cudaMalloc / cudaFree) use this entry point; its scratch is
one static device array shared by every call.  Each case is called twice in a
row, so that leftovers of the previous call in that shared array would show.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1408_6527_gb300 import PolFMM, _lib  # noqa: E402


def _morton(c):
    k = np.zeros(c.shape[0], dtype=np.int64)
    for b in range(10):
        for a in range(3):
            k |= ((c[:, a].astype(np.int64) >> b) & 1) << (3 * b + a)
    return k


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _positions(index):
    if index == "max":
        # exactly the largest size the static scratch holds: uniform sites in a cube
        n = _lib.NOALLOC_MAX_SITES
        rng = np.random.default_rng(7)
        return rng.uniform(0.0, 140.0, size=(n, 3)), np.zeros(n), np.ones(n)
    w = synth.workload(index)
    return w.pos, w.q, w.alpha


@pytest.mark.parametrize("index,depth", [(1, 3), (2, 4), (2, 7), ("max", 6)])
def test_noalloc_sort_matches_allocating_path(index, depth):
    lib = _lib.load()
    wpos, wq, walpha = _positions(index)

    class w:  # noqa: N801
        n = wpos.shape[0]

    pos = torch.as_tensor(wpos, dtype=torch.float64, device="cuda")
    with PolFMM(pos, torch.as_tensor(wq, device="cuda"), torch.as_tensor(walpha, device="cuda"), p=2,
                depth=depth) as f:
        ref_cells = f.leaf_cells().cpu().numpy()
        ref_lo, ref_side = f.root_box()
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        cells = torch.full((w.n, 3), -1, dtype=torch.int32, device="cuda")
        keys = torch.full((w.n,), -1, dtype=torch.int32, device="cuda")
        perm = torch.full((w.n,), -1, dtype=torch.int32, device="cuda")
        lo = np.zeros(3)
        side = np.zeros(1)
        st = lib.fmm_sort_sites_noalloc(w.n, _ptr(pos), depth, lo.ctypes.data_as(ctypes.c_void_p),
                                        side.ctypes.data_as(ctypes.c_void_p), _ptr(cells), _ptr(keys), _ptr(perm),
                                        ctypes.c_void_p(stream))
        assert st == 0
        c = cells.cpu().numpy()
        np.testing.assert_array_equal(c, ref_cells)
        assert np.array_equal(lo, ref_lo) and side[0] == ref_side
        pm = perm.cpu().numpy().astype(np.int64)
        k = keys.cpu().numpy().view(np.uint32).astype(np.int64)
        np.testing.assert_array_equal(np.sort(pm), np.arange(w.n))
        np.testing.assert_array_equal(k, _morton(c)[pm])
        assert np.all(np.diff(k) >= 0)
        same = np.diff(k) == 0
        assert np.all(np.diff(pm)[same] > 0)  # stable: equal keys keep caller order


def test_noalloc_rejects_more_sites_than_its_scratch_holds():
    lib = _lib.load()
    n = _lib.NOALLOC_MAX_SITES + 1
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    lo = np.zeros(3)
    side = np.zeros(1)
    st = lib.fmm_sort_sites_noalloc(n, _ptr(dummy), 4, lo.ctypes.data_as(ctypes.c_void_p),
                                    side.ctypes.data_as(ctypes.c_void_p), _ptr(dummy), _ptr(dummy), _ptr(dummy),
                                    None)
    assert st == _lib.ERR_INVALID_ARG
