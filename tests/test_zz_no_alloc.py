"""The allocation-free entry point, ph0_barcodes_noalloc, against the
workspace entry point ph0_barcodes.

Callers that cannot allocate device memory at the point where they need
barcodes (while a stream is being captured, inside latency-critical loops,
or under a host that owns all device memory through its own pool) use
ph0_barcodes_noalloc, which takes its workspace from a fixed 16 MiB array in
the library instead of from the caller.  Its bars must be the same as those
of ph0_barcodes, bit for bit (the tolerance of every parity test here), on
consecutive calls that reuse the array.  This file is collected last, so
that a run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2203_02527_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _bars_workspace(lib, pts):
    n, d = pts.shape
    nbytes = lib.ph0_workspace_bytes(n, d)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    bars = torch.empty((n - 1, 40), dtype=torch.uint8, device="cuda")
    vp = ctypes.c_void_p
    rc = lib.ph0_barcodes(vp(pts.data_ptr()), n, d, d, vp(bars.data_ptr()), vp(ws.data_ptr()),
                          nbytes, None)
    assert rc == 0
    assert lib.ph0_finish(vp(ws.data_ptr()), None, None) == 0
    return bars.cpu().numpy()


def _bars_noalloc(lib, pts):
    n, d = pts.shape
    bars = torch.full((n - 1, 40), 0xAB, dtype=torch.uint8, device="cuda")
    vp = ctypes.c_void_p
    rc = lib.ph0_barcodes_noalloc(vp(pts.data_ptr()), n, d, d, vp(bars.data_ptr()), None)
    assert rc == 0, rc
    return bars.cpu().numpy()


def test_noalloc_matches_workspace_entry_point_on_consecutive_calls():
    from paper_2203_02527_gb300 import _lib
    lib = _lib.load()
    clouds = [inputs.uniform(700, 3, seed=71),                       # the paper's largest N
              inputs.gaussian_mixture(613, 16, k=5, sigma=0.3, seed=72),
              inputs.lattice(9, 2)]                                  # many exact ties
    for x in clouds:
        pts = torch.from_numpy(x).cuda()
        want = _bars_workspace(lib, pts)
        first = _bars_noalloc(lib, pts)
        second = _bars_noalloc(lib, pts)  # the array keeps the previous call's contents
        np.testing.assert_array_equal(first, want)
        np.testing.assert_array_equal(second, want)


def test_noalloc_rejects_clouds_beyond_its_array():
    from paper_2203_02527_gb300 import _lib
    lib = _lib.load()
    n, d = 2000, 3  # needs more than 16 MiB of workspace
    assert lib.ph0_workspace_bytes(n, d) > 16 << 20
    pts = torch.zeros((n, d), device="cuda")
    bars = torch.empty((n - 1, 40), dtype=torch.uint8, device="cuda")
    vp = ctypes.c_void_p
    assert lib.ph0_barcodes_noalloc(vp(pts.data_ptr()), n, d, d, vp(bars.data_ptr()), None) == 3
