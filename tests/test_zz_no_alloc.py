"""The allocation-free entry point, ph0_barcodes_noalloc, against the
workspace entry point ph0_barcodes and against the oracle.

Some callers cannot allocate device memory at the point where they need
barcodes: latency-critical loops, where a cudaMalloc can synchronize the
device or take a driver lock, and hosts that own all device memory through
their own pool, where a raw allocation fails or fragments it.  They use
ph0_barcodes_noalloc, which takes its workspace from a fixed 16 MiB array in
the library instead of from the caller.  Its bars must be the same as those
of ph0_barcodes, bit for bit (the tolerance of every parity test here), on
consecutive calls that reuse the array.  This file is collected last, so
that a run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2203_02527_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

vp = ctypes.c_void_p


def _lib():
    from paper_2203_02527_gb300 import _lib
    return _lib


def _bars_workspace(lib, pts, d=None):
    n = pts.shape[0]
    d = pts.shape[1] if d is None else d
    ld = pts.stride(0)
    nbytes = lib.ph0_workspace_bytes(n, d)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    bars = torch.empty((max(n - 1, 1), 40), dtype=torch.uint8, device="cuda")
    rc = lib.ph0_barcodes(vp(pts.data_ptr()), n, d, ld, vp(bars.data_ptr()), None, vp(ws.data_ptr()),
                          nbytes, None)
    assert rc == 0
    assert lib.ph0_finish(vp(ws.data_ptr()), None, None) == 0
    return bars[: n - 1].cpu().numpy()


def _bars_noalloc(lib, pts, d=None):
    n = pts.shape[0]
    d = pts.shape[1] if d is None else d
    bars = torch.full((max(n - 1, 1), 40), 0xAB, dtype=torch.uint8, device="cuda")
    inf = torch.full((24,), 0xAB, dtype=torch.uint8, device="cuda")
    rc = lib.ph0_barcodes_noalloc(vp(pts.data_ptr()), n, d, pts.stride(0), vp(bars.data_ptr()),
                                  vp(inf.data_ptr()), None)
    assert rc == 0, rc
    b = _lib().InfBar.from_buffer_copy(inf.cpu().numpy().tobytes())
    assert (b.vertex, b.birth, b.death) == (0, 0.0, float("inf"))
    return bars[: n - 1].cpu().numpy()


def _oracle_raw(x):
    want, inf_v, _ = oracle.barcodes(x)
    assert inf_v == 0
    return np.ascontiguousarray(want).view(np.uint8).reshape(-1, 40)


def test_noalloc_matches_workspace_entry_point_on_consecutive_calls():
    lib = _lib().load()
    clouds = [inputs.uniform(700, 3, seed=71),                       # the paper's largest N
              inputs.gaussian_mixture(613, 16, k=5, sigma=0.3, seed=72),
              inputs.lattice(9, 2)]                                  # many exact ties
    for i, x in enumerate(clouds):
        pts = torch.from_numpy(x).cuda()
        want = _bars_workspace(lib, pts)
        first = _bars_noalloc(lib, pts)
        second = _bars_noalloc(lib, pts)  # the array keeps the previous call's contents
        np.testing.assert_array_equal(first, want)
        np.testing.assert_array_equal(second, want)
        if i == 0:  # and against the oracle, which shares nothing with either
            np.testing.assert_array_equal(first, _oracle_raw(x))


def test_noalloc_size_limit_edge():
    lib = _lib().load()
    # n = 889 at d = 3 is the largest cloud whose workspace fits 16 MiB
    assert lib.ph0_workspace_bytes(889, 3) <= 16 << 20 < lib.ph0_workspace_bytes(890, 3)
    x = inputs.uniform(889, 3, seed=73)
    pts = torch.from_numpy(x).cuda()
    np.testing.assert_array_equal(_bars_noalloc(lib, pts), _oracle_raw(x))
    y = torch.from_numpy(inputs.uniform(890, 3, seed=74)).cuda()
    bars = torch.empty((889, 40), dtype=torch.uint8, device="cuda")
    assert lib.ph0_barcodes_noalloc(vp(y.data_ptr()), 890, 3, 3, vp(bars.data_ptr()), None, None) == 3


def test_noalloc_strided_and_trivial_clouds():
    lib = _lib().load()
    # rows of 5 floats of which the first 3 are the coordinates (ld > d)
    x = inputs.uniform(300, 5, seed=75)
    pts = torch.from_numpy(x).cuda()
    got = _bars_noalloc(lib, pts, d=3)
    np.testing.assert_array_equal(got, _oracle_raw(np.ascontiguousarray(x[:, :3])))
    np.testing.assert_array_equal(got, _bars_workspace(lib, pts, d=3))
    for n in (1, 2):
        z = inputs.uniform(n, 3, seed=76 + n)
        got = _bars_noalloc(lib, torch.from_numpy(z).cuda())
        assert len(got) == n - 1
        if n == 2:
            np.testing.assert_array_equal(got, _oracle_raw(z))


def test_noalloc_rejects_clouds_beyond_its_array():
    lib = _lib().load()
    n, d = 2000, 3  # needs more than 16 MiB of workspace
    assert lib.ph0_workspace_bytes(n, d) > 16 << 20
    pts = torch.zeros((n, d), device="cuda")
    bars = torch.empty((n - 1, 40), dtype=torch.uint8, device="cuda")
    assert lib.ph0_barcodes_noalloc(vp(pts.data_ptr()), n, d, d, vp(bars.data_ptr()), None, None) == 3


def test_noalloc_refuses_a_stream_under_capture():
    """The call waits for its stream, which a capture forbids: on a stream
    being captured it returns PH0_EINVAL at once and queues nothing, so the
    caller's capture ends normally and replays; then the same call outside the
    capture gives the oracle's bars."""
    lib = _lib().load()
    x = inputs.uniform(200, 3, seed=77)
    pts = torch.from_numpy(x).cuda()
    bars = torch.empty((199, 40), dtype=torch.uint8, device="cuda")
    src = torch.arange(1024, dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        rc = lib.ph0_barcodes_noalloc(vp(pts.data_ptr()), 200, 3, 3, vp(bars.data_ptr()), None,
                                      vp(s.cuda_stream))
        out = src * 2
    assert rc == 1  # PH0_EINVAL
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, src * 2)
    np.testing.assert_array_equal(_bars_noalloc(lib, pts), _oracle_raw(x))
