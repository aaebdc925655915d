"""Python binding of the serving context (ph0_ctx_* in include/ph0.h).

    srv = Server(mem_budget=8 << 30)
    srv.submit(points_float32_nd, tag=7)       # copies the points
    for r in srv.poll(wait_ms=10):             # finished clouds, any order
        r.bars, r.latency                      # numpy structured bars (copy)
    srv.close()

The context admits clouds as they arrive, by device-memory budget, runs large
clouds concurrently on several streams and batches small ones into one launch
of a fused kernel; every cloud's bars equal those of ph0.barcodes.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _lib
from ._lib import BAR_DTYPE, check

EBUSY = 7


@dataclass
class Finished:
    tag: int
    status: int
    n: int
    d: int
    bars: np.ndarray
    submit_time: float
    done_time: float
    inf_vertex: int = 0        # vertex of the bar that never dies

    @property
    def latency(self) -> float:
        return self.done_time - self.submit_time


class Server:
    def __init__(self, mem_budget: int = 4 << 30, host_budget: int = 1 << 30, streams: int = 4,
                 small_max_n: int = 180, batch_max: int = 512):
        import torch  # the context lives on torch's current device
        torch.cuda.current_device()
        self._lib = _lib.load()
        opt = _lib.Options(mem_budget, host_budget, streams, small_max_n, batch_max, 0)
        h = ctypes.c_void_p()
        check(self._lib.ph0_ctx_create(ctypes.byref(opt), ctypes.byref(h)), "ph0_ctx_create")
        self._h = h
        self._buf = (_lib.Result * 256)()

    def submit(self, pts: np.ndarray, tag: int) -> int:
        """Queue a cloud; returns 0, or PH0_EBUSY when the pinned pool is full
        (poll and release, then retry).  Other errors raise."""
        x = np.ascontiguousarray(pts, dtype=np.float32)
        n, d = x.shape
        rc = self._lib.ph0_submit(self._h, x.ctypes.data_as(ctypes.c_void_p), n, d, tag)
        if rc not in (0, EBUSY):
            check(rc, "ph0_submit")
        return rc

    def poll(self, max_results: int = 256, wait_ms: int = 0, release: bool = True):
        got = ctypes.c_int32(0)
        k = min(max_results, len(self._buf))
        check(self._lib.ph0_poll(self._h, self._buf, k, ctypes.byref(got), wait_ms), "ph0_poll")
        out = []
        for i in range(got.value):
            r = self._buf[i]
            nb = int(r.n_bars)
            if nb > 0:
                raw = (ctypes.c_char * (nb * BAR_DTYPE.itemsize)).from_address(r.bars)
                bars = np.frombuffer(raw, dtype=BAR_DTYPE).copy()
            else:
                bars = np.zeros(0, BAR_DTYPE)
            out.append(Finished(int(r.tag), int(r.status), int(r.n), int(r.d), bars,
                                float(r.submit_time), float(r.done_time), int(r.inf_vertex)))
            if release:
                check(self._lib.ph0_release(self._h, r.tag), "ph0_release")
        return out

    def close(self):
        if self._h:
            self._lib.ph0_ctx_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def run_stream(server: Server, clouds, arrivals=None, tag0: int = 0):
    """Submit `clouds` (at `arrivals` seconds from now, if given) and collect
    every result; returns {tag: Finished}."""
    import time
    t0 = time.perf_counter()
    done = {}
    i = 0
    total = len(clouds)
    while len(done) < total:
        now = time.perf_counter() - t0
        while i < total and (arrivals is None or arrivals[i] <= now):
            if server.submit(clouds[i], tag0 + i) == EBUSY:
                break
            i += 1
        for f in server.poll(wait_ms=0 if i < total else 1):
            done[f.tag] = f
    return done
