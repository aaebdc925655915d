"""Torch-facing wrappers of the C ABI: device buffers and the current stream
come from PyTorch; all computation is in libph0's CUDA kernels.

    bars = barcodes(points)          # points: float32 [N, d] CUDA tensor
    bars.death, bars.u, bars.v ...   # CUDA tensors, filtration order
    bars.numpy()                     # structured array (host copy)
    bars.inf                         # the bar that never dies: (vertex, 0.0, inf)
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import BAR_BYTES, BAR_DTYPE, Stats, check

_FIELDS = {  # name -> (byte offset, byte size, torch dtype) in the 40-byte ph0_bar
    "u": (0, 4, torch.int32), "v": (4, 4, torch.int32), "a": (8, 4, torch.int32),
    "low": (12, 4, torch.int32), "order": (16, 8, torch.int64),
    "death_sq": (24, 8, torch.float64), "death": (32, 8, torch.float64),
}


def _stream(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor | None):
    return ctypes.c_void_p(t.data_ptr() if t is not None and t.numel() else None)


class Workspace:
    """Caller-owned device workspace for clouds up to (n, d)."""

    def __init__(self, n: int, d: int, device=None):
        nbytes = _lib.workspace_bytes(n, d)
        if nbytes == 0:
            raise _lib.Ph0Error(3, f"workspace_bytes(n={n}, d={d})")
        self.n, self.d, self.nbytes = n, d, nbytes
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")

    @property
    def ptr(self):
        return ctypes.c_void_p(self.buf.data_ptr())

    def fits(self, n: int, d: int) -> bool:
        return _lib.workspace_bytes(n, d) <= self.nbytes


_ws_cache: dict = {}


def _workspace(n: int, d: int, device) -> Workspace:
    key = (device.index if device.index is not None else torch.cuda.current_device())
    ws = _ws_cache.get(key)
    if ws is None or not ws.fits(n, d):
        ws = Workspace(n, d, device)
        _ws_cache[key] = ws
    return ws


@dataclass
class Bars:
    raw: torch.Tensor          # uint8 [n-1, 40] device buffer
    n: int
    stats: dict | None = None
    inf_raw: torch.Tensor | None = None   # uint8 [24] device buffer (ph0_inf_bar)

    def __getattr__(self, name):
        if name in _FIELDS:
            off, size, dt = _FIELDS[name]
            nb = self.raw.shape[0]
            return self.raw[:, off:off + size].contiguous().view(dt).reshape(nb)
        raise AttributeError(name)

    def numpy(self) -> np.ndarray:
        return self.raw.cpu().numpy().reshape(-1).view(BAR_DTYPE).copy()

    @property
    def inf(self) -> tuple:
        """The bar that never dies, as written by the kernels: (vertex, birth, death)."""
        b = _lib.InfBar.from_buffer_copy(self.inf_raw.cpu().numpy().tobytes())
        return int(b.vertex), float(b.birth), float(b.death)

    @property
    def inf_vertex(self) -> int:
        return self.inf[0]


def _inf_buffer(device) -> torch.Tensor:
    return torch.empty(_lib.INF_BAR_BYTES, dtype=torch.uint8, device=device)


def _points(pts: torch.Tensor):
    if not isinstance(pts, torch.Tensor) or not pts.is_cuda:
        raise TypeError("points must be a CUDA tensor (there is no CPU path)")
    if pts.dtype != torch.float32 or pts.dim() != 2:
        raise TypeError("points must be float32 [N, d]")
    if pts.stride(1) != 1:
        pts = pts.contiguous()
    return pts, pts.shape[0], pts.shape[1], pts.stride(0)


def _tuning(n: int, d: int, tuning):
    """Explicit tuning, else the autotuner's cached choice for this cloud size
    and dimension (None: the library's built-in choice)."""
    if tuning is not None:
        return tuning if isinstance(tuning, _lib.Tuning) else _lib.Tuning.make(**tuning)
    from . import autotune
    t = autotune.cached(d, n)
    return _lib.Tuning.make(**t) if t else None


def barcodes(pts: torch.Tensor, ws: Workspace | None = None, stats: bool = False,
             sync: bool = True, tuning=None) -> Bars:
    """Finite bars of the 0th persistent homology of the point cloud (steps 1-5)."""
    pts, n, d, ld = _points(pts)
    ws = ws or _workspace(n, d, pts.device)
    bars = torch.empty((max(n - 1, 0), BAR_BYTES), dtype=torch.uint8, device=pts.device)
    inf = _inf_buffer(pts.device)
    s = _stream()
    lib = _lib.load()
    t = _tuning(n, d, tuning)
    check(lib.ph0_barcodes_tuned(_ptr(pts), n, d, ld, _ptr(bars), _ptr(inf), ws.ptr, ws.nbytes, s,
                                 ctypes.byref(t) if t is not None else None), "ph0_barcodes")
    st = None
    if sync or stats:
        st = finish(ws)
    return Bars(bars, n, st, inf)


def barcodes_early(pts: torch.Tensor, ws: Workspace | None = None, rounds: bool | None = None,
                   tuning: dict | None = None) -> Bars:
    """The same bars as barcodes(), sorting only the prefix of the edge order
    the reduction needs (ph0_barcodes_early_tuned; waits for the GPU).  The
    stats report the prefix length as sorted_edges.  rounds: None lets the
    library choose (rounds from 2^27 edges on), True always sorts in rounds,
    False runs the whole path."""
    pts, n, d, ld = _points(pts)
    ws = ws or _workspace(n, d, pts.device)
    bars = torch.empty((max(n - 1, 0), BAR_BYTES), dtype=torch.uint8, device=pts.device)
    inf = _inf_buffer(pts.device)
    t = _lib.Tuning.make(**{**(tuning or {}), "early_rounds": -1 if rounds is None else int(bool(rounds))})
    st = Stats()
    check(_lib.load().ph0_barcodes_early_tuned(_ptr(pts), n, d, ld, _ptr(bars), _ptr(inf), ws.ptr, ws.nbytes,
                                               _stream(), ctypes.byref(t), ctypes.byref(st)), "ph0_barcodes_early")
    return Bars(bars, n, st.as_dict(), inf)


def barcodes_profiled(pts: torch.Tensor, ws: Workspace | None = None, bars: torch.Tensor | None = None,
                      tuning=None):
    """ph0_barcodes with CUDA events between the stages (waits for the stream).
    Returns (Bars, per-stage milliseconds)."""
    pts, n, d, ld = _points(pts)
    ws = ws or _workspace(n, d, pts.device)
    if bars is None:
        bars = torch.empty((max(n - 1, 0), BAR_BYTES), dtype=torch.uint8, device=pts.device)
    prof = _lib.Profile()
    inf = _inf_buffer(pts.device)
    t = _tuning(n, d, tuning)
    check(_lib.load().ph0_barcodes_profiled(_ptr(pts), n, d, ld, _ptr(bars), _ptr(inf), ws.ptr, ws.nbytes,
                                            _stream(), ctypes.byref(t) if t is not None else None,
                                            ctypes.byref(prof)), "ph0_barcodes_profiled")
    return Bars(bars, n, None, inf), prof.as_dict()


def h1(pts: torch.Tensor):
    """First-homology bars of the Vietoris-Rips 2-skeleton (ph0_h1; waits
    for the GPU): (structured host array in triangle order, stats).  Every
    positive edge is paired, zero-length bars included; n <= 4096."""
    pts, n, d, ld = _points(pts)
    lib = _lib.load()
    nbytes = int(lib.ph0_h1_workspace_bytes(n, d))
    if nbytes == 0:
        raise _lib.Ph0Error(3, f"ph0_h1_workspace_bytes(n={n}, d={d})")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=pts.device)
    nb = max(n * (n - 1) // 2 - (n - 1), 0)
    bars = torch.empty((max(nb, 1), _lib.H1_BAR_BYTES), dtype=torch.uint8, device=pts.device)
    st = _lib.H1Stats()
    check(lib.ph0_h1(_ptr(pts), n, d, ld, _ptr(bars), _ptr(ws), nbytes, _stream(), ctypes.byref(st)), "ph0_h1")
    out = bars[:nb].cpu().numpy().reshape(-1).view(_lib.H1_DTYPE).copy()
    return out, st.as_dict()


def trace_windows(ws: Workspace, n: int, d: int, max_windows: int = 256):
    """Per-window records of the last reduction on `ws` (tracing aid)."""
    out = np.zeros((max_windows, 12), np.uint64)
    check(_lib.load().ph0_trace_windows(ws.ptr, n, d, _stream(), out.ctypes.data_as(ctypes.c_void_p),
                                        max_windows), "ph0_trace_windows")
    rows = []
    for r in out:
        if r[1] == 0:
            break
        t0 = int(r[6])
        rows.append({"pos0": int(r[0]), "window": int(r[1]), "candidates": int(r[2]),
                     "grid_rounds": int(r[3]), "tail_rounds": int(r[4]), "pivots": int(r[5]),
                     "filter_us": (int(r[7]) - t0) / 1e3, "grid_us": (int(r[8]) - int(r[7])) / 1e3,
                     "tail_us": (int(r[9]) - int(r[8])) / 1e3, "flatten_us": (int(r[10]) - int(r[9])) / 1e3})
    return rows


def finish(ws: Workspace) -> dict:
    st = Stats()
    rc = _lib.load().ph0_finish(ws.ptr, _stream(), ctypes.byref(st))
    check(rc, "device status")
    return st.as_dict()


# ---------------------------------------------------------------- steps ---

def distances(pts: torch.Tensor, ws: Workspace | None = None):
    """Step 1: (key int64 [E] = binary64 bits of d2, val int32 [E] = u<<16|v),
    edges in lexicographic (u, v) order."""
    pts, n, d, ld = _points(pts)
    ws = ws or _workspace(n, d, pts.device)
    m = n * (n - 1) // 2
    key = torch.empty(m, dtype=torch.int64, device=pts.device)
    val = torch.empty(m, dtype=torch.int32, device=pts.device)
    check(_lib.load().ph0_distances(_ptr(pts), n, d, ld, _ptr(key), _ptr(val), ws.ptr, ws.nbytes,
                                    _stream()), "ph0_distances")
    finish(ws)
    return key, val


def sort_pairs(key: torch.Tensor, val: torch.Tensor, ws: Workspace | None = None):
    """Step 2: stable sort of (key, val) by key (unsigned), in place."""
    m = key.numel()
    assert key.dtype == torch.int64 and val.dtype == torch.int32 and val.numel() == m
    n = 2
    while n * (n - 1) // 2 < m:
        n += 1
    ws = ws or _workspace(n, 1, key.device)
    check(_lib.load().ph0_sort(_ptr(key), _ptr(val), m, ws.ptr, ws.nbytes, _stream()), "ph0_sort")
    finish(ws)
    return key, val


def dedupe(key_sorted: torch.Tensor, ws: Workspace | None = None):
    """Step 3: a (int32 [m], 1-based index in D) of sorted keys, and |D|."""
    m = key_sorted.numel()
    n = 2
    while n * (n - 1) // 2 < m:
        n += 1
    ws = ws or _workspace(n, 1, key_sorted.device)
    a = torch.empty(m, dtype=torch.int32, device=key_sorted.device)
    check(_lib.load().ph0_dedupe(_ptr(key_sorted), m, _ptr(a), ws.ptr, ws.nbytes, _stream()),
          "ph0_dedupe")
    st = finish(ws)
    return a, st["n_distinct"]


def reduce(n: int, val_sorted: torch.Tensor, a: torch.Tensor, key_sorted: torch.Tensor,
           ws: Workspace | None = None) -> Bars:
    """Steps 4-5 on sorted edges: the n-1 bars."""
    ws = ws or _workspace(n, 1, val_sorted.device)
    bars = torch.empty((max(n - 1, 0), BAR_BYTES), dtype=torch.uint8, device=val_sorted.device)
    check(_lib.load().ph0_reduce(n, _ptr(val_sorted), _ptr(a), _ptr(key_sorted), _ptr(bars),
                                 ws.ptr, ws.nbytes, _stream()), "ph0_reduce")
    return Bars(bars, n, finish(ws))


def backward(pts: torch.Tensor, bars: Bars, dl_ddeath: torch.Tensor,
             ws: Workspace | None = None) -> torch.Tensor:
    """d loss / d points for fixed killing edges (float32 [N, d])."""
    pts, n, d, ld = _points(pts)
    ws = ws or _workspace(n, d, pts.device)
    g = dl_ddeath.to(dtype=torch.float64).contiguous()
    grad = torch.empty((n, d), dtype=torch.float32, device=pts.device)
    nb = bars.raw.shape[0]
    check(_lib.load().ph0_barcodes_backward(_ptr(pts), n, d, ld, _ptr(bars.raw), nb, _ptr(g),
                                            _ptr(grad), ws.ptr, ws.nbytes, _stream()),
          "ph0_barcodes_backward")
    return grad


# ------------------------------------------------------------ autograd ---

class DeathValues(torch.autograd.Function):
    """death_i = distance of the i-th killing edge (filtration order), as a
    differentiable function of the points.  The pairing (which edges kill) is
    piecewise constant in the points, so the derivative is that of the
    killing edges' lengths; the backward pass is the hand-written kernel."""

    @staticmethod
    def forward(ctx, pts, ws=None):
        bars = barcodes(pts, ws)
        ctx.save_for_backward(pts)
        ctx.bars = bars
        ctx.ws = ws
        return bars.death

    @staticmethod
    def backward(ctx, grad_death):
        (pts,) = ctx.saved_tensors
        return backward(pts, ctx.bars, grad_death, ctx.ws), None


def death_values(pts: torch.Tensor, ws: Workspace | None = None) -> torch.Tensor:
    """Finite death values (float64 [N-1], filtration order), differentiable."""
    return DeathValues.apply(pts, ws)


class DeathValuesBatch(torch.autograd.Function):
    """DeathValues over many clouds at once: every cloud's forward path and
    backward kernel is queued on one of several CUDA streams, so the clouds'
    kernels overlap on the GPU; the statuses are read once all are queued.
    While the current stream is being captured into a CUDA graph nothing
    waits: the statuses are left to Batch.check() after each replay."""

    @staticmethod
    def forward(ctx, workspaces, streams, *pts):
        cur = torch.cuda.current_stream()
        bars = []
        for i, p in enumerate(pts):
            s = streams[i % len(streams)]
            s.wait_stream(cur)
            with torch.cuda.stream(s):
                bars.append(barcodes(p, workspaces[i], sync=False))
        if not torch.cuda.is_current_stream_capturing():
            for i, ws in enumerate(workspaces[:len(pts)]):
                with torch.cuda.stream(streams[i % len(streams)]):
                    finish(ws)  # waits for that stream; raises on a device error
        for s in streams:
            cur.wait_stream(s)
        out = [b.death for b in bars]  # on the current stream, after every cloud finished
        ctx.save_for_backward(*pts)
        ctx.bars, ctx.workspaces, ctx.streams = bars, workspaces, streams
        return tuple(out)

    @staticmethod
    def backward(ctx, *grads):
        pts = ctx.saved_tensors
        cur = torch.cuda.current_stream()
        out = []
        for i, (p, g) in enumerate(zip(pts, grads)):
            s = ctx.streams[i % len(ctx.streams)]
            s.wait_stream(cur)
            with torch.cuda.stream(s):
                gp = backward(p, ctx.bars[i], g.contiguous(), ctx.workspaces[i])
            gp.record_stream(cur)  # made on s, used on the current stream
            out.append(gp)
        for s in ctx.streams:
            cur.wait_stream(s)
        return (None, None, *out)


class Batch:
    """Workspaces and streams for death_values over a fixed set of cloud
    shapes (one workspace per cloud, so that clouds on different streams
    never share one)."""

    def __init__(self, shapes, streams: int = 8, device=None):
        self.workspaces = [Workspace(n, d, device) for n, d in shapes]
        self.streams = [torch.cuda.Stream(device=device) for _ in range(streams)]

    def death_values(self, pts_list):
        """Finite death values of every cloud (a tuple of float64 tensors),
        differentiable with respect to each cloud's points."""
        return DeathValuesBatch.apply(self.workspaces, self.streams, *pts_list)

    def check(self):
        """Raise on a device error of the last calls on these workspaces
        (after replaying a captured step): every status word in one copy."""
        for i, st in enumerate(statuses(self.workspaces)):
            if st != 0:
                raise _lib.Ph0Error(int(st), f"cloud {i}")


def statuses(workspaces) -> list:
    """The ph0_status of the last call on each workspace (one device copy,
    then a wait for the current stream)."""
    off = int(_lib.load().ph0_status_offset())
    words = torch.stack([w.buf[off:off + 4] for w in workspaces]).view(torch.int32)
    return words.flatten().tolist()
