"""CPU oracle for the 0th persistent homology barcode path -- TEST
INFRASTRUCTURE ONLY.

A thin ctypes wrapper over ``ph0_oracle.c`` (plain single-threaded C, binary64
arithmetic, compiled with ``-ffp-contract=off``).  It restates Rawson's barcode
algorithm (Sec. 2; Sec. 4 steps 1-5) literally: distances, sort, de-duplication
into D, the vertex-by-edge matrix over F2[t], and a left-to-right column
reduction of every column with no early exit.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It shares no code with the CUDA library and
imports nothing from it.

Pins that keep the oracle honest live in ``tests/test_oracle_*.py``; the
functions here with no such pin are listed there as "parity unpinned" (none at
present).

``barcodes_paper_cpu`` is not the oracle: it wraps ``paper_cpu.c``, the
paper-style multi-core CPU baseline (OpenMP loops, Sec. 3) that the benchmark
times beside the GPU path; the CPU tests check it against the oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ph0_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libph0_oracle.so")
_CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
           "-shared", "-fPIC"]

_lock = threading.Lock()
_lib = None

BAR_DTYPE = np.dtype([
    ("u", np.int32), ("v", np.int32), ("a", np.uint32), ("low", np.int32),
    ("order", np.int64), ("death_sq", np.float64), ("death", np.float64),
])


_PAPER_SRC = os.path.join(_HERE, "paper_cpu.c")
_PAPER_LIB = os.path.join(_OUT_DIR, "libph0_paper_cpu.so")
_paper = None


def _compile(src: str, out: str, flags, force: bool) -> str:
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src)
    if force or stale:
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *flags, "-o", tmp, src, "-lm"])
        os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle (and the paper-style CPU baseline) with gcc (host
    architecture, no native tuning)."""
    _compile(_PAPER_SRC, _PAPER_LIB, [*_CFLAGS, "-fopenmp"], force)
    return _compile(_SRC, _LIB_PATH, _CFLAGS, force)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64, i32, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
            sig = {
                "ph0o_edge_endpoints": [i64, vp, vp],
                "ph0o_distances": [vp, i64, i32, i64, vp],
                "ph0o_distances_f64": [vp, i64, i32, i64, vp],
                "ph0o_sort_edges": [vp, vp, vp, i64, vp],
                "ph0o_dedupe": [vp, i64, vp, vp],
                "ph0o_reduce": [i64, vp, vp, i64, vp, vp, vp],
                "ph0o_reduce_dense": [i64, vp, vp, vp, i64, vp, vp, vp],
                "ph0o_barcodes": [vp, i64, i32, i64, vp, vp, vp, vp],
                "ph0o_death_gradient": [vp, i64, i32, i64, vp, vp, vp, i64, vp],
                "ph0o_barcodes_below": [vp, i64, i32, i64, ctypes.c_double, vp, vp, vp, vp],
                "ph0o_h1": [vp, i64, i32, i64, vp, vp, vp],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def _points(x) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    if x.ndim != 2:
        raise ValueError("points must be [N, d]")
    return x


def n_edges(n: int) -> int:
    return n * (n - 1) // 2


def edge_endpoints(n: int):
    """(u, v) of every edge in lexicographic order (the edge id order)."""
    m = n_edges(n)
    u = np.empty(m, np.int32)
    v = np.empty(m, np.int32)
    _check(_load().ph0o_edge_endpoints(n, _ptr(u), _ptr(v)), "endpoints")
    return u, v


def distances(x) -> np.ndarray:
    """Step 1: binary64 squared distance of every edge, in edge id order."""
    x = _points(x)
    n, d = x.shape
    out = np.empty(n_edges(n), np.float64)
    _check(_load().ph0o_distances(_ptr(x), n, d, d, _ptr(out)), "distances")
    return out


def distances_f64(x) -> np.ndarray:
    """Squared distances of binary64 points (finite differences)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    n, d = x.shape
    out = np.empty(n_edges(n), np.float64)
    _check(_load().ph0o_distances_f64(_ptr(x), n, d, d, _ptr(out)), "distances_f64")
    return out


def sort_edges(d2: np.ndarray, u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Step 2: edge ids sorted by (squared distance, u, v)."""
    d2 = np.ascontiguousarray(d2, np.float64)
    u = np.ascontiguousarray(u, np.int32)
    v = np.ascontiguousarray(v, np.int32)
    order = np.empty(len(d2), np.int64)
    _check(_load().ph0o_sort_edges(_ptr(d2), _ptr(u), _ptr(v), len(d2),
                                   _ptr(order)), "sort")
    return order


def dedupe(d2_sorted: np.ndarray):
    """Step 3: a (1-based index into D) per sorted position, and |D|."""
    d2_sorted = np.ascontiguousarray(d2_sorted, np.float64)
    a = np.empty(len(d2_sorted), np.uint32)
    nd = ctypes.c_int64(0)
    _check(_load().ph0o_dedupe(_ptr(d2_sorted), len(d2_sorted), _ptr(a),
                               ctypes.byref(nd)), "dedupe")
    return a, int(nd.value)


def reduce(n: int, u_sorted: np.ndarray, v_sorted: np.ndarray):
    """Steps 4-5 (sparse F2 supports): low per column (-1 = zero column),
    pivot_of per row (-1 = never a pivot), and the number of column additions."""
    u_sorted = np.ascontiguousarray(u_sorted, np.int32)
    v_sorted = np.ascontiguousarray(v_sorted, np.int32)
    m = len(u_sorted)
    low = np.empty(m, np.int32)
    pivot_of = np.empty(n, np.int64)
    steps = ctypes.c_int64(0)
    _check(_load().ph0o_reduce(n, _ptr(u_sorted), _ptr(v_sorted), m, _ptr(low),
                               _ptr(pivot_of), ctypes.byref(steps)), "reduce")
    return low, pivot_of, int(steps.value)


def reduce_dense(n: int, u_sorted, v_sorted, a):
    """Steps 4-5 on the literal N x E matrix over F2[t] (N <= 64, E <= 4096):
    low per column, exponent b of each pivot entry t^b, homogeneity flags."""
    u_sorted = np.ascontiguousarray(u_sorted, np.int32)
    v_sorted = np.ascontiguousarray(v_sorted, np.int32)
    a = np.ascontiguousarray(a, np.uint32)
    m = len(u_sorted)
    low = np.empty(m, np.int32)
    b = np.empty(m, np.int32)
    hom = np.empty(m, np.int32)
    _check(_load().ph0o_reduce_dense(n, _ptr(u_sorted), _ptr(v_sorted), _ptr(a),
                                     m, _ptr(low), _ptr(b), _ptr(hom)),
           "reduce_dense")
    return low, b, hom


def barcodes(x):
    """Whole path: (bars structured array in filtration order, infinite-bar
    vertex, |D|)."""
    x = _points(x)
    n, d = x.shape
    bars = np.zeros(max(n - 1, 1), BAR_DTYPE)
    nb = ctypes.c_int64(0)
    inf_v = ctypes.c_int32(-1)
    nd = ctypes.c_int64(0)
    _check(_load().ph0o_barcodes(_ptr(x), n, d, d, _ptr(bars), ctypes.byref(nb),
                                 ctypes.byref(inf_v), ctypes.byref(nd)),
           "barcodes")
    return bars[: nb.value].copy(), int(inf_v.value), int(nd.value)


def barcodes_below(x, t_max: float):
    """The bars whose squared death is at most t_max, computed from the
    prefix of the filtration alone (edges with d2 <= t_max): (bars, edges
    kept, distinct distances among them).  With t_max at least the largest
    death these are exactly barcodes()'s bars, positions and indices
    included."""
    x = _points(x)
    n, d = x.shape
    bars = np.zeros(max(n - 1, 1), BAR_DTYPE)
    nb = ctypes.c_int64(0)
    kept = ctypes.c_int64(0)
    nd = ctypes.c_int64(0)
    _check(_load().ph0o_barcodes_below(_ptr(x), n, d, d, float(t_max), _ptr(bars), ctypes.byref(nb),
                                       ctypes.byref(kept), ctypes.byref(nd)), "barcodes_below")
    return bars[: nb.value].copy(), int(kept.value), int(nd.value)


H1_DTYPE = np.dtype([
    ("eu", np.int32), ("ev", np.int32), ("tu", np.int32), ("tv", np.int32), ("tw", np.int32),
    ("birth_a", np.uint32), ("death_a", np.uint32), ("pad", np.int32),
    ("birth_order", np.int64), ("death_order", np.int64), ("death_rank", np.int64),
    ("birth_sq", np.float64), ("death_sq", np.float64),
])


def h1(x):
    """First-homology bars of the Vietoris-Rips 2-skeleton (the extension the
    paper names): (bars in triangle order, triangle count).  Each bar pairs a
    positive edge (birth) with the triangle whose reduced column has that
    edge as its low (death); zero-length bars included."""
    x = _points(x)
    n, d = x.shape
    m = n * (n - 1) // 2
    bars = np.zeros(max(m, 1), H1_DTYPE)
    nb = ctypes.c_int64(0)
    nt = ctypes.c_int64(0)
    _check(_load().ph0o_h1(_ptr(x), n, d, d, _ptr(bars), ctypes.byref(nb), ctypes.byref(nt)), "h1")
    return bars[: nb.value].copy(), int(nt.value)


def death_gradient(x64, bar_u, bar_v, dl_ddeath):
    """d loss / d points in binary64 for fixed killing edges."""
    x64 = np.ascontiguousarray(np.asarray(x64, np.float64))
    n, d = x64.shape
    bar_u = np.ascontiguousarray(bar_u, np.int32)
    bar_v = np.ascontiguousarray(bar_v, np.int32)
    g = np.ascontiguousarray(dl_ddeath, np.float64)
    out = np.empty((n, d), np.float64)
    _check(_load().ph0o_death_gradient(_ptr(x64), n, d, d, _ptr(bar_u),
                                       _ptr(bar_v), _ptr(g), len(bar_u),
                                       _ptr(out)), "gradient")
    return out


def barcodes_f64(x64):
    """Bars of binary64 points (for finite differences): (order, u, v, d2)
    of the killing edges in filtration order."""
    x64 = np.ascontiguousarray(np.asarray(x64, np.float64))
    n = len(x64)
    u, v = edge_endpoints(n)
    d2 = distances_f64(x64)
    order = sort_edges(d2, u, v)
    low, _, _ = reduce(n, u[order], v[order])
    piv = np.flatnonzero(low >= 0)
    return order[piv], u[order][piv], v[order][piv], d2[order][piv]


def pipeline(x):
    """Every intermediate of the path, for step-by-step parity tests:
    dict with d2 (edge id order), order, sorted u/v/d2, a, |D|, low, bars."""
    x = _points(x)
    n = x.shape[0]
    u, v = edge_endpoints(n)
    d2 = distances(x)
    order = sort_edges(d2, u, v)
    us, vs, d2s = u[order], v[order], d2[order]
    a, nd = dedupe(d2s)
    low, pivot_of, steps = reduce(n, us, vs)
    bars, inf_v, _ = barcodes(x)
    return dict(u=u, v=v, d2=d2, order=order, u_sorted=us, v_sorted=vs,
                d2_sorted=d2s, a=a, n_distinct=nd, low=low, pivot_of=pivot_of,
                steps=steps, bars=bars, inf_vertex=inf_v)


def _load_paper():
    global _paper
    with _lock:
        if _paper is None:
            build()
            lib = ctypes.CDLL(_PAPER_LIB)
            i64, i32, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
            lib.ph0p_barcodes.argtypes = [vp, i64, i32, i64, vp, vp, vp, vp]
            lib.ph0p_barcodes.restype = ctypes.c_int
            lib.ph0p_threads.argtypes = []
            lib.ph0p_threads.restype = ctypes.c_int
            _paper = lib
    return _paper


def paper_cpu_threads() -> int:
    """Threads the paper-style CPU baseline runs on (OpenMP's default: every
    core the process may use, or OMP_NUM_THREADS)."""
    return int(_load_paper().ph0p_threads())


def barcodes_paper_cpu(x):
    """The paper-style multi-core CPU baseline (not the oracle): the same
    (bars, infinite-bar vertex, |D|) as barcodes(), computed with OpenMP
    loops (Sec. 3) and a sequential reduction that stops at n-1 pivots."""
    x = _points(x)
    n, d = x.shape
    bars = np.zeros(max(n - 1, 1), BAR_DTYPE)
    nb = ctypes.c_int64(0)
    inf_v = ctypes.c_int32(-1)
    nd = ctypes.c_int64(0)
    _check(_load_paper().ph0p_barcodes(_ptr(x), n, d, d, _ptr(bars), ctypes.byref(nb),
                                       ctypes.byref(inf_v), ctypes.byref(nd)), "paper_cpu")
    return bars[: nb.value].copy(), int(inf_v.value), int(nd.value)
