"""ctypes binding of libph0.so (the C ABI in include/ph0.h).

Argument marshalling only: every step of the barcode path runs in the CUDA
kernels of the library.  Torch tensors serve as device buffers and torch's
current stream is passed through.  If the library is missing the binding
raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libph0.so")

BAR_DTYPE = np.dtype([
    ("u", np.int32), ("v", np.int32), ("a", np.uint32), ("low", np.int32),
    ("order", np.int64), ("death_sq", np.float64), ("death", np.float64),
])
BAR_BYTES = BAR_DTYPE.itemsize  # 40

STATUS = {
    0: "PH0_OK", 1: "PH0_EINVAL", 2: "PH0_ENONFINITE", 3: "PH0_ETOOBIG",
    4: "PH0_ENOMEM", 5: "PH0_ETIMEOUT", 6: "PH0_ECUDA", 7: "PH0_EBUSY",
    8: "PH0_EINTERNAL",
}


class Ph0Error(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {STATUS.get(code, code)} ({strerror(code)})")


class Stats(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32), ("sort_passes", ctypes.c_int32),
        ("key_bits", ctypes.c_int32), ("windows", ctypes.c_int32),
        ("n_distinct", ctypes.c_int64), ("edges_scanned", ctypes.c_int64),
        ("candidates", ctypes.c_int64), ("rounds", ctypes.c_int64),
        ("n_bars", ctypes.c_int64), ("dist_tiles", ctypes.c_int64),
        ("dist_tiles_int", ctypes.c_int64), ("sorted_edges", ctypes.c_int64),
        ("inf_vertex", ctypes.c_int32), ("claim_rounds_max", ctypes.c_int32),
        ("claim_attempts", ctypes.c_int64), ("sort_form", ctypes.c_int32), ("_pad", ctypes.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Tuning(ctypes.Structure):
    _fields_ = [("dist_split16", ctypes.c_int32), ("dist_tile", ctypes.c_int32),
                ("sort_top_bits", ctypes.c_int32), ("reduce_spin_limit", ctypes.c_int32),
                ("wide_ids", ctypes.c_int32), ("early_rounds", ctypes.c_int32),
                ("split_sort", ctypes.c_int32), ("packed_sort", ctypes.c_int32)]

    @classmethod
    def make(cls, dist_split16=-1, dist_tile=-1, sort_top_bits=-1, reduce_spin_limit=-1, wide_ids=-1,
             early_rounds=-1, split_sort=-1, packed_sort=-1):
        t = cls()
        t.dist_split16, t.dist_tile, t.sort_top_bits = dist_split16, dist_tile, sort_top_bits
        t.reduce_spin_limit, t.wide_ids, t.early_rounds = reduce_spin_limit, wide_ids, early_rounds
        t.split_sort, t.packed_sort = split_sort, packed_sort
        return t

    def as_dict(self):
        return {"dist_split16": self.dist_split16, "dist_tile": self.dist_tile,
                "sort_top_bits": self.sort_top_bits}


class Profile(ctypes.Structure):
    _fields_ = [
        ("total_ms", ctypes.c_float), ("dist_ms", ctypes.c_float), ("sort_ms", ctypes.c_float),
        ("pass_ms", ctypes.c_float * 8), ("dedupe_ms", ctypes.c_float),
        ("reduce_ms", ctypes.c_float), ("emit_ms", ctypes.c_float), ("fixup_ms", ctypes.c_float),
    ]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "pass_ms"}
        d["pass_ms"] = list(self.pass_ms)
        return d


class Options(ctypes.Structure):
    _fields_ = [
        ("mem_budget", ctypes.c_size_t), ("host_budget", ctypes.c_size_t),
        ("streams", ctypes.c_int32), ("small_max_n", ctypes.c_int32),
        ("batch_max", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


H1_DTYPE = np.dtype([
    ("eu", np.int32), ("ev", np.int32), ("tu", np.int32), ("tv", np.int32), ("tw", np.int32),
    ("birth_a", np.uint32), ("death_a", np.uint32), ("_pad", np.int32),
    ("birth_order", np.int64), ("death_order", np.int64), ("death_rank", np.int64),
    ("birth_sq", np.float64), ("death_sq", np.float64),
])
H1_BAR_BYTES = H1_DTYPE.itemsize  # 72


class H1Stats(ctypes.Structure):
    _fields_ = [("n_bars", ctypes.c_int64), ("n_triangles", ctypes.c_int64),
                ("apparent", ctypes.c_int64), ("reduced", ctypes.c_int64),
                ("additions", ctypes.c_int64), ("max_column", ctypes.c_int64),
                ("pool_entries", ctypes.c_int64), ("edges_ms", ctypes.c_float),
                ("scan_ms", ctypes.c_float), ("reduce_ms", ctypes.c_float),
                ("emit_ms", ctypes.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class InfBar(ctypes.Structure):
    _fields_ = [("vertex", ctypes.c_int32), ("_pad", ctypes.c_int32),
                ("birth", ctypes.c_double), ("death", ctypes.c_double)]


INF_BAR_BYTES = ctypes.sizeof(InfBar)  # 24


class Result(ctypes.Structure):
    _fields_ = [
        ("tag", ctypes.c_uint64), ("status", ctypes.c_int32), ("n", ctypes.c_int32),
        ("d", ctypes.c_int32), ("inf_vertex", ctypes.c_int32), ("n_bars", ctypes.c_int64),
        ("bars", ctypes.c_void_p), ("submit_time", ctypes.c_double),
        ("done_time", ctypes.c_double),
    ]


_lock = threading.Lock()
_lib = None

_I64, _I32, _VP, _SZ = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t

# name -> (restype, argtypes); the same names as include/ph0.h
SIGNATURES = {
    "ph0_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "ph0_abi_version": (ctypes.c_int32, []),
    "ph0_workspace_bytes": (_SZ, [_I64, _I32]),
    "ph0_barcodes": (ctypes.c_int, [_VP, _I64, _I32, _I64, _VP, _VP, _VP, _SZ, _VP]),
    "ph0_barcodes_early": (ctypes.c_int, [_VP, _I64, _I32, _I64, _VP, _VP, _VP, _SZ, _VP]),
    "ph0_barcodes_early_tuned": (ctypes.c_int, [_VP, _I64, _I32, _I64, _VP, _VP, _VP, _SZ, _VP,
                                                ctypes.POINTER(Tuning), ctypes.POINTER(Stats)]),
    "ph0_finish": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(Stats)]),
    "ph0_status_offset": (ctypes.c_size_t, []),
    "ph0_barcodes_tuned": (ctypes.c_int, [_VP, _I64, _I32, _I64, _VP, _VP, _VP, _SZ, _VP,
                                          ctypes.POINTER(Tuning)]),
    "ph0_barcodes_profiled": (ctypes.c_int, [_VP, _I64, _I32, _I64, _VP, _VP, _VP, _SZ, _VP,
                                             ctypes.POINTER(Tuning), ctypes.POINTER(Profile)]),
    "ph0_trace_windows": (ctypes.c_int, [_VP, _I64, _I32, _VP, _VP, _I32]),
    "ph0_barcodes_noalloc": (ctypes.c_int, [_VP, _I64, _I32, _I64, _VP, _VP, _VP]),
    "ph0_distances": (ctypes.c_int, [_VP, _I64, _I32, _I64, _VP, _VP, _VP, _SZ, _VP]),
    "ph0_ctx_create": (ctypes.c_int, [ctypes.POINTER(Options), ctypes.POINTER(_VP)]),
    "ph0_submit": (ctypes.c_int, [_VP, _VP, _I64, _I32, ctypes.c_uint64]),
    "ph0_poll": (ctypes.c_int, [_VP, ctypes.POINTER(Result), _I32, ctypes.POINTER(_I32), _I32]),
    "ph0_release": (ctypes.c_int, [_VP, ctypes.c_uint64]),
    "ph0_ctx_destroy": (ctypes.c_int, [_VP]),
    "ph0_sort": (ctypes.c_int, [_VP, _VP, _I64, _VP, _SZ, _VP]),
    "ph0_dedupe": (ctypes.c_int, [_VP, _I64, _VP, _VP, _SZ, _VP]),
    "ph0_reduce": (ctypes.c_int, [_I64, _VP, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "ph0_barcodes_backward": (ctypes.c_int, [_VP, _I64, _I32, _I64, _VP, _I64, _VP, _VP,
                                             _VP, _SZ, _VP]),
    "ph0_h1_workspace_bytes": (_SZ, [_I64, _I32]),
    "ph0_h1": (ctypes.c_int, [_VP, _I64, _I32, _I64, _VP, _VP, _SZ, _VP, ctypes.POINTER(H1Stats)]),
}


def load(path: str | None = None):
    """Load libph0.so (fails loudly if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(
                f"libph0.so not found at {p}: build it with "
                "`python -m paper_2203_02527_gb300.build` (there is no CPU fallback)")
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = lib
        return lib


def strerror(code: int) -> str:
    try:
        return load().ph0_strerror(code).decode()
    except Exception:  # pragma: no cover - library missing
        return "?"


def check(code: int, what: str):
    if code != 0:
        raise Ph0Error(code, what)


def workspace_bytes(n: int, d: int) -> int:
    return int(load().ph0_workspace_bytes(n, d))
