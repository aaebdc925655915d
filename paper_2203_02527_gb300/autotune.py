"""Autotuner of the kernels' tuning knobs (ph0_tuning in include/ph0.h).

For a dimension d it times candidate settings on a synthetic cloud of that
dimension (the stages they affect, with CUDA events between the stages of
ph0_barcodes_profiled) and keeps the fastest:
  * dist_split16  -- rows of each 16 of a distance tile that take the running
                     sums on the binary64 units (the rest all in integers),
  * dist_tile     -- points per side of a distance tile (32, 64, 128),
  * sort_top_bits -- width of the single top radix pass (8 or 9),
  * packed_sort   -- the packed sort (1) or the short sort (0), timed on the
                     whole path (clouds from 2^22 edges up to 32768 points;
                     in few dimensions the keys often do not pack).
Results are cached in a JSON file keyed by GPU name, dimension bucket and
cloud-size bucket ($PH0_TUNING_CACHE, default ~/.cache/ph0_gb300/tuning.json):
the best distance tile depends on how many tiles a cloud has to fill the GPU.  No setting
changes any result bit; ph0.barcodes uses the cached choice when present.
"""
from __future__ import annotations

import json
import os
import threading

_lock = threading.Lock()
_cache = None

BUCKETS = (1, 2, 3, 4, 8, 16, 32, 64, 128, 256, 512, 1024)


def bucket(d: int) -> int:
    for b in BUCKETS:
        if d <= b:
            return b
    return BUCKETS[-1]


N_BUCKETS = (2048, 8192, 24576, 65535)


def n_bucket(n: int) -> int:
    for b in N_BUCKETS:
        if n <= b:
            return b
    return N_BUCKETS[-1]


def _key(d: int, n: int) -> str:
    return f"{_device_key()}/d{bucket(d)}/n{n_bucket(n)}"


def cache_path() -> str:
    return os.environ.get("PH0_TUNING_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "ph0_gb300", "tuning.json"))


def _device_key() -> str:
    import torch
    return torch.cuda.get_device_name().replace(" ", "_")


def _load():
    global _cache
    with _lock:
        if _cache is None:
            try:
                with open(cache_path()) as f:
                    _cache = json.load(f)
            except (OSError, ValueError):
                _cache = {}
    return _cache


def cached(d: int, n: int):
    """The cached tuning for an n-point cloud of dimension d on this GPU, or None."""
    try:
        key = _key(d, n)
    except Exception:
        return None
    return _load().get(key)


def _store(d: int, n: int, tuning: dict):
    c = _load()
    with _lock:
        c[_key(d, n)] = tuning
        path = cache_path()
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(c, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def tune(d: int, n: int = 8192, repeats: int = 3, seed: int = 7, verbose: bool = False) -> dict:
    """Measure the candidates for dimension d on an n-point cloud; cache and
    return the fastest setting (for clouds of n's size bucket)."""
    import torch

    from . import inputs, ph0
    if d >= 2:
        x = inputs.noisy_circles(max(n // 4, 2), 4, d, noise=0.02, center_range=5.0, seed=seed)
    else:
        x = inputs.uniform(n, d, seed=seed)
    pts = torch.from_numpy(x).cuda()
    ws = ph0.Workspace(len(x), d)

    def stage_ms(tuning: dict, stage: str) -> float:
        best = float("inf")
        for _ in range(repeats + 1):  # first run warms up
            _, prof = ph0.barcodes_profiled(pts, ws, tuning=tuning)
            best = min(best, prof[stage])
        return best

    chosen = {"dist_split16": -1, "dist_tile": -1, "sort_top_bits": -1}
    # distance kernel: split x tile
    dist = {}
    for split in (0, 4, 8, 12, 16):
        for tile in (64, 128):
            t = dict(chosen, dist_split16=split, dist_tile=tile)
            dist[(split, tile)] = stage_ms(t, "dist_ms")
    (split, tile), _ = min(dist.items(), key=lambda kv: kv[1])
    chosen.update(dist_split16=split, dist_tile=tile)
    # top radix pass width (the short sort's)
    sort = {bits: stage_ms(dict(chosen, sort_top_bits=bits, packed_sort=0), "sort_ms") for bits in (8, 9)}
    chosen["sort_top_bits"] = min(sort, key=sort.get)
    # the packed sort against the short sort, on the whole path
    whole = {}
    if len(x) * (len(x) - 1) // 2 >= 1 << 22 and len(x) <= 32768:
        whole = {p: stage_ms(dict(chosen, packed_sort=p), "total_ms") for p in (0, 1)}
        chosen["packed_sort"] = min(whole, key=whole.get)
    if verbose:
        print({"d": d, "dist_ms": {f"{k[0]}/{k[1]}": v for k, v in dist.items()},
               "sort_ms": sort, "whole_ms": whole, "chosen": chosen})
    _store(d, n, chosen)
    return chosen
