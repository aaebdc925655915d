"""Stored barcodes (text fixtures) and the seeded inputs they belong to.

The paper prints no barcode values, so every fixture here was written by
make_golden.py from the CPU oracle alone; each file's header names its
input and the passage it follows (the bars (0, b) of Sec. 2).  This module
only reads them: it imports neither the oracle nor the CUDA library."""
import os

import numpy as np

from paper_2203_02527_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))

# name -> (description of the input, points)
FIXTURES = {
    "uniform256": ("inputs.config_points('uniform256'): N=256, d=3, U[0,1)^3, seed 20260101",
                   lambda: inputs.config_points("uniform256")),
    "lattice12": ("inputs.lattice(12, 2): the 12 x 12 integer grid (every bar dies at 1, a = 1)",
                  lambda: inputs.lattice(12, 2)),
    "duplicates": ("inputs.with_duplicates(120, 3, 40, seed=34): 120 points drawn from 40 (zero-length bars)",
                   lambda: inputs.with_duplicates(120, 3, 40, seed=34)),
}


def points(name: str) -> np.ndarray:
    return FIXTURES[name][1]()


def path(name: str) -> str:
    return os.path.join(HERE, name + "_bars.txt")


def bar_lines(bars) -> list:
    """One text line per bar: u v a low order death_sq death (binary64 bits
    in hex), in filtration order."""
    out = []
    for b in bars:
        out.append("%d %d %d %d %d %016x %016x" % (
            b["u"], b["v"], b["a"], b["low"], b["order"],
            np.float64(b["death_sq"]).view(np.uint64), np.float64(b["death"]).view(np.uint64)))
    return out


def stored(name: str):
    """(header fields as a dict, bar lines) of a fixture file."""
    meta, lines = {}, []
    with open(path(name)) as f:
        for line in f:
            line = line.rstrip("\n")
            if line.startswith("# n="):
                meta = dict(kv.split("=") for kv in line[2:].split())
            elif line and not line.startswith("#"):
                lines.append(line)
    return {k: int(v) for k, v in meta.items()}, lines
