"""Writes the stored barcodes under tests/golden/ from the CPU oracle alone
(the paper prints no barcode values, so these fixtures pin the oracle's
output of the paper's bars (0, b) of Sec. 2 on seeded inputs against later
changes, and give the GPU tests expected values that do not need the
oracle at test time).  Run from the repository root:

    python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from tests import golden  # noqa: E402


def write(name: str) -> str:
    desc, make = golden.FIXTURES[name]
    x = make()
    bars, inf_v, nd = oracle.barcodes(x)
    with open(golden.path(name), "w") as f:
        f.write("# bars (0, b) of the Vietoris-Rips filtration (Rawson, Sec. 2), from the CPU oracle\n")
        f.write("# input: %s\n" % desc)
        f.write("# n=%d infinite_bar_vertex=%d distinct_distances=%d\n" % (len(x), inf_v, nd))
        f.write("# u v a low order death_sq(binary64 bits, hex) death(binary64 bits, hex)\n")
        for line in golden.bar_lines(bars):
            f.write(line + "\n")
    return golden.path(name)


if __name__ == "__main__":
    for name in golden.FIXTURES:
        print(write(name))
