"""The stored barcodes (tests/golden/, written by make_golden.py from the
oracle): the oracle still produces them bit for bit, and they hold what the
paper's bars must (n-1 finite bars in filtration order, one pivot on every
row but row 0; on the integer grid every bar dies at 1 with a = 1, the
closed form of the grid)."""
import numpy as np
import pytest

import oracle
from tests import golden


@pytest.mark.parametrize("name", sorted(golden.FIXTURES))
def test_oracle_reproduces_the_stored_bars(name):
    meta, lines = golden.stored(name)
    x = golden.points(name)
    bars, inf_v, nd = oracle.barcodes(x)
    assert meta == {"n": len(x), "infinite_bar_vertex": inf_v, "distinct_distances": nd}
    assert golden.bar_lines(bars) == lines


@pytest.mark.parametrize("name", sorted(golden.FIXTURES))
def test_stored_bars_are_well_formed(name):
    meta, lines = golden.stored(name)
    assert len(lines) == meta["n"] - 1 and meta["infinite_bar_vertex"] == 0
    rows = [line.split() for line in lines]
    order = [int(r[4]) for r in rows]
    assert order == sorted(order) and len(set(order)) == len(order)
    for r in rows:
        u, v, a, low = int(r[0]), int(r[1]), int(r[2]), int(r[3])
        # the pivot row is the larger of the two component minima: at most v,
        # never row 0 (the infinite bar's vertex)
        assert 0 <= u < v < meta["n"] and 0 < low <= v and 1 <= a <= meta["distinct_distances"]
    lows = [int(r[3]) for r in rows]
    assert sorted(lows) == list(range(1, meta["n"]))  # every row but 0 is a pivot once
    if name == "lattice12":
        assert all(int(r[2]) == 1 for r in rows)
        assert all(np.uint64(int(r[5], 16)).view(np.float64) == 1.0 for r in rows)
