"""Pins of the oracle's filtration-prefix path (oracle.barcodes_below): on
the edges with d2 <= t_max alone it must give exactly the bars of the whole
path whose squared death is at most t_max -- same killing edges, positions in
the full sorted order, indices a and deaths -- because every edge that comes
before a kept edge in the total order (d2, u, v) is kept.  Checked against
oracle.barcodes (itself pinned in test_oracle_pins.py) and against a brute
count of the kept edges."""
import numpy as np
import pytest

import oracle
from paper_2203_02527_gb300 import inputs

CLOUDS = {
    "uniform2d": lambda: inputs.uniform(300, 2, seed=81),
    "mixture": lambda: inputs.gaussian_mixture(250, 3, k=4, sigma=0.3, seed=82),
    "lattice": lambda: inputs.lattice(9, 2),           # exact ties at the threshold
    "duplicates": lambda: inputs.with_duplicates(120, 3, 30, seed=83),
}


def _same(got, want):
    assert len(got) == len(want)
    assert got.tobytes() == want.tobytes()


@pytest.mark.parametrize("name", sorted(CLOUDS))
def test_prefix_at_or_above_the_last_death_is_the_whole_barcode(name):
    x = CLOUDS[name]()
    want, _, nd = oracle.barcodes(x)
    d2 = oracle.distances(x)
    top = float(want["death_sq"].max())
    for t in (top, float(np.nextafter(top, np.inf)), float("inf")):
        got, kept, nd_k = oracle.barcodes_below(x, t)
        _same(got, want)
        assert kept == int((d2 <= t).sum())
    assert oracle.barcodes_below(x, float("inf"))[2] == nd


@pytest.mark.parametrize("name", sorted(CLOUDS))
def test_prefix_below_a_death_keeps_the_earlier_bars(name):
    x = CLOUDS[name]()
    want, _, _ = oracle.barcodes(x)
    d2 = oracle.distances(x)
    deaths = np.unique(want["death_sq"])
    for t in deaths[len(deaths) // 2:len(deaths) // 2 + 3]:
        below = float(np.nextafter(t, -np.inf))
        got, kept, nd = oracle.barcodes_below(x, below)
        _same(got, want[want["death_sq"] <= below])
        assert kept == int((d2 <= below).sum())
        assert nd == len(np.unique(d2[d2 <= below]))
    got, kept, nd = oracle.barcodes_below(x, -1.0)
    assert len(got) == 0 and kept == 0 and nd == 0
