"""First homology on the GPU (ph0_h1: the pairs of the Vietoris-Rips
2-skeleton through the coboundary matrix, apparent pairs, the dimension-0
forest cleared, the other columns reduced) against the oracle's literal
left-to-right reduction of the edge-by-triangle boundary matrix, every field
of every bar, bit for bit: the birth edge, the death triangle, the indices a
of both, their positions in the edge and triangle orders, and the squared
distances.  The two share no step beyond the edge order."""
import numpy as np
import pytest

import oracle
from paper_2203_02527_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CLOUDS = {
    "square": lambda: np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float32),
    "uniform2d_64": lambda: inputs.uniform(64, 2, seed=31),
    "uniform2d_200": lambda: inputs.uniform(200, 2, seed=32),
    "uniform3d_150": lambda: inputs.uniform(150, 3, seed=33),
    "mixture_d8": lambda: inputs.gaussian_mixture(120, 8, k=4, sigma=0.3, seed=34),
    "mixture_d16": lambda: inputs.gaussian_mixture(200, 16, k=5, sigma=0.3, seed=39),
    "circles_d4": lambda: inputs.noisy_circles(40, 3, 4, noise=0.05, seed=35),
    "lattice_ties": lambda: inputs.lattice(9, 2),
    "duplicates": lambda: inputs.with_duplicates(90, 2, 30, seed=36),
    "negative_zero": lambda: inputs.negative_zero_mix(60, 3, seed=37),
}


def _check(x):
    from paper_2203_02527_gb300 import ph0
    want, ntri = oracle.h1(x)
    got, st = ph0.h1(torch.from_numpy(np.ascontiguousarray(x)).cuda())
    assert st["n_triangles"] == ntri and st["n_bars"] == len(want)
    for f in ("eu", "ev", "tu", "tv", "tw", "birth_a", "death_a", "birth_order", "death_order", "death_rank"):
        np.testing.assert_array_equal(got[f], want[f], err_msg=f)
    for f in ("birth_sq", "death_sq"):
        np.testing.assert_array_equal(got[f].view(np.uint64), want[f].view(np.uint64), err_msg=f)
    return st


@pytest.mark.parametrize("name", sorted(CLOUDS))
def test_h1_equals_oracle(name):
    _check(CLOUDS[name]())


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 33])
def test_h1_small_and_ragged(n):
    _check(inputs.uniform(n, 2, seed=300 + n))


def test_h1_reduced_columns_and_counts():
    # 300 points: 4.5M triangles, dozens of columns that need additions
    x = inputs.uniform(300, 2, seed=38)
    st = _check(x)
    n, m = 300, 300 * 299 // 2
    assert st["n_triangles"] == n * (n - 1) * (n - 2) // 6
    assert st["reduced"] > 10 and st["additions"] >= st["reduced"]
    assert st["apparent"] + st["reduced"] == m - (n - 1)
    assert st["max_column"] >= n - 2 and st["pool_entries"] > 0
    # every stage ran on the device and was timed on the call's stream
    assert all(st[k] > 0 for k in ("edges_ms", "scan_ms", "reduce_ms", "emit_ms"))


@pytest.mark.parametrize("n", [700, 2048])
def test_h1_structure_at_large_sizes(n):
    """700 uniform points in the unit square (the paper's largest N; 57M
    triangles, too many for the oracle's literal reduction in a test) and
    2048 points (1.4G triangles): every positive edge dies, the births are
    exactly the edges that end no class in dimension 0 (from the GPU's own
    dimension-0 bars, themselves checked against the oracle elsewhere), each
    death comes at or after its birth, the death triangle's diameter is its
    latest edge, and the indices follow the sorted distances."""
    from paper_2203_02527_gb300 import ph0
    x = inputs.uniform(n, 2, seed=39 if n == 700 else 40)
    pts = torch.from_numpy(x).cuda()
    bars, st = ph0.h1(pts)
    m = n * (n - 1) // 2
    assert st["n_triangles"] == n * (n - 1) * (n - 2) // 6
    assert st["n_bars"] == len(bars) == m - (n - 1)
    h0 = ph0.barcodes(pts).numpy()
    killing = set(zip(h0["u"].tolist(), h0["v"].tolist()))
    births = set(zip(bars["eu"].tolist(), bars["ev"].tolist()))
    assert len(births) == len(bars) and births.isdisjoint(killing) and len(births) + len(killing) == m
    assert (bars["death_order"] >= bars["birth_order"]).all()
    assert (np.diff(bars["death_rank"]) > 0).all()
    assert (bars["death_sq"] >= bars["birth_sq"]).all()
    assert np.array_equal(bars["birth_a"] <= bars["death_a"], np.ones(len(bars), bool))
    # a agrees with the order of the squared distances
    o = np.argsort(bars["birth_order"])
    assert (np.diff(bars["birth_a"][o].astype(np.int64)) >= 0).all()
    # on a sample of bars: the death triangle's longest edge (binary64
    # distances of the binary32 points) and the birth edge give the bar's
    # squared distances
    x64 = x.astype(np.float64)
    rng = np.random.default_rng(41)
    for i in rng.choice(len(bars), size=200, replace=False):
        r = bars[i]
        t = (int(r["tu"]), int(r["tv"]), int(r["tw"]))
        assert t[0] < t[1] < t[2]
        d2 = [float(((x64[p] - x64[q]) ** 2).sum()) for p, q in ((t[0], t[1]), (t[0], t[2]), (t[1], t[2]))]
        assert np.isclose(max(d2), r["death_sq"], rtol=1e-12)
        e = (int(r["eu"]), int(r["ev"]))
        assert np.isclose(float(((x64[e[0]] - x64[e[1]]) ** 2).sum()), r["birth_sq"], rtol=1e-12)
