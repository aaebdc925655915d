"""Pins of the oracle's first-homology path (oracle.h1: the edge-by-triangle
boundary matrix of the Vietoris-Rips 2-skeleton reduced left to right, the
extension the paper names in Sec. 1 and Sec. 4.2), each independent of the
reduction it checks:
  * closed form: the unit square has one nonzero bar, born at the side
    (d2 = 1) and dying at the diagonal (d2 = 2);
  * every positive edge dies (the full simplex has no first homology): the
    bars number n(n-1)/2 - (n-1), and their birth edges are exactly the
    edges that end no class in dimension 0 (the complement of the oracle's
    killing edges);
  * brute force on tiny clouds: at every filtration value, the number of bars
    alive equals the first Betti number of the complex, computed as
    #edges - #vertices + #components - rank_F2(boundary of the triangles);
  * positions and indices agree with the dimension-0 pipeline's sorted
    edges and a."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2203_02527_gb300 import inputs


def gf2_rank(mat: np.ndarray) -> int:
    m = (mat.copy() & 1).astype(np.uint8)
    rank, rows, cols = 0, m.shape[0], m.shape[1]
    for c in range(cols):
        piv = next((r for r in range(rank, rows) if m[r, c]), None)
        if piv is None:
            continue
        m[[rank, piv]] = m[[piv, rank]]
        for r in range(rows):
            if r != rank and m[r, c]:
                m[r] ^= m[rank]
        rank += 1
    return rank


def components(n, edges):
    parent = list(range(n))

    def find(i):
        while parent[i] != i:
            parent[i] = parent[parent[i]]
            i = parent[i]
        return i
    for u, v in edges:
        parent[find(u)] = find(v)
    return len({find(i) for i in range(n)})


def betti1(x, eps):
    """First Betti number of the 2-skeleton at squared scale eps (edges and
    triangles with d2 <= eps), by ranks over F2."""
    n = len(x)
    d2 = {}
    for u, v in itertools.combinations(range(n), 2):
        d2[(u, v)] = oracle.distances(np.stack([x[u], x[v]]))[0]
    edges = [e for e in d2 if d2[e] <= eps]
    index = {e: i for i, e in enumerate(edges)}
    tris = [t for t in itertools.combinations(range(n), 3)
            if all(d2[p] <= eps for p in itertools.combinations(t, 2))]
    if tris and edges:
        bd = np.zeros((len(edges), len(tris)), np.uint8)
        for j, t in enumerate(tris):
            for p in itertools.combinations(t, 2):
                bd[index[p], j] = 1
        r = gf2_rank(bd)
    else:
        r = 0
    return len(edges) - n + components(n, edges) - r


def test_unit_square_closed_form():
    x = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float32)
    bars, ntri = oracle.h1(x)
    assert ntri == 4 and len(bars) == 3
    live = bars[bars["death_sq"] > bars["birth_sq"]]
    assert len(live) == 1
    assert (live["birth_sq"][0], live["death_sq"][0]) == (1.0, 2.0)


@pytest.mark.parametrize("make", [
    lambda: inputs.uniform(40, 2, seed=11),
    lambda: inputs.gaussian_mixture(35, 3, k=3, sigma=0.3, seed=12),
    lambda: inputs.lattice(5, 2),
    lambda: inputs.with_duplicates(30, 2, 12, seed=13),
    lambda: inputs.noisy_circles(12, 2, 4, noise=0.05, seed=14),
])
def test_every_positive_edge_dies_and_births_complement_the_killing_edges(make):
    x = make()
    n = len(x)
    bars, _ = oracle.h1(x)
    m = n * (n - 1) // 2
    assert len(bars) == m - (n - 1)
    h0, _, _ = oracle.barcodes(x)
    killing = set(zip(h0["u"].tolist(), h0["v"].tolist()))
    births = set(zip(bars["eu"].tolist(), bars["ev"].tolist()))
    assert len(births) == len(bars) and births.isdisjoint(killing)
    assert len(births) + len(killing) == m
    # positions and indices from the dimension-0 pipeline
    ref = oracle.pipeline(x)
    bo, do = bars["birth_order"], bars["death_order"]
    np.testing.assert_array_equal(ref["u_sorted"][bo], bars["eu"])
    np.testing.assert_array_equal(ref["v_sorted"][bo], bars["ev"])
    np.testing.assert_array_equal(ref["a"][bo], bars["birth_a"])
    np.testing.assert_array_equal(ref["a"][do], bars["death_a"])
    np.testing.assert_array_equal(ref["d2_sorted"][bo], bars["birth_sq"])
    np.testing.assert_array_equal(ref["d2_sorted"][do], bars["death_sq"])
    assert (do >= bo).all() and (np.diff(bars["death_rank"]) > 0).all()


@pytest.mark.parametrize("seed", [21, 22, 23, 24])
def test_bars_alive_equal_betti1_by_brute_force(seed):
    x = inputs.uniform(8, 2, seed=seed)
    bars, _ = oracle.h1(x)
    for eps in np.unique(oracle.distances(x)):
        alive = int(((bars["birth_sq"] <= eps) & (eps < bars["death_sq"])).sum())
        assert alive == betti1(x, eps), eps


def test_circle_has_one_long_bar():
    # 12 points on a circle (radius 1, tiny noise): the cycle is born at the
    # side of the 12-gon and dies once a triangle reaches around the centre,
    # at the chord spanning 4 of the 12 steps (the equilateral triangle)
    th = np.arange(12) * (2 * np.pi / 12)
    rng = np.random.default_rng(5)
    x = (np.stack([np.cos(th), np.sin(th)], 1) + rng.normal(0, 1e-4, (12, 2))).astype(np.float32)
    bars, _ = oracle.h1(x)
    life = bars["death_sq"] - bars["birth_sq"]
    top = bars[np.argmax(life)]
    side2, tri2 = (2 * np.sin(np.pi / 12)) ** 2, (2 * np.sin(4 * np.pi / 12)) ** 2
    assert abs(top["birth_sq"] - side2) < 1e-2 and abs(top["death_sq"] - tri2) < 1e-2
    assert (np.sort(life)[-2] < 0.1 * life.max())
