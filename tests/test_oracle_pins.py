"""Pins for the CPU oracle: it is checked against exact arithmetic, library
routines, Kruskal/union-find, Prim, brute-force sweeps and closed forms -- never
against itself.  Each mistake-planting test shows that a plausible error in the
oracle (a dropped term, a wrong index, a transposed tie-break, an off-by-one)
is caught by at least one pin."""
import math

import numpy as np
import pytest

import oracle
from paper_2203_02527_gb300 import inputs
from tests import pins


# ---------------------------------------------------------------- step 1 ---

def test_edge_enumeration():
    for n in (0, 1, 2, 5, 17):
        u, v = oracle.edge_endpoints(n)
        assert pins.check_edge_enumeration(n, u, v) is None


@pytest.mark.parametrize("d", [1, 2, 3, 7])
def test_distances_integer_exact(d):
    rng = np.random.default_rng(d)
    x = rng.integers(-1000, 1000, size=(23, d)).astype(np.float32)
    assert pins.check_d2_integer_exact(x, oracle.distances(x)) is None


@pytest.mark.parametrize("gen", ["uniform", "gaps", "negzero", "mixture"])
def test_distances_rational_replay(gen):
    x = {
        "uniform": lambda: inputs.uniform(14, 5, seed=3),
        "gaps": lambda: inputs.exponent_gaps(14, 4, seed=4),
        "negzero": lambda: inputs.negative_zero_mix(12, 3, seed=5),
        "mixture": lambda: inputs.gaussian_mixture(14, 16, k=3, seed=6),
    }[gen]()
    assert pins.check_d2_replay(x, oracle.distances(x)) is None


def test_distances_error_bound():
    x = inputs.uniform(20, 16, seed=7)
    assert pins.check_d2_error_bound(x, oracle.distances(x)) is None


def test_distances_signed_zero_and_one_dim():
    x = np.array([[0.0], [-0.0], [1.5], [-2.25]], np.float32)
    d2 = oracle.distances(x)
    # (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)
    assert d2.tolist() == [0.0, 2.25, 5.0625, 2.25, 5.0625, 14.0625]
    assert not np.signbit(d2[0])


def test_distances_rounding_cases():
    # fp32 values whose difference is not a binary64 number: must round
    x = np.array([[1.0], [1e-30]], np.float32)
    got = oracle.distances(x)[0]
    t = float(np.float64(np.float32(1e-30))) - 1.0
    assert got == pins.replay_d2([np.float32(1.0)], [np.float32(1e-30)])
    assert got == t * t


# ---------------------------------------------------------- steps 2 and 3 ---

@pytest.mark.parametrize("case", ["lattice", "dups", "uniform"])
def test_sort_matches_library_lexsort(case):
    x = {"lattice": lambda: inputs.lattice(5, 2),
         "dups": lambda: inputs.with_duplicates(40, 2, 9, seed=1),
         "uniform": lambda: inputs.uniform(60, 3, seed=2)}[case]()
    n = len(x)
    u, v = oracle.edge_endpoints(n)
    d2 = oracle.distances(x)
    assert pins.check_sorted(d2, u, v, oracle.sort_edges(d2, u, v)) is None


@pytest.mark.parametrize("case", ["lattice", "dups", "uniform", "allsame"])
def test_dedupe_matches_library_unique(case):
    x = {"lattice": lambda: inputs.lattice(6, 2),
         "dups": lambda: inputs.with_duplicates(50, 3, 7, seed=3),
         "uniform": lambda: inputs.uniform(50, 2, seed=4),
         "allsame": lambda: np.zeros((9, 2), np.float32)}[case]()
    n = len(x)
    u, v = oracle.edge_endpoints(n)
    d2 = oracle.distances(x)
    o = oracle.sort_edges(d2, u, v)
    a, nd = oracle.dedupe(d2[o])
    assert pins.check_dedupe(d2[o], a, nd) is None
    if case == "allsame":
        assert nd == 1 and set(a.tolist()) == {1}


# ---------------------------------------------------------- steps 4 and 5 ---

SMALL = {
    "uniform12": lambda: inputs.uniform(12, 2, seed=11),
    "uniform40": lambda: inputs.uniform(40, 3, seed=12),
    "mixture64": lambda: inputs.gaussian_mixture(64, 3, k=4, sigma=0.3, seed=13),
    "lattice4": lambda: inputs.lattice(4, 2),
    "lattice3x3x3": lambda: inputs.lattice(3, 3),
    "dups30": lambda: inputs.with_duplicates(30, 2, 6, seed=14),
    "gaps20": lambda: inputs.exponent_gaps(20, 3, seed=15),
    "negzero16": lambda: inputs.negative_zero_mix(16, 2, seed=16),
}


@pytest.mark.parametrize("case", sorted(SMALL))
def test_bars_against_kruskal_prim_and_rank(case):
    x = SMALL[case]()
    bars, inf_v, _ = oracle.barcodes(x)
    assert pins.check_bars_structure(len(x), bars, inf_v) is None
    assert pins.check_bars_kruskal(x, bars) is None
    assert pins.check_bars_prim(x, bars) is None
    assert pins.check_bars_a(x, bars) is None


@pytest.mark.parametrize("case", ["uniform12", "lattice4", "dups30", "negzero16"])
def test_bars_brute_force_sweep(case):
    x = SMALL[case]()
    bars, _, _ = oracle.barcodes(x)
    assert pins.check_bars_sweep(x, bars) is None


@pytest.mark.parametrize("case", ["uniform12", "lattice4", "dups30", "gaps20"])
def test_dense_f2t_reduction_agrees_and_is_homogeneous(case):
    x = SMALL[case]()
    p = oracle.pipeline(x)
    low_d, b_exp, hom = oracle.reduce_dense(len(x), p["u_sorted"], p["v_sorted"], p["a"])
    assert np.array_equal(low_d, p["low"])
    assert hom.all()
    piv = low_d >= 0
    assert np.array_equal(b_exp[piv], p["a"][piv].astype(np.int32))
    assert (b_exp[~piv] == -1).all()


def test_degenerate_sizes():
    b, iv, nd = oracle.barcodes(np.zeros((1, 3), np.float32))
    assert len(b) == 0 and iv == 0 and nd == 0
    b, iv, nd = oracle.barcodes(np.array([[0, 0], [3, 4]], np.float32))
    assert len(b) == 1 and iv == 0 and nd == 1
    assert (b[0]["u"], b[0]["v"], b[0]["a"], b[0]["low"], b[0]["order"]) == (0, 1, 1, 1, 0)
    assert b[0]["death_sq"] == 25.0 and b[0]["death"] == 5.0


# ------------------------------------------------------------ closed forms ---

def test_closed_form_collinear():
    # integer positions with distinct gaps on a line, vertex ids shuffled:
    # the killing edges join neighbours along the line, deaths = the gaps.
    rng = np.random.default_rng(21)
    pos = np.cumsum(rng.permutation(np.arange(1, 40)))  # distinct gaps 1..39
    pos = np.concatenate([[0], pos])
    perm = rng.permutation(len(pos))
    x = np.zeros((len(pos), 2), np.float32)
    x[perm, 0] = pos
    bars, inf_v, _ = oracle.barcodes(x)
    gaps = np.diff(pos)
    assert np.array_equal(np.sort(bars["death"]), np.sort(gaps.astype(np.float64)))
    neighbours = {tuple(sorted((int(perm[k]), int(perm[k + 1])))) for k in range(len(pos) - 1)}
    assert {(int(b["u"]), int(b["v"])) for b in bars} == neighbours
    # deaths come out increasing, one new distance each: a = 1..N-1 in order
    assert np.all(np.diff(bars["death"]) > 0)


def test_closed_form_regular_simplex():
    n = 9
    x = np.eye(n, dtype=np.float32)  # all squared distances exactly 2
    bars, inf_v, nd = oracle.barcodes(x)
    assert nd == 1
    assert [(int(b["u"]), int(b["v"])) for b in bars] == [(0, j) for j in range(1, n)]
    assert (bars["a"] == 1).all() and (bars["death_sq"] == 2.0).all()
    assert (bars["death"] == math.sqrt(2.0)).all()
    assert bars["low"].tolist() == list(range(1, n))


def test_closed_form_two_far_clusters():
    rng = np.random.default_rng(22)
    a = rng.random((15, 3)).astype(np.float32)
    b = (rng.random((17, 3)) + 100.0).astype(np.float32)
    x = np.concatenate([a, b])
    bars, _, _ = oracle.barcodes(x)
    x64 = x.astype(np.float64)
    cross = ((x64[:15, None, :] - x64[None, 15:, :]) ** 2).sum(-1).min()
    diam = max(((x64[:15, None] - x64[None, :15]) ** 2).sum(-1).max(),
               ((x64[15:, None] - x64[None, 15:]) ** 2).sum(-1).max())
    long_bars = bars[bars["death_sq"] > diam]
    assert len(long_bars) == 1
    assert long_bars[0]["death_sq"] == pytest.approx(cross, rel=1e-12)
    assert int(long_bars[0]["order"]) == int(bars["order"].max())


def test_closed_form_grid():
    x = inputs.lattice(7, 2)
    bars, _, nd = oracle.barcodes(x)
    assert (bars["death_sq"] == 1.0).all() and (bars["a"] == 1).all()
    assert len(bars) == 48


# ---------------------------------------------------- planted mistakes ----

def test_pins_catch_planted_mistakes():
    x = np.random.default_rng(5).integers(-9, 9, size=(11, 3)).astype(np.float32)
    n = len(x)
    d2 = oracle.distances(x)
    # dropped term in the distance (last dimension ignored)
    dropped = oracle.distances(x[:, :2])
    assert pins.check_d2_integer_exact(x, dropped) is not None
    # wrong index: v - v instead of v - u in one dimension
    assert pins.check_d2_integer_exact(x, d2 * 0.5) is not None
    u, v = oracle.edge_endpoints(n)
    order = oracle.sort_edges(d2, u, v)
    # transposed tie-break (v before u)
    wrong = np.lexsort((u, v, d2))
    if not np.array_equal(wrong, order):
        assert pins.check_sorted(d2, u, v, wrong) is not None
    # off-by-one index a
    a, nd = oracle.dedupe(d2[order])
    assert pins.check_dedupe(d2[order], a - 1, nd) is not None
    # missing a bar / wrong pivot convention / wrong death
    bars, inf_v, _ = oracle.barcodes(x)
    assert pins.check_bars_structure(n, bars[:-1], inf_v) is not None
    wrong_low = bars.copy()
    wrong_low["low"] = np.minimum(wrong_low["u"], wrong_low["v"])
    assert pins.check_bars_kruskal(x, wrong_low) is not None
    wrong_edge = bars.copy()
    wrong_edge["death_sq"][-1] = np.nextafter(wrong_edge["death_sq"][-1], np.inf)
    assert pins.check_bars_kruskal(x, wrong_edge) is not None
    assert pins.check_bars_prim(x, wrong_edge) is not None
    # a bar that dies one level late breaks the sweep
    late = bars.copy()
    late["death_sq"][0] = late["death_sq"][-1] + 1.0
    assert pins.check_bars_sweep(x, late) is not None
