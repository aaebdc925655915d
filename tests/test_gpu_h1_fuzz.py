"""First homology on seeded random clouds of every kind the dimension-0 fuzz
covers (uniform, Gaussian mixtures, duplicates, exponent gaps, signed zeros,
lattices, two crowded clusters, perturbed simplices, noisy circles) plus all
points identical and points on a line, at sizes the oracle's literal
boundary-matrix reduction finishes quickly: ph0_h1 (coboundary form) against
it, every field of every bar, bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2203_02527_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KINDS = 11
FIELDS = ("eu", "ev", "tu", "tv", "tw", "birth_a", "death_a", "birth_order", "death_order", "death_rank")


def _cloud(rng: np.random.Generator, kind: int) -> np.ndarray:
    n = int(rng.integers(3, 80))
    d = int(rng.choice([1, 2, 3, 5, 8, 16]))
    s = int(rng.integers(1 << 30))
    if kind == 0:
        x = inputs.uniform(n, d, seed=s)
    elif kind == 1:
        x = inputs.gaussian_mixture(n, d, k=int(rng.integers(1, 6)), sigma=float(rng.uniform(0.001, 0.3)), seed=s)
    elif kind == 2:
        x = inputs.with_duplicates(n, d, max(1, n // int(rng.integers(2, 10))), seed=s)
    elif kind == 3:
        x = inputs.exponent_gaps(n, d, seed=s)
    elif kind == 4:
        x = inputs.negative_zero_mix(n, d, seed=s)
    elif kind == 5:
        x = inputs.lattice(int(rng.integers(2, 7)), int(rng.integers(1, 4)))
    elif kind == 6:  # two clusters within 1e-12 of two points at distance 1
        a = rng.random((n // 2 + 1, 3)) * 1e-12
        b = rng.random((n // 2 + 1, 3)) * 1e-12
        b[:, 1] = 1.0
        x = np.concatenate([a, b])
    elif kind == 7:  # simplex vertices with tiny off-diagonal perturbations
        x = np.eye(n) + rng.random((n, n)) * float(rng.choice([3e-16, 1e-12, 1e-8]))
        np.fill_diagonal(x, 1.0)
    elif kind == 8:
        x = inputs.noisy_circles(max(1, n // 3), 3, max(d, 2), noise=float(rng.uniform(0.0, 0.05)), seed=s)
    elif kind == 9:  # every point the same: all distances tie at zero
        x = np.tile(rng.random((1, d)), (n, 1))
    else:  # points on a line
        x = np.outer(rng.random(n), rng.random(d))
    return np.ascontiguousarray(x, dtype=np.float32)


@pytest.mark.parametrize("seed", list(range(201, 211)))
def test_h1_random_clouds_bit_exact(seed):
    from paper_2203_02527_gb300 import ph0
    rng = np.random.default_rng(seed)
    for kind in range(KINDS):
        x = _cloud(rng, kind)
        want, ntri = oracle.h1(x)
        got, st = ph0.h1(torch.from_numpy(x).cuda())
        where = (seed, kind, x.shape)
        assert st["n_triangles"] == ntri and len(got) == len(want), where
        assert st["apparent"] + st["reduced"] == len(want), where
        for f in FIELDS:
            np.testing.assert_array_equal(got[f], want[f], err_msg=f"{f} {where}")
        for f in ("birth_sq", "death_sq"):
            np.testing.assert_array_equal(got[f].view(np.uint64), want[f].view(np.uint64), err_msg=f"{f} {where}")
