"""Seeded random clouds of every kind the parity cases cover (uniform,
Gaussian mixtures, duplicates, exponent gaps, signed zeros, lattices, two
crowded clusters, perturbed simplices, noisy circles) with random sizes and
dimensions: the whole path, the early-terminating path and the large-cloud
form against the oracle, bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2203_02527_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KINDS = 9


def _cloud(rng: np.random.Generator, kind: int) -> np.ndarray:
    n = int(rng.integers(2, 2500))
    d = int(rng.choice([1, 2, 3, 5, 8, 16, 32, 40]))
    s = int(rng.integers(1 << 30))
    if kind == 0:
        x = inputs.uniform(n, d, seed=s)
    elif kind == 1:
        x = inputs.gaussian_mixture(n, d, k=int(rng.integers(1, 9)), sigma=float(rng.uniform(0.001, 0.3)), seed=s)
    elif kind == 2:
        x = inputs.with_duplicates(n, d, max(1, n // int(rng.integers(2, 20))), seed=s)
    elif kind == 3:
        x = inputs.exponent_gaps(n, d, seed=s)
    elif kind == 4:
        x = inputs.negative_zero_mix(n, d, seed=s)
    elif kind == 5:
        k = max(2, int(round(n ** (1.0 / min(d, 3)))))
        x = inputs.lattice(min(k, 40), min(d, 3))
    elif kind == 6:  # two clusters within 1e-12 of two points at distance 1
        a = rng.random((n // 2 + 1, 3)) * 1e-12
        b = rng.random((n // 2 + 1, 3)) * 1e-12
        b[:, 1] = 1.0
        x = np.concatenate([a, b])
    elif kind == 7:  # simplex vertices with tiny off-diagonal perturbations
        m = min(n, 200)
        x = np.eye(m) + rng.random((m, m)) * float(rng.choice([3e-16, 1e-15, 1e-14, 1e-12, 1e-10, 1e-8]))
        np.fill_diagonal(x, 1.0)
    else:
        x = inputs.noisy_circles(max(1, n // 4), 4, max(d, 2), noise=float(rng.uniform(0.0, 0.05)), seed=s)
    return np.ascontiguousarray(x, dtype=np.float32)


def _equal(got: np.ndarray, want: np.ndarray) -> bool:
    if len(got) != len(want):
        return False
    for f in ("u", "v", "a", "low", "order"):
        if not np.array_equal(got[f], want[f]):
            return False
    return all(np.array_equal(got[f].view(np.uint64), want[f].view(np.uint64)) for f in ("death_sq", "death"))


@pytest.mark.parametrize("seed", [101, 102, 103, 104, 105])
def test_random_clouds_bit_exact(seed):
    from paper_2203_02527_gb300 import ph0
    rng = np.random.default_rng(seed)
    for kind in range(KINDS):
        x = _cloud(rng, kind)
        want = oracle.barcodes(x)[0]
        pts = torch.from_numpy(x).cuda()
        assert _equal(ph0.barcodes(pts).numpy(), want), (seed, kind, x.shape)
        assert _equal(ph0.barcodes_early(pts, rounds=True).numpy(), want), (seed, kind, x.shape, "early")
        # the large-cloud form (edge-index records), forced on
        assert _equal(ph0.barcodes(pts, tuning={"wide_ids": 1}).numpy(), want), (seed, kind, x.shape, "wide")
