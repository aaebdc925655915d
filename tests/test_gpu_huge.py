"""Clouds of more than 2^32 edges (92,683 to 131,071 points): the edge index
has 33 bits, its bit 32 carried in the key's sign bit; the whole path sorts
the two halves of the edge array (each below 2^32 records) and merges them
by value, the first half first among equal values.  Checked element by
element against the oracle:
  * with the split sort forced on small clouds (ph0_tuning.split_sort = 1),
    on every parity case, alone and with the edge-index records forced too,
    on ragged sizes and on crowded keys whose halves take the complete sort;
  * on 100,000 uniform points in the unit square (the paper's workload, Sec.
    3.1 and Sec. 4; 4,999,950,000 edges), against the oracle's
    filtration-prefix path, which yields every bar with its position in the
    whole sorted order and its index a."""
import numpy as np
import pytest

import oracle
from paper_2203_02527_gb300 import inputs
from tests.test_gpu_parity import CASES, assert_bars_equal

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPLIT = {"split_sort": 1}
SPLIT_WIDE = {"split_sort": 1, "wide_ids": 1}


@pytest.mark.parametrize("case", sorted(CASES))
def test_forced_split_sort_matches_oracle(case):
    from paper_2203_02527_gb300 import ph0
    x = CASES[case]()
    want, inf_v, nd = oracle.barcodes(x)
    pts = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    for tuning in (SPLIT, SPLIT_WIDE):
        got = ph0.barcodes(pts, tuning=tuning)
        assert_bars_equal(got.numpy(), want)
        assert got.stats["n_distinct"] == nd
        assert got.inf == (inf_v, 0.0, float("inf"))


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 33, 257, 1000])
def test_forced_split_small_and_ragged(n):
    from paper_2203_02527_gb300 import ph0
    x = inputs.uniform(n, 3, seed=1900 + n)
    got = ph0.barcodes(torch.from_numpy(x).cuda(), tuning=SPLIT)
    assert_bars_equal(got.numpy(), oracle.barcodes(x)[0])


def test_forced_split_crowded_halves_take_the_complete_sort():
    """Two clusters within 1e-12 of two points at distance 1: the cross
    distances form long groups of equal key >> 16 out of order in both
    halves, so each half's fix-up hands over to its complete sort."""
    from paper_2203_02527_gb300 import ph0
    rng = np.random.default_rng(43)
    a = rng.random((900, 3)) * 1e-12
    b = rng.random((900, 3)) * 1e-12
    b[:, 1] = 1.0
    x = np.ascontiguousarray(np.concatenate([a, b]), dtype=np.float32)
    got = ph0.barcodes(torch.from_numpy(x).cuda(), tuning=SPLIT)
    assert_bars_equal(got.numpy(), oracle.barcodes(x)[0])


def test_hundred_thousand_points_equal_the_prefix_oracle():
    from paper_2203_02527_gb300 import ph0
    n = 100000
    m = n * (n - 1) // 2
    assert m > 2 ** 32  # 705M edge indices have bit 32 set
    x = inputs.uniform(n, 2, seed=20260110)
    ws = ph0.Workspace(n, 2)
    got = ph0.barcodes(torch.from_numpy(x).cuda(), ws=ws)
    bars = got.numpy()
    assert got.stats["status"] == 0 and got.stats["n_bars"] == n - 1
    assert got.stats["sorted_edges"] == m
    assert got.inf == (0, 0.0, float("inf"))
    want, kept, _ = oracle.barcodes_below(x, float(bars["death_sq"].max()))
    assert len(want) == n - 1 and kept < 2 * 10 ** 8
    assert_bars_equal(bars, want)
    # killing edges whose index has bit 32 set decode to the right (u, v)
    e = bars["u"].astype(np.int64) * (2 * n - bars["u"].astype(np.int64) - 1) // 2 + bars["v"] - bars["u"] - 1
    assert (e >= 2 ** 32).sum() > 1000
    del ws, got
    torch.cuda.empty_cache()
