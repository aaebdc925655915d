"""The large-cloud form of the whole path: above 65535 points an edge record
holds the edge's lexicographic index instead of (u << 16) | v, and the
reduction reads its root snapshot from global memory (n up to 92681, where
E = n(n-1)/2 is just below 2^32).  Checked element by element against the
oracle:
  * on the parity cases, with the large-cloud form forced on small clouds
    (ph0_tuning.wide_ids = 1);
  * at the largest supported size, 92681 uniform points in the unit square
    (the paper's workload, Sec. 3.1 and Sec. 4; 4,294,837,140 edges), against
    the oracle's filtration-prefix path, which sorts and reduces only the
    edges up to the largest death and so yields every bar with its position
    in the whole sorted order and its index a."""
import numpy as np
import pytest

import oracle
from paper_2203_02527_gb300 import inputs
from tests.test_gpu_parity import CASES, assert_bars_equal

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WIDE = {"wide_ids": 1}


@pytest.mark.parametrize("case", sorted(CASES))
def test_forced_wide_records_match_oracle(case):
    from paper_2203_02527_gb300 import ph0
    x = CASES[case]()
    want, inf_v, nd = oracle.barcodes(x)
    got = ph0.barcodes(torch.from_numpy(np.ascontiguousarray(x)).cuda(), tuning=WIDE)
    assert_bars_equal(got.numpy(), want)
    assert got.stats["n_distinct"] == nd
    assert got.inf == (inf_v, 0.0, float("inf"))


@pytest.mark.parametrize("case", sorted(CASES))
def test_forced_wide_records_in_early_rounds_match_oracle(case):
    from paper_2203_02527_gb300 import ph0
    x = CASES[case]()
    want = oracle.barcodes(x)[0]
    got = ph0.barcodes_early(torch.from_numpy(np.ascontiguousarray(x)).cuda(), rounds=True, tuning=WIDE)
    assert_bars_equal(got.numpy(), want)


@pytest.mark.parametrize("n", [2, 3, 33, 257, 1000])
def test_forced_wide_small_and_ragged(n):
    from paper_2203_02527_gb300 import ph0
    x = inputs.uniform(n, 3, seed=900 + n)
    got = ph0.barcodes(torch.from_numpy(x).cuda(), tuning=WIDE)
    assert_bars_equal(got.numpy(), oracle.barcodes(x)[0])


def test_largest_cloud_equals_the_prefix_oracle():
    from paper_2203_02527_gb300 import ph0
    n = 92681
    x = inputs.uniform(n, 2, seed=20260108)
    ws = ph0.Workspace(n, 2)
    got = ph0.barcodes(torch.from_numpy(x).cuda(), ws=ws)
    bars = got.numpy()
    assert got.stats["status"] == 0 and got.stats["n_bars"] == n - 1
    assert got.stats["sorted_edges"] == n * (n - 1) // 2 > 2 ** 32 - 2 ** 18
    assert got.inf == (0, 0.0, float("inf"))
    want, kept, _ = oracle.barcodes_below(x, float(bars["death_sq"].max()))
    assert len(want) == n - 1 and kept < 10 ** 8
    assert_bars_equal(bars, want)
    # the early-terminating entry point sorts in rounds here too (a prefix of
    # the edges; its records hold edge indices as well)
    early = ph0.barcodes_early(torch.from_numpy(x).cuda(), ws=ws)
    assert_bars_equal(early.numpy(), want)
    assert early.stats["sorted_edges"] < n * (n - 1) // 2 // 10
    del ws, got, early
    torch.cuda.empty_cache()
