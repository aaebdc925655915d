"""Element-by-element parity with the oracle on a cloud with more edges than
one reduction window holds (E > 2^26), the regime of the 32768-point
benchmark cloud: 4 noisy circles of 3071 points in R^16 plus 4 far outliers,
N = 12288, 75,491,328 edges.  The outliers' edges are the longest, so the
last killing edges sit at the end of the edge order and the reduction scans
nearly every edge, through windows capped at 2^26 columns; the sort's fix-up
and the de-duplication counts run over 295k chunks.

Every field of every bar (Sec. 2: the bar (0, b) of each remaining pivot;
its killing edge, b = a, the pivot row, the position in the sorted order and
the squared and plain distance) is compared bit for bit, with |D| and the
bar that never dies, for the whole path and for the early-terminating path.
The oracle (single-threaded, all 75M columns reduced) takes about half a
minute here."""
import numpy as np
import pytest

import oracle
from paper_2203_02527_gb300 import inputs
from tests.test_gpu_parity import assert_bars_equal

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cloud():
    x = inputs.circles_with_outliers(3071, 4, 16, 4, seed=20260107)
    n = len(x)
    assert n == 12288 and n * (n - 1) // 2 > 2 ** 26
    want, inf_v, nd = oracle.barcodes(x)
    return x, want, inf_v, nd


def test_whole_path_equals_oracle_beyond_one_window(cloud):
    from paper_2203_02527_gb300 import ph0
    x, want, inf_v, nd = cloud
    m = len(x) * (len(x) - 1) // 2
    got = ph0.barcodes(torch.from_numpy(x).cuda())
    assert_bars_equal(got.numpy(), want)
    assert got.stats["n_distinct"] == nd
    assert got.inf == (inf_v, 0.0, float("inf"))
    # the scan really crossed capped windows and ended near the last edge
    assert got.stats["edges_scanned"] > 2 ** 26 and int(want["order"][-1]) > m - 50000
    assert got.stats["windows"] >= 3


def test_early_path_equals_oracle_beyond_one_window(cloud):
    from paper_2203_02527_gb300 import ph0
    x, want, inf_v, nd = cloud
    got = ph0.barcodes_early(torch.from_numpy(x).cuda(), rounds=True)
    assert_bars_equal(got.numpy(), want)
    assert got.inf == (inf_v, 0.0, float("inf"))
    # the prefix had to grow to every edge: its distinct count is |D|
    assert got.stats["sorted_edges"] == len(x) * (len(x) - 1) // 2
    assert got.stats["n_distinct"] == nd
    torch.cuda.empty_cache()


def test_large_cloud_form_equals_oracle_beyond_one_window(cloud):
    """The same cloud through the large-cloud form (edge-index records, the
    reduction's snapshot in global memory), forced on."""
    from paper_2203_02527_gb300 import ph0
    x, want, inf_v, nd = cloud
    got = ph0.barcodes(torch.from_numpy(x).cuda(), tuning={"wide_ids": 1})
    assert_bars_equal(got.numpy(), want)
    assert got.stats["n_distinct"] == nd
    assert got.inf == (inf_v, 0.0, float("inf"))
    torch.cuda.empty_cache()
