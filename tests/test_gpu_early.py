"""The early-terminating path (ph0_barcodes_early): it sorts only a prefix of
the edge order, grown in rounds until the reduction finds n-1 pivots in it,
and must return exactly the bars of the whole path (and of the oracle):
same killing edges, positions in the full sorted order, indices a and
deaths.  Covers the parity cases, small and ragged sizes, clouds whose
prefix must grow to all edges (a prefix of 45% is not enough, or all keys
fall in one bin), and the benchmark cloud at full size."""
import numpy as np
import pytest

import oracle
from paper_2203_02527_gb300 import inputs
from tests.test_gpu_parity import CASES, assert_bars_equal

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ph0():
    from paper_2203_02527_gb300 import ph0
    return ph0


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("case", sorted(CASES))
def test_early_matches_oracle(case):
    x = CASES[case]()
    want, inf_v, _ = oracle.barcodes(x)
    got = _ph0().barcodes_early(_cuda(x), rounds=True)
    assert_bars_equal(got.numpy(), want)
    assert got.stats["status"] == 0 and got.stats["n_bars"] == len(x) - 1
    assert got.inf == (inf_v, 0.0, float("inf"))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 31, 33, 129, 257, 1000])
def test_early_small_and_ragged(n):
    x = inputs.uniform(n, 3, seed=500 + n)
    want, inf_v, _ = oracle.barcodes(x)
    got = _ph0().barcodes_early(_cuda(x), rounds=True)
    assert_bars_equal(got.numpy(), want)
    assert got.inf == (inf_v, 0.0, float("inf"))


def test_early_sorts_a_short_prefix_of_a_uniform_cloud():
    # uniform cloud: the longest killing edge is far shorter than a typical
    # distance, so the first round's prefix already holds every killing edge
    x = inputs.uniform(4096, 3, seed=21)
    got = _ph0().barcodes_early(_cuda(x), rounds=True)
    assert_bars_equal(got.numpy(), oracle.barcodes(x)[0])
    m = len(x) * (len(x) - 1) // 2
    assert 0 < got.stats["sorted_edges"] < m // 10


def test_early_on_a_gaussian_mixture():
    # 8 clusters: the last merge comes late in the edge order (fallback or
    # a late round); the result is the same either way
    x = inputs.config_points("mixture4096")
    assert_bars_equal(_ph0().barcodes_early(_cuda(x), rounds=True).numpy(), oracle.barcodes(x)[0])


def test_early_sorts_everything_when_the_prefix_is_not_enough():
    # two far clusters of equal size: the bridge comes after all edges inside
    # the clusters (about half of the edges), past the last round
    rng = np.random.default_rng(7)
    a = rng.random((150, 3)).astype(np.float32)
    x = np.concatenate([a, a[::-1] + np.float32(100.0)]).astype(np.float32)
    got = _ph0().barcodes_early(_cuda(x), rounds=True)
    assert_bars_equal(got.numpy(), oracle.barcodes(x)[0])
    assert got.stats["sorted_edges"] == len(x) * (len(x) - 1) // 2  # every class
    # all points equal: one key, one bin
    y = np.full((60, 4), 0.5, np.float32)
    assert_bars_equal(_ph0().barcodes_early(_cuda(y), rounds=True).numpy(), oracle.barcodes(y)[0])


def test_early_reports_nonfinite_input():
    from paper_2203_02527_gb300._lib import Ph0Error
    x = inputs.uniform(50, 3, seed=9)
    x[3, 2] = np.nan
    with pytest.raises(Ph0Error) as e:
        _ph0().barcodes_early(_cuda(x), rounds=True)
    assert e.value.code == 2


def test_early_equals_whole_path_on_the_benchmark_cloud():
    ph0 = _ph0()
    x = inputs.config_points("circles32768")
    pts = _cuda(x)
    ws = ph0.Workspace(len(x), x.shape[1])
    whole = ph0.barcodes(pts, ws=ws).numpy()
    got = ph0.barcodes_early(pts, ws=ws, rounds=True)
    assert_bars_equal(got.numpy(), whole)
    m = len(x) * (len(x) - 1) // 2
    assert got.stats["sorted_edges"] < m
    del ws
    torch.cuda.empty_cache()


def test_built_in_choice_takes_the_whole_path_below_2_27_edges():
    # a 4096-point cloud (8.4M edges): the rounds would cost more than they save
    ph0 = _ph0()
    x = inputs.uniform(4096, 3, seed=21)
    m = len(x) * (len(x) - 1) // 2
    want = oracle.barcodes(x)[0]
    for rounds in (None, False):
        got = ph0.barcodes_early(_cuda(x), rounds=rounds)
        assert_bars_equal(got.numpy(), want)
        assert got.stats["sorted_edges"] == m
