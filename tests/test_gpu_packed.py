"""The packed sort of the whole path: each edge one 64-bit word (the number
of its key's top part among the values that occur, key bits 22..47,
(u << 15) | v), sorted by four radix passes, then a fix-up that orders every
group of equal key >> 22 by the whole key and writes the records of steps 3-5.
Checked element by element against the oracle on every bar field (Rawson,
Sec. 2: the bars (0, b), b the index of the killing edge's distance in D;
its edge, position and pivot row), with |D| and the bar that never dies:
  * forced (ph0_tuning.packed_sort = 1) on every parity case and on ragged
    sizes, and by the built-in choice (from 2^22 edges) on clouds whose
    groups of equal key >> 22 reach across the fix-up's chunks;
  * the form that ran (ph0_stats.sort_form) equals the one the oracle's keys
    call for: packed when the top part spans fewer than 512 values of which at
    most 256 occur, else the short sort; and the complete sort when a group
    longer than 32 records is out of edge order or longer than 4096."""
import numpy as np
import pytest

import oracle
from paper_2203_02527_gb300 import inputs
from tests.test_gpu_parity import CASES, assert_bars_equal

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PACKED = {"packed_sort": 1}


def expected_form(ref, n):
    """0 short sort, 1 packed sort, 2 complete sort, from the oracle's keys in
    edge order (d2) and sorted order (d2_sorted, order = edge index)."""
    if n < 2:
        return 0
    k = ref["d2"].view(np.uint64)
    top = k >> np.uint64(48)
    packs = int(top.max() - top.min()) < 512 and len(np.unique(top)) <= 256
    ks = ref["d2_sorted"].view(np.uint64)
    e = ref["order"].astype(np.int64)
    g = ks >> np.uint64(22 if packs else 16)
    starts = np.flatnonzero(np.concatenate([[True], g[1:] != g[:-1]]))
    sizes = np.diff(np.append(starts, len(g)))
    for st, sz in zip(starts[sizes > 32], sizes[sizes > 32]):
        if packs and sz > 4096:
            return 2
        if np.any(np.diff(e[st:st + sz]) < 0):  # equal key >> shift out of edge order
            return 2
    return 1 if packs else 0


def run_and_check(x, tuning, want_form=None):
    from paper_2203_02527_gb300 import ph0
    ref = oracle.pipeline(x)
    got = ph0.barcodes(torch.from_numpy(np.ascontiguousarray(x)).cuda(), tuning=tuning)
    assert_bars_equal(got.numpy(), ref["bars"])
    assert got.stats["status"] == 0
    assert got.stats["n_distinct"] == ref["n_distinct"]
    assert got.inf == (ref["inf_vertex"], 0.0, float("inf"))
    form = expected_form(ref, len(x))
    assert got.stats["sort_form"] == form
    if want_form is not None:
        assert form == want_form
    return got, ref


@pytest.mark.parametrize("case", sorted(CASES))
def test_forced_packed_sort_matches_oracle(case):
    run_and_check(CASES[case](), PACKED)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 33, 91, 92, 129, 1000, 2897])
def test_forced_packed_small_and_ragged(n):
    # 91 points: 4095 edges, one short tile; 92: one full tile and a ragged one
    run_and_check(inputs.uniform(n, 3, seed=2100 + n), PACKED, want_form=1 if n > 1 else 0)


def test_keys_that_do_not_pack_take_the_short_sort():
    """Duplicated points: zero distances beside distances near 1, a top part
    spanning more than 512 values; the short sort runs in the same call."""
    run_and_check(inputs.with_duplicates(500, 3, 50, seed=2201), PACKED, want_form=0)


def test_long_groups_of_equal_distances_are_checked():
    """A 25 x 25 lattice: 259 groups of equal distances longer than 32
    records (up to 3144), each in edge order, hence sorted; the packed form
    stands.  A 40 x 40 lattice has a longer group: the complete sort."""
    run_and_check(inputs.lattice(25, 2), PACKED, want_form=1)
    run_and_check(inputs.lattice(40, 2), PACKED, want_form=2)


def test_crowded_groups_out_of_order_take_the_complete_sort():
    """Two clusters within 1e-12 of two points at distance 1: the cross
    distances form long groups of equal key >> 22 out of edge order."""
    rng = np.random.default_rng(43)
    a = rng.random((300, 3)) * 1e-12
    b = rng.random((300, 3)) * 1e-12
    b[:, 1] = 1.0
    x = np.ascontiguousarray(np.concatenate([a, b]), dtype=np.float32)
    run_and_check(x, PACKED, want_form=2)


def test_built_in_choice_with_groups_across_chunks():
    """4000 points on four noisy circles in dimension 16 (7,998,000 edges,
    above the built-in 2^22): the packed sort; its groups of equal key >> 22
    include some that reach across a 256-edge chunk (the second kernel)."""
    x = inputs.noisy_circles(1000, 4, 16, seed=2301)
    got, ref = run_and_check(x, None, want_form=1)
    g = ref["d2_sorted"].view(np.uint64) >> np.uint64(22)
    starts = np.flatnonzero(np.concatenate([[True], g[1:] != g[:-1]]))
    ends = np.append(starts[1:], len(g)) - 1
    multi = ends > starts
    crossing = (starts[multi] // 256) != (ends[multi] // 256)
    assert crossing.sum() > 0
    assert got.stats["sort_passes"] == 4


def test_packed_and_short_sorts_agree_and_profile():
    from paper_2203_02527_gb300 import ph0
    x = inputs.uniform(3000, 8, seed=2401)
    pts = torch.from_numpy(x).cuda()
    packed = ph0.barcodes(pts, tuning=PACKED)
    short = ph0.barcodes(pts, tuning={"packed_sort": 0})
    assert packed.stats["sort_form"] == 1 and short.stats["sort_form"] == 0
    assert_bars_equal(packed.numpy(), short.numpy())
    assert packed.stats["n_distinct"] == short.stats["n_distinct"]
    bars, prof = ph0.barcodes_profiled(pts, tuning=PACKED)
    assert_bars_equal(bars.numpy(), short.numpy())
    assert all(t > 0 for t in prof["pass_ms"][:4])
    assert all(t < 0.05 for t in prof["pass_ms"][4:])
