"""Parity of the CUDA path (through the C ABI) with the CPU oracle: every
step, element by element, bit-exact (integer, index and binary64 results are
all exact by construction, so the tolerance is zero)."""
import numpy as np
import pytest

import oracle
from paper_2203_02527_gb300 import inputs
from tests import golden, pins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ph0():
    from paper_2203_02527_gb300 import ph0
    return ph0


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def assert_bars_equal(got: np.ndarray, want: np.ndarray):
    assert len(got) == len(want)
    for f in ("u", "v", "a", "low", "order"):
        np.testing.assert_array_equal(got[f], want[f], err_msg=f)
    for f in ("death_sq", "death"):
        np.testing.assert_array_equal(got[f].view(np.uint64), want[f].view(np.uint64), err_msg=f)


CASES = {
    "uniform256": lambda: inputs.config_points("uniform256"),
    "uniform_ragged1000": lambda: inputs.uniform(1000, 3, seed=31),
    "mixture_ragged777_d8": lambda: inputs.gaussian_mixture(777, 8, k=5, sigma=0.2, seed=32),
    "circles_small_d16": lambda: inputs.noisy_circles(300, 4, 16, seed=33),
    "lattice_ties": lambda: inputs.lattice(12, 2),
    "lattice3d_ties": lambda: inputs.lattice(7, 3),
    "duplicates": lambda: inputs.with_duplicates(400, 3, 37, seed=34),
    "exponent_gaps": lambda: inputs.exponent_gaps(300, 5, seed=35),
    "negative_zero": lambda: inputs.negative_zero_mix(200, 3, seed=36),
    "simplex": lambda: np.eye(64, dtype=np.float32),
    "uniform_d1": lambda: inputs.uniform(500, 1, seed=37),
    "uniform_d33": lambda: inputs.uniform(300, 33, seed=38),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_steps_bit_exact(case):
    ph0 = _ph0()
    x = CASES[case]()
    n = len(x)
    ref = oracle.pipeline(x)
    pts = _cuda(x)
    # step 1
    key, val = ph0.distances(pts)
    np.testing.assert_array_equal(_u64(key), ref["d2"].view(np.uint64))
    want_val = (ref["u"].astype(np.uint32) << 16) | ref["v"].astype(np.uint32)
    np.testing.assert_array_equal(_u32(val), want_val)
    # step 2
    ph0.sort_pairs(key, val)
    np.testing.assert_array_equal(_u64(key), ref["d2_sorted"].view(np.uint64))
    want_sorted_val = (ref["u_sorted"].astype(np.uint32) << 16) | ref["v_sorted"].astype(np.uint32)
    np.testing.assert_array_equal(_u32(val), want_sorted_val)
    # step 3
    a, nd = ph0.dedupe(key)
    np.testing.assert_array_equal(_u32(a), ref["a"])
    assert nd == ref["n_distinct"]
    # steps 4-5
    bars = ph0.reduce(n, val, a, key)
    assert_bars_equal(bars.numpy(), ref["bars"])
    # the whole path in one call, with the bar that never dies
    whole = ph0.barcodes(pts)
    assert_bars_equal(whole.numpy(), ref["bars"])
    assert whole.stats["n_distinct"] == ref["n_distinct"]
    assert whole.stats["n_bars"] == n - 1
    assert whole.inf == (ref["inf_vertex"], 0.0, float("inf"))
    assert whole.stats["inf_vertex"] == ref["inf_vertex"]


@pytest.mark.parametrize("name", sorted(golden.FIXTURES))
def test_stored_bars(name):
    """The GPU paths against the stored barcodes (no oracle at test time)."""
    ph0 = _ph0()
    meta, lines = golden.stored(name)
    pts = _cuda(golden.points(name))
    whole = ph0.barcodes(pts)
    assert golden.bar_lines(whole.numpy()) == lines
    assert whole.stats["n_distinct"] == meta["distinct_distances"]
    assert golden.bar_lines(ph0.barcodes_early(pts, rounds=True).numpy()) == lines


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 31, 32, 33, 64, 65, 127, 129, 255, 257])
def test_small_and_ragged_sizes(n):
    ph0 = _ph0()
    x = inputs.uniform(n, 3, seed=100 + n)
    want, inf_v, nd = oracle.barcodes(x)
    got = ph0.barcodes(_cuda(x))
    assert_bars_equal(got.numpy(), want)
    assert inf_v == 0
    assert got.inf == (inf_v, 0.0, float("inf"))


def test_mixture4096_bit_exact():
    ph0 = _ph0()
    x = inputs.config_points("mixture4096")
    want, inf_v, nd = oracle.barcodes(x)
    got = ph0.barcodes(_cuda(x))
    assert_bars_equal(got.numpy(), want)
    assert got.stats["n_distinct"] == nd


def test_all_points_equal():
    ph0 = _ph0()
    x = np.full((50, 4), 0.25, np.float32)
    got = ph0.barcodes(_cuda(x)).numpy()
    assert (got["death_sq"] == 0).all() and (got["a"] == 1).all()
    assert [(int(b["u"]), int(b["v"])) for b in got] == [(0, j) for j in range(1, 50)]


def test_repeat_calls_identical_and_workspace_reuse():
    ph0 = _ph0()
    x = inputs.uniform(700, 4, seed=41)
    ws = ph0.Workspace(700, 4)
    first = ph0.barcodes(_cuda(x), ws=ws).numpy()
    y = inputs.uniform(300, 2, seed=42)
    other = ph0.barcodes(_cuda(y), ws=ws).numpy()
    again = ph0.barcodes(_cuda(x), ws=ws).numpy()
    assert_bars_equal(again, first)
    assert_bars_equal(other, oracle.barcodes(y)[0])


def test_nonfinite_input_reported():
    ph0 = _ph0()
    from paper_2203_02527_gb300._lib import Ph0Error
    x = inputs.uniform(40, 3, seed=43)
    x[7, 1] = np.nan
    with pytest.raises(Ph0Error) as e:
        ph0.barcodes(_cuda(x))
    assert e.value.code == 2
    x[7, 1] = np.inf
    with pytest.raises(Ph0Error) as e:
        ph0.barcodes(_cuda(x))
    assert e.value.code == 2
    # the context stays usable
    y = inputs.uniform(40, 3, seed=44)
    assert_bars_equal(ph0.barcodes(_cuda(y)).numpy(), oracle.barcodes(y)[0])


def test_invalid_arguments():
    import ctypes
    from paper_2203_02527_gb300 import _lib
    lib = _lib.load()
    assert lib.ph0_workspace_bytes(0, 3) == 0
    assert lib.ph0_workspace_bytes(131072, 3) == 0 and lib.ph0_workspace_bytes(131071, 3) > 0
    assert lib.ph0_workspace_bytes(10, 2000) == 0
    ws = torch.empty(lib.ph0_workspace_bytes(10, 3), dtype=torch.uint8, device="cuda")
    pts = torch.from_numpy(inputs.uniform(10, 3, seed=46)).cuda()
    bars = torch.empty((9, 40), dtype=torch.uint8, device="cuda")
    inf = torch.full((24,), 0xAB, dtype=torch.uint8, device="cuda")
    vp = ctypes.c_void_p
    args = (vp(pts.data_ptr()), 10, 3, 3, vp(bars.data_ptr()), vp(inf.data_ptr()), vp(ws.data_ptr()),
            ws.numel(), None)
    assert lib.ph0_barcodes(*args) == 0
    st = _lib.Stats()
    assert lib.ph0_finish(vp(ws.data_ptr()), None, ctypes.byref(st)) == 0
    # the bar that never dies, through the C ABI: vertex 0, birth 0, death +inf
    b = _lib.InfBar.from_buffer_copy(inf.cpu().numpy().tobytes())
    assert (b.vertex, b.birth, b.death) == (0, 0.0, float("inf")) and st.inf_vertex == 0
    assert lib.ph0_barcodes(*args[:5], None, *args[6:]) == 0                    # inf may be null
    assert lib.ph0_finish(vp(ws.data_ptr()), None, None) == 0
    assert lib.ph0_barcodes(args[0], 10, 3, 2, *args[4:]) == 1                  # ld < d
    assert lib.ph0_barcodes(args[0], 0, 3, 3, *args[4:]) == 1                   # n < 1
    assert lib.ph0_barcodes(args[0], 131072, 3, 3, *args[4:]) == 3              # n too big
    assert lib.ph0_barcodes(*args[:6], args[6], ws.numel() - 1, None) == 4     # small ws
    assert lib.ph0_barcodes(*args[:6], vp(ws.data_ptr() + 8), ws.numel(), None) == 1  # misaligned
    assert lib.ph0_barcodes(*args[:5], vp(inf.data_ptr() + 4), *args[6:]) == 1  # misaligned inf


def test_step_oracle_pins_hold_on_gpu_output():
    # the GPU result satisfies the oracle's independent pins directly
    ph0 = _ph0()
    x = inputs.uniform(60, 3, seed=45)
    got = ph0.barcodes(_cuda(x)).numpy()
    assert pins.check_bars_structure(60, got, 0) is None
    assert pins.check_bars_kruskal(x, got) is None
    assert pins.check_bars_sweep(x[:12], ph0.barcodes(_cuda(x[:12])).numpy()) is None


def test_short_sort_fixes_groups_in_place():
    """Simplex vertices (n=24) with off-diagonal perturbations of ~1e-10: the
    276 squared distances fall into 27 groups of equal key >> 16 holding up to
    25 records, 129 of them out of order; the fix-up sorts every group in
    place (no group is long enough for the complete sort)."""
    ph0 = _ph0()
    rng = np.random.default_rng(13)
    x = np.eye(24, dtype=np.float32)
    off = (rng.random((24, 24)) * 1e-10).astype(np.float32)
    np.fill_diagonal(off, 0)
    x = (x + off).astype(np.float32)
    ref = oracle.pipeline(x)
    keys = ref["d2"].view(np.uint64)
    groups, counts = np.unique(keys >> np.uint64(16), return_counts=True)
    assert 2 <= counts.max() <= 32 and len(groups) < len(keys) // 4
    assert_bars_equal(ph0.barcodes(_cuda(x)).numpy(), ref["bars"])


def test_crowded_distances_take_the_complete_sort():
    """Simplex vertices with off-diagonal perturbations of ~1e-12: all 190
    squared distances (189 distinct) lie within 2^-36 below 2, so the sort's
    passes over key bits 16 and up leave one long group out of order, and
    the fix-up hands over to the complete sort (the same bars)."""
    ph0 = _ph0()
    rng = np.random.default_rng(12)
    x = np.eye(20, dtype=np.float32)
    off = (rng.random((20, 20)) * 1e-12).astype(np.float32)
    np.fill_diagonal(off, 0)
    x = (x + off).astype(np.float32)
    assert np.all(np.diag(x) == 1)
    want = oracle.barcodes(x)[0]
    assert_bars_equal(ph0.barcodes(_cuda(x)).numpy(), want)
    d2 = want["death_sq"]
    assert d2.min() < 2 and d2.max() - d2.min() < 2.0 ** -36
    # the early path's class sort falls back the same way
    assert_bars_equal(ph0.barcodes_early(_cuda(x), rounds=True).numpy(), want)
    # and the plain step sequence agrees
    ref = oracle.pipeline(x)
    key, val = ph0.distances(_cuda(x))
    ph0.sort_pairs(key, val)
    np.testing.assert_array_equal(_u64(key), ref["d2_sorted"].view(np.uint64))


def test_distances_within_a_few_units_in_the_last_place():
    """Simplex vertices with off-diagonal perturbations of ~1e-14: all 190
    squared distances lie within 2^8 units in the last place of each other
    (only the lowest key byte varies), so the plan has no more than the two
    low passes that the short sort skips; the records stay where the
    distance kernel wrote them and the fix-up sorts them (or hands over to
    the complete sort)."""
    ph0 = _ph0()
    rng = np.random.default_rng(5)
    x = (np.eye(20) + rng.random((20, 20)) * 1e-14).astype(np.float32)
    np.fill_diagonal(x, 1.0)
    ref = oracle.pipeline(x)
    keys = ref["d2"].view(np.uint64)
    assert 0 < int(keys.min() ^ keys.max()).bit_length() <= 8
    assert_bars_equal(ph0.barcodes(_cuda(x)).numpy(), ref["bars"])
    assert_bars_equal(ph0.barcodes_early(_cuda(x), rounds=True).numpy(), ref["bars"])
    key, val = ph0.distances(_cuda(x))
    ph0.sort_pairs(key, val)
    np.testing.assert_array_equal(_u64(key), ref["d2_sorted"].view(np.uint64))


def test_crowded_cross_distances_take_the_complete_sort_on_many_tiles():
    """Two clusters of 1500 points each, every coordinate within 1e-12 of 0
    except the second cluster's y = 1: all 2.25M cross distances lie within
    ~2e-12 of 1, one long group of equal key >> 16 out of order, so the
    fix-up hands over to the complete sort, whose radix passes (the
    persistent instance, on fewer CTAs than the 1099 tiles) do real work."""
    ph0 = _ph0()
    rng = np.random.default_rng(41)
    a = rng.random((1500, 3)) * 1e-12
    b = rng.random((1500, 3)) * 1e-12
    b[:, 1] = 1.0
    x = np.concatenate([a, b]).astype(np.float32)
    ref = oracle.pipeline(x)
    keys = ref["d2"].view(np.uint64)  # in (u, v) order
    cross = keys.reshape(-1)[(ref["u"] < 1500) & (ref["v"] >= 1500)]
    assert len(np.unique(cross >> np.uint64(16))) <= 2 and np.any(np.diff(cross.astype(np.int64)) < 0)
    assert_bars_equal(ph0.barcodes(_cuda(x)).numpy(), ref["bars"])
    # the early path sorts the crowded class the same way (its own fallback)
    early = ph0.barcodes_early(_cuda(x), rounds=True)
    assert_bars_equal(early.numpy(), ref["bars"])


def test_two_top_passes_on_many_tiles():
    """Uniform points with two duplicated pairs: the zero distance makes the
    key range's top part span more than 9 bits, so the sort takes two top
    passes (the second in the persistent instance on the whole path) over
    4.5M edges (1099 tiles)."""
    ph0 = _ph0()
    x = inputs.uniform(3000, 3, seed=42)
    x[17] = x[2999]
    x[5] = x[1234]
    ref = oracle.pipeline(x)
    keys = ref["d2"].view(np.uint64)
    assert int(keys.max() >> np.uint64(48)) - int(keys.min() >> np.uint64(48)) >= 512
    assert_bars_equal(ph0.barcodes(_cuda(x)).numpy(), ref["bars"])
    key, val = ph0.distances(_cuda(x))
    ph0.sort_pairs(key, val)
    np.testing.assert_array_equal(_u64(key), ref["d2_sorted"].view(np.uint64))


@pytest.mark.parametrize("split,tile,top", [(0, 128, 9), (5, 64, 9), (16, 32, 8), (11, 128, 8)])
def test_tuning_changes_no_bit(split, tile, top):
    """Every tuning (distance split, tile size, top radix width) gives the
    oracle's bars; clouds with zero distances make the key range span more
    than 9 top bits (two top passes)."""
    ph0 = _ph0()
    t = {"dist_split16": split, "dist_tile": tile, "sort_top_bits": top}
    for x in (inputs.noisy_circles(150, 4, 8, seed=91), inputs.with_duplicates(500, 3, 300, seed=92),
              inputs.exponent_gaps(200, 4, seed=93)):
        got = ph0.barcodes(_cuda(x), tuning=t).numpy()
        assert_bars_equal(got, oracle.barcodes(x)[0])


def test_autotuner_picks_valid_settings(tmp_path, monkeypatch):
    monkeypatch.setenv("PH0_TUNING_CACHE", str(tmp_path / "tuning.json"))
    from paper_2203_02527_gb300 import autotune
    monkeypatch.setattr(autotune, "_cache", None)
    t = autotune.tune(3, n=1024, repeats=1)
    assert t["dist_split16"] in (0, 4, 8, 12, 16)
    assert t["dist_tile"] in (64, 128) and t["sort_top_bits"] in (8, 9)
    assert "packed_sort" not in t  # below 2^22 edges the packed sort is not a candidate
    assert autotune.cached(3, 1024) == t
    # from 2^22 edges the whole path is timed with both sorts
    t = autotune.tune(16, n=4096, repeats=1)
    assert t["packed_sort"] in (0, 1)
    assert autotune.cached(16, 4096) == t
