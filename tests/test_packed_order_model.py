"""Host model of the packed sort's ordering argument (the word layout of
csrc/ph0_common.cuh, kPackIdBits and pack_shift): words
    (number of key >> 48 among the values that occur) << 56
  | (key bits 22..47) << 30
  | (u << 15) | v
formed in edge order and sorted by four stable least-significant-digit
passes of 9, 9, 8 and 8 bits over word bits 30..63, then every group of
equal key >> 22 sorted stably by the whole key, give exactly the oracle's
order of the edges (Rawson, Sec. 2: the distances in increasing order,
ties in edge order).  numpy only; no GPU."""
import numpy as np
import pytest

import oracle
from paper_2203_02527_gb300 import inputs

DIGITS = [(30, 9), (39, 9), (48, 8), (56, 8)]


def packed_model_order(x):
    n = len(x)
    d2 = oracle.distances(x)
    k = d2.view(np.uint64)
    u, v = oracle.edge_endpoints(n)
    u = u.astype(np.uint64)
    v = v.astype(np.uint64)
    top = k >> np.uint64(48)
    occurring = np.unique(top)
    if len(occurring) > 256 or int(occurring[-1] - occurring[0]) >= 512:
        return None  # the keys do not pack: the short sort runs
    code = np.searchsorted(occurring, top).astype(np.uint64)
    w = (code << np.uint64(56)) | (((k >> np.uint64(22)) & np.uint64((1 << 26) - 1)) << np.uint64(30)) \
        | (u << np.uint64(15)) | v
    order = np.arange(len(w))
    for shift, bits in DIGITS:  # one stable pass per digit, lowest first
        digit = (w[order] >> np.uint64(shift)) & np.uint64((1 << bits) - 1)
        order = order[np.argsort(digit, kind="stable")]
    # the fix-up: each group of equal word >> 30 by the whole key, stably
    g = w[order] >> np.uint64(30)
    starts = np.flatnonzero(np.concatenate([[True], g[1:] != g[:-1]]))
    ends = np.append(starts[1:], len(g))
    for s, e in zip(starts, ends):
        if e - s > 1:
            seg = order[s:e]
            order[s:e] = seg[np.argsort(k[seg], kind="stable")]
    return order, w


@pytest.mark.parametrize("make", [
    lambda: inputs.uniform(300, 16, seed=3001),
    lambda: inputs.noisy_circles(100, 4, 16, seed=3002),
    lambda: inputs.gaussian_mixture(400, 8, k=5, sigma=0.2, seed=3003),
    lambda: inputs.lattice(12, 2),
    lambda: np.eye(40, dtype=np.float32),
])
def test_packed_order_equals_the_oracle_order(make):
    x = make()
    got = packed_model_order(x)
    assert got is not None
    order, w = got
    u, v = oracle.edge_endpoints(len(x))
    want = oracle.sort_edges(oracle.distances(x), u, v)
    np.testing.assert_array_equal(order, want)


def test_edge_field_orders_as_the_edge_index():
    # (u << 15) | v increases with the lexicographic edge index and fits 30 bits
    for n in (2, 3, 100, 200):
        uu, vv = oracle.edge_endpoints(n)
        f = (uu.astype(np.int64) << 15) | vv
        assert np.all(np.diff(f) > 0)
    assert (32766 << 15 | 32767) < (1 << 30)


def test_keys_that_do_not_pack_are_recognised():
    # duplicated points: zero distances beside distances near 1
    assert packed_model_order(inputs.with_duplicates(300, 3, 30, seed=3004)) is None
