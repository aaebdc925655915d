"""Full-size checks in the launch configuration the benchmark times (the
32768-point, d=16 circles cloud: 536,854,528 edges) and at the largest
cloud of the 16-bit record form (N = 65535).  Every bar is compared field by
field with the oracle's filtration-prefix path (oracle.barcodes_below: the
paper's steps on the edges up to the largest death, which gives the same
positions in the whole sorted order and the same indices a; on the
benchmark cloud that is 167,668,042 of the 536,854,528 edges, a few minutes
of host time).  Sampled outputs are also recomputed by the oracle one edge
at a time, and the rest is checked through properties that hold at any
size --
  * the bars are a spanning tree built in filtration order (Sec. 1: an edge
    ends a class exactly when it joins two disconnected subgraphs), and each
    bar's pivot row is the larger of the two component minima;
  * every non-tree edge sampled closes a cycle whose tree edges all come
    earlier in the total order (cycle property: the tree is the minimum one);
  * orders are increasing and a (the index in D) is non-decreasing, equal
    exactly when the squared distances are equal.
"""
import numpy as np
import pytest

import oracle
from paper_2203_02527_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def edge_d2(x, u, v):
    """binary64 squared distances of the given edges, from the oracle."""
    out = np.empty(len(u))
    for i, (a, b) in enumerate(zip(u, v)):
        out[i] = oracle.distances(np.stack([x[a], x[b]]))[0]
    return out


def tree_checks(x, bars, rng, samples=400):
    n = len(x)
    assert len(bars) == n - 1
    order = bars["order"].astype(np.int64)
    assert np.all(np.diff(order) > 0)
    a = bars["a"].astype(np.int64)
    dsq = bars["death_sq"]
    assert np.all(np.diff(a) >= 0) and np.all(np.diff(dsq) >= 0)
    assert np.array_equal(np.diff(a) == 0, np.diff(dsq) == 0)
    assert np.array_equal(bars["death"].view(np.uint64), np.sqrt(dsq).view(np.uint64))
    # spanning tree in filtration order; pivot = max of the component minima
    parent = np.arange(n)

    def find(i):
        while parent[i] != i:
            parent[i] = parent[parent[i]]
            i = parent[i]
        return i

    lows = set()
    for b in bars:
        ru, rv = find(int(b["u"])), find(int(b["v"]))
        assert ru != rv, "a bar closes a cycle"
        lo, hi = min(ru, rv), max(ru, rv)
        assert int(b["low"]) == hi
        lows.add(hi)
        parent[hi] = lo
    assert len(lows) == n - 1 and 0 not in lows
    # sampled deaths against the oracle, edge by edge
    pick = rng.choice(n - 1, min(samples, n - 1), replace=False)
    want = edge_d2(x, bars["u"][pick], bars["v"][pick])
    assert np.array_equal(want.view(np.uint64), dsq[pick].view(np.uint64))
    # cycle property on sampled non-tree edges, by binary lifting over the tree
    adj = [[] for _ in range(n)]
    for i, b in enumerate(bars):
        adj[int(b["u"])].append((int(b["v"]), i))
        adj[int(b["v"])].append((int(b["u"]), i))
    up = np.zeros(n, np.int64)
    upe = np.full(n, -1, np.int64)  # tree edge (bar index) to the parent
    depth = np.zeros(n, np.int64)
    seen = np.zeros(n, bool)
    stack = [0]
    seen[0] = True
    while stack:
        w = stack.pop()
        for y, e in adj[w]:
            if not seen[y]:
                seen[y] = True
                up[y], upe[y], depth[y] = w, e, depth[w] + 1
                stack.append(y)
    assert seen.all()
    levels = int(np.ceil(np.log2(n))) + 1
    anc = [up]
    mx = [upe]  # largest bar index (= latest in filtration order) on the jump
    for _ in range(1, levels):
        prev_a, prev_m = anc[-1], mx[-1]
        anc.append(prev_a[prev_a])
        mx.append(np.maximum(prev_m, prev_m[prev_a]))
    tree = set(zip(bars["u"].tolist(), bars["v"].tolist()))
    checked = 0
    while checked < samples:
        u, v = sorted(rng.choice(n, 2, replace=False).tolist())
        if (u, v) in tree:
            continue
        # latest tree edge on the path u..v
        best = -1
        a_, b_ = u, v
        if depth[a_] < depth[b_]:
            a_, b_ = b_, a_
        diff = depth[a_] - depth[b_]
        for k in range(levels):
            if diff >> k & 1:
                best = max(best, mx[k][a_])
                a_ = anc[k][a_]
        if a_ != b_:
            for k in range(levels - 1, -1, -1):
                if anc[k][a_] != anc[k][b_]:
                    best = max(best, mx[k][a_], mx[k][b_])
                    a_, b_ = anc[k][a_], anc[k][b_]
            best = max(best, mx[0][a_], mx[0][b_])
        d_uv = edge_d2(x, [u], [v])[0]
        t = bars[best]
        # the non-tree edge comes after every tree edge on its cycle: (d2, u, v)
        assert (t["death_sq"], int(t["u"]), int(t["v"])) < (d_uv, u, v)
        checked += 1


def assert_bars_equal(got, want):
    assert len(got) == len(want)
    for f in ("u", "v", "a", "low", "order"):
        np.testing.assert_array_equal(got[f], want[f], err_msg=f)
    for f in ("death_sq", "death"):
        np.testing.assert_array_equal(got[f].view(np.uint64), want[f].view(np.uint64), err_msg=f)


def test_benchmark_cloud_full_size():
    from paper_2203_02527_gb300 import ph0
    x = inputs.config_points("circles32768")
    pts = torch.from_numpy(x).cuda()
    ws = ph0.Workspace(len(x), x.shape[1])
    got = ph0.barcodes(pts, ws=ws)
    bars = got.numpy()
    assert got.stats["n_bars"] == 32767 and got.stats["status"] == 0
    assert got.inf == (0, 0.0, float("inf"))
    early = ph0.barcodes_early(pts, ws=ws).numpy()
    want, kept, _ = oracle.barcodes_below(x, float(bars["death_sq"].max()))
    assert len(want) == 32767 and kept == int(want["order"][-1]) + 1
    assert_bars_equal(bars, want)
    assert_bars_equal(early, want)
    tree_checks(x, bars, np.random.default_rng(1), samples=100)
    del ws, got
    torch.cuda.empty_cache()


def test_largest_supported_cloud():
    from paper_2203_02527_gb300 import ph0
    x = inputs.uniform(65535, 2, seed=3)
    ws = ph0.Workspace(65535, 2)
    got = ph0.barcodes(torch.from_numpy(x).cuda(), ws=ws)
    bars = got.numpy()
    assert got.stats["n_bars"] == 65534 and got.stats["status"] == 0
    want, _, _ = oracle.barcodes_below(x, float(bars["death_sq"].max()))
    assert_bars_equal(bars, want)
    tree_checks(x, bars, np.random.default_rng(2), samples=100)
    del ws, got
    torch.cuda.empty_cache()
