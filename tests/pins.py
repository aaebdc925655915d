"""Independent checks ("pins") for the barcode path.

Each check is written from what the paper and the mathematics fix, not from
the oracle's code: exact integer arithmetic, an exact-rational replay of each
binary64 rounding, numpy's library sort and unique, union-find Kruskal, dense
Prim, brute-force connectivity sweeps, and closed forms.  The functions return
None when the check passes and a message string when it fails, so that tests
can also show that a planted mistake is caught.

Sec. 1: an edge joins two points once epsilon reaches their distance; an edge
removes a homology class exactly when it joins two disconnected subgraphs.
Sec. 2: barcodes are the intervals (0, b) read from the reduced matrix.
"""
from __future__ import annotations

from collections import deque
from fractions import Fraction

import numpy as np


# ---------------------------------------------------------------------------
# Step 1: distances
# ---------------------------------------------------------------------------

def rn64(q: Fraction) -> Fraction:
    """Round an exact rational to the nearest binary64 (ties to even).
    CPython's int/int true division is correctly rounded."""
    return Fraction(q.numerator / q.denominator) if q else Fraction(0)


def replay_d2(xu, xv) -> float:
    """The squared distance with one binary64 rounding after each subtraction,
    multiplication and addition, in dimension order, carried out in exact
    rational arithmetic with explicit rounding."""
    s = Fraction(0)
    for a, b in zip(xv, xu):
        t = rn64(Fraction(float(a)) - Fraction(float(b)))
        p = rn64(t * t)
        s = rn64(s + p)
    return float(s)


def check_d2_integer_exact(x: np.ndarray, d2: np.ndarray):
    """Integer coordinates: every rounding is exact, so d2 must equal the
    integer sum of squared differences."""
    xi = np.asarray(x, dtype=np.float64).astype(np.int64)
    if not np.array_equal(xi.astype(np.float64), np.asarray(x, np.float64)):
        return "coordinates are not integers"
    n = len(xi)
    iu, iv = np.triu_indices(n, 1)
    exact = ((xi[iv] - xi[iu]) ** 2).sum(axis=1)
    if not np.array_equal(exact.astype(np.float64), d2):
        bad = int(np.flatnonzero(exact.astype(np.float64) != d2)[0])
        return f"edge {bad}: {d2[bad]!r} != {int(exact[bad])}"
    return None


def check_d2_replay(x: np.ndarray, d2: np.ndarray):
    n = len(x)
    e = 0
    for i in range(n):
        for j in range(i + 1, n):
            want = replay_d2(x[i], x[j])
            if np.float64(want).view(np.uint64) != np.float64(d2[e]).view(np.uint64):
                return f"edge ({i},{j}): {d2[e]!r} != replay {want!r}"
            e += 1
    return None


def check_d2_error_bound(x: np.ndarray, d2: np.ndarray):
    """Relative error against the exact squared distance within the standard
    bound for d rounded products and sums (plus the rounded differences)."""
    n, d = x.shape
    u = 2.0 ** -53
    bound = (2 * d + 2) * u
    e = 0
    for i in range(n):
        for j in range(i + 1, n):
            exact = sum((Fraction(float(a)) - Fraction(float(b))) ** 2
                        for a, b in zip(x[j], x[i]))
            got = Fraction(float(d2[e]))
            if exact == 0:
                if got != 0:
                    return f"edge ({i},{j}) should be 0"
            elif abs(got - exact) / exact > bound:
                return f"edge ({i},{j}): relative error above {bound}"
            e += 1
    return None


def check_edge_enumeration(n: int, u: np.ndarray, v: np.ndarray):
    iu, iv = np.triu_indices(n, 1)
    if not (np.array_equal(u, iu) and np.array_equal(v, iv)):
        return "edge ids are not the lexicographic pairs u<v"
    return None


# ---------------------------------------------------------------------------
# Steps 2-3: sort and de-duplication
# ---------------------------------------------------------------------------

def check_sorted(d2, u, v, order):
    want = np.lexsort((v, u, d2))  # last key is primary
    if not np.array_equal(want, order):
        bad = int(np.flatnonzero(want != order)[0])
        return f"sorted position {bad}: {order[bad]} != {want[bad]}"
    return None


def check_dedupe(d2_sorted, a, n_distinct=None):
    uniq = np.unique(d2_sorted)
    want = np.searchsorted(uniq, d2_sorted) + 1
    if not np.array_equal(want, np.asarray(a, np.int64)):
        bad = int(np.flatnonzero(want != a)[0])
        return f"position {bad}: a={a[bad]} want {want[bad]}"
    if n_distinct is not None and n_distinct != len(uniq):
        return f"|D|={n_distinct} want {len(uniq)}"
    return None


# ---------------------------------------------------------------------------
# Steps 4-5: pairing
# ---------------------------------------------------------------------------

def numpy_d2(x: np.ndarray) -> np.ndarray:
    """Squared distances by numpy vector operations (one binary64 rounding
    per element-wise operation), in lexicographic edge order."""
    x64 = np.asarray(x, np.float64)
    n, d = x64.shape
    iu, iv = np.triu_indices(n, 1)
    s = np.zeros(len(iu))
    for k in range(d):
        t = x64[iv, k] - x64[iu, k]
        s = s + t * t
    return s


def kruskal(n: int, d2: np.ndarray):
    """Union-find Kruskal over the total order (d2, u, v) with the root of each
    component its smallest vertex.  Returns, in order, tuples
    (sorted position, u, v, d2, max(min A, min B))."""
    iu, iv = np.triu_indices(n, 1)
    order = np.lexsort((iv, iu, d2))
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    out = []
    for pos, e in enumerate(order):
        a, b = find(int(iu[e])), find(int(iv[e]))
        if a == b:
            continue
        lo, hi = (a, b) if a < b else (b, a)
        parent[hi] = lo
        out.append((pos, int(iu[e]), int(iv[e]), float(d2[e]), hi))
        if len(out) == n - 1:
            break
    return out


def prim_weights(d2_matrix: np.ndarray) -> np.ndarray:
    """Dense O(N^2) Prim: sorted MST edge weights (squared)."""
    n = len(d2_matrix)
    if n <= 1:
        return np.zeros(0)
    in_tree = np.zeros(n, bool)
    best = np.full(n, np.inf)
    best[0] = 0.0
    weights = []
    for _ in range(n):
        cand = np.where(in_tree, np.inf, best)
        j = int(np.argmin(cand))
        if in_tree.sum() > 0:
            weights.append(best[j])
        in_tree[j] = True
        best = np.minimum(best, d2_matrix[j])
    return np.sort(np.array(weights))


def d2_matrix(x: np.ndarray) -> np.ndarray:
    n = len(x)
    iu, iv = np.triu_indices(n, 1)
    m = np.zeros((n, n))
    s = numpy_d2(x)
    m[iu, iv] = s
    m[iv, iu] = s
    return m


def check_bars_structure(n: int, bars, inf_vertex):
    if len(bars) != max(n - 1, 0):
        return f"{len(bars)} finite bars, want {n - 1}"
    if inf_vertex != 0:
        return f"infinite bar at vertex {inf_vertex}, want 0"
    lows = np.asarray(bars["low"])
    if len(np.unique(lows)) != len(lows):
        return "pivot rows are not unique"
    if len(lows) and (lows.min() < 1 or lows.max() >= n):
        return "pivot row out of range"
    if np.any(np.diff(np.asarray(bars["order"])) <= 0):
        return "bars not in filtration order"
    if np.any(np.asarray(bars["u"]) >= np.asarray(bars["v"])):
        return "killing edge not u<v"
    return None


def check_bars_kruskal(x: np.ndarray, bars):
    n = len(x)
    ref = kruskal(n, numpy_d2(x))
    if len(ref) != len(bars):
        return f"{len(bars)} bars vs {len(ref)} Kruskal edges"
    for i, (pos, u, v, w, hi) in enumerate(ref):
        b = bars[i]
        if (int(b["order"]), int(b["u"]), int(b["v"])) != (pos, u, v):
            return f"bar {i}: edge {(int(b['order']), int(b['u']), int(b['v']))} != {(pos, u, v)}"
        if np.float64(b["death_sq"]).view(np.uint64) != np.float64(w).view(np.uint64):
            return f"bar {i}: death_sq {b['death_sq']!r} != {w!r}"
        if int(b["low"]) != hi:
            return f"bar {i}: pivot row {int(b['low'])} != max(min A, min B) = {hi}"
        if np.float64(b["death"]).view(np.uint64) != np.float64(np.sqrt(w)).view(np.uint64):
            return f"bar {i}: death is not sqrt(death_sq)"
    return None


def check_bars_prim(x: np.ndarray, bars):
    w = prim_weights(d2_matrix(x))
    got = np.sort(np.asarray(bars["death_sq"], np.float64))
    if not np.array_equal(w, got):
        return "death multiset differs from Prim's MST weights"
    return None


def check_bars_a(x: np.ndarray, bars):
    """a of every bar = 1-based rank of its squared distance among the distinct
    squared distances."""
    uniq = np.unique(numpy_d2(x))
    want = np.searchsorted(uniq, np.asarray(bars["death_sq"])) + 1
    if not np.array_equal(want, np.asarray(bars["a"], np.int64)):
        return "bar index a differs from rank in D"
    return None


def components(n: int, edges) -> int:
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    seen = [False] * n
    count = 0
    for s in range(n):
        if seen[s]:
            continue
        count += 1
        seen[s] = True
        q = deque([s])
        while q:
            a = q.popleft()
            for b in adj[a]:
                if not seen[b]:
                    seen[b] = True
                    q.append(b)
    return count


def check_bars_sweep(x: np.ndarray, bars):
    """For every epsilon in D (and below its minimum): the number of connected
    components of the graph with the edges of squared length <= epsilon equals
    1 + the number of finite bars still alive (death_sq > epsilon)."""
    n = len(x)
    d2 = numpy_d2(x)
    iu, iv = np.triu_indices(n, 1)
    deaths = np.asarray(bars["death_sq"], np.float64)
    levels = [-1.0] + list(np.unique(d2))
    for eps in levels:
        keep = d2 <= eps
        c = components(n, zip(iu[keep].tolist(), iv[keep].tolist()))
        alive = int((deaths > eps).sum())
        if c != 1 + alive:
            return f"eps={eps}: {c} components, {alive} bars alive"
    return None
