"""Pins for the oracle's binary64 death gradient: the closed form of the loss
sum(death^2) (its derivative is 2 (x_u - x_v) per killing edge) and central
finite differences of the loss evaluated from scratch at perturbed points,
compared only where the pairing does not change within the step."""
import numpy as np
import pytest

import oracle
from paper_2203_02527_gb300 import inputs


def loss_f64(x64):
    _, _, _, d2 = oracle.barcodes_f64(x64)
    return float(d2.sum())  # sum of squared deaths


def test_gradient_closed_form_sum_of_squares():
    x = inputs.uniform(150, 3, seed=61)
    bars, _, _ = oracle.barcodes(x)
    g = oracle.death_gradient(x.astype(np.float64), bars["u"], bars["v"], 2.0 * bars["death"])
    want = np.zeros_like(g)
    x64 = x.astype(np.float64)
    for b in bars:
        diff = x64[b["u"]] - x64[b["v"]]
        want[b["u"]] += 2 * diff
        want[b["v"]] -= 2 * diff
    np.testing.assert_allclose(g, want, rtol=1e-12, atol=1e-12)


def test_gradient_against_central_differences():
    x = inputs.uniform(90, 3, seed=62).astype(np.float64)
    order0, u0, v0, _ = oracle.barcodes_f64(x)
    bars = oracle.barcodes(x.astype(np.float32))[0]
    g = oracle.death_gradient(x, bars["u"], bars["v"], 2.0 * bars["death"])
    h = 1e-4
    rng = np.random.default_rng(3)
    checked = 0
    for idx in rng.choice(x.size, 60, replace=False):
        i, k = divmod(int(idx), x.shape[1])
        xp, xm = x.copy(), x.copy()
        xp[i, k] += h
        xm[i, k] -= h
        sp, sm = oracle.barcodes_f64(xp), oracle.barcodes_f64(xm)
        same = all(np.array_equal(np.sort(s[1] * 65536 + s[2]), np.sort(u0 * 65536 + v0)) for s in (sp, sm))
        if not same:
            continue  # a tie within the step: the pairing changes
        fd = (sp[3].sum() - sm[3].sum()) / (2 * h)
        assert abs(fd - g[i, k]) <= 1e-6 * max(1.0, abs(fd)), (i, k, fd, g[i, k])
        checked += 1
    assert checked >= 40
