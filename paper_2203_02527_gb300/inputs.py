"""Seeded synthetic point clouds shared by the CUDA path's tests, the oracle's
tests and the benchmark.

This module holds only input generation (numpy PCG64 streams, drawn in fp64
and cast to fp32 so that every consumer sees the same bits).  It contains none
of the barcode method's arithmetic and imports neither the CUDA binding nor the
oracle.

The workloads stand in for the paper's experiments, which use uniformly random
points in the unit square (Sec. 3.1, Sec. 4); there is no public dataset.
"""
from __future__ import annotations

import math

import numpy as np

DEFAULT_SEED = 20260101


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform(n: int, d: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """n points i.i.d. uniform in [0,1)^d, fp32 [n, d] row-major."""
    return _rng(seed).random((n, d)).astype(np.float32)


def gaussian_mixture(n: int, d: int, k: int = 8, sigma: float = 0.05,
                     center_range: float = 10.0,
                     seed: int = DEFAULT_SEED) -> np.ndarray:
    """Mixture of k isotropic Gaussians with equal weights.

    Component of each point ~ integers(k); centres ~ U[0, center_range)^d;
    point = centre + N(0, sigma^2 I).
    """
    rng = _rng(seed)
    comp = rng.integers(k, size=n)
    centers = rng.random((k, d)) * center_range
    pts = centers[comp] + rng.standard_normal((n, d)) * sigma
    return pts.astype(np.float32)


def noisy_circles(n_per: int, n_circles: int, d: int, noise: float = 0.02,
                  center_range: float = 5.0,
                  seed: int = DEFAULT_SEED) -> np.ndarray:
    """n_circles unit circles, each in a random orthonormal 2-plane of R^d with
    centre ~ U[0, center_range)^d, n_per points each at angle ~ U[0, 2pi),
    plus N(0, noise^2 I) noise.  Circles are stored one after another.
    """
    rng = _rng(seed)
    out = []
    for _ in range(n_circles):
        q, _r = np.linalg.qr(rng.standard_normal((d, 2)))
        c = rng.random(d) * center_range
        theta = rng.random(n_per) * (2.0 * math.pi)
        ring = np.stack([np.cos(theta), np.sin(theta)], axis=1) @ q.T
        out.append(c + ring + rng.standard_normal((n_per, d)) * noise)
    return np.concatenate(out, axis=0).astype(np.float32)


def circles_with_outliers(n_per: int, n_circles: int, d: int, n_out: int,
                          far: float = 60.0, seed: int = DEFAULT_SEED) -> np.ndarray:
    """noisy_circles(n_per, n_circles, d) followed by n_out outliers at
    far * e_i (i = 0..n_out-1, n_out <= d): every edge from an outlier is
    longer than every edge among the circles, so the last edges to join a
    class come at the end of the edge order."""
    pts = noisy_circles(n_per, n_circles, d, seed=seed).astype(np.float64)
    out = np.zeros((n_out, d))
    out[np.arange(n_out), np.arange(n_out)] = far
    return np.concatenate([pts, out]).astype(np.float32)


# ---------------------------------------------------------------------------
# Named workloads (sizes and distributions of the benchmark configurations)
# ---------------------------------------------------------------------------

def config_points(name: str, seed: int = DEFAULT_SEED) -> np.ndarray:
    """The three single-cloud workloads.

    uniform256    N=256,   d=3,  U[0,1)^3                    (32,640 edges)
    mixture4096   N=4096,  d=3,  8 Gaussians, sigma=0.05      (~8.4M edges)
    circles32768  N=32768, d=16, 4 noisy unit circles         (~537M edges)
    """
    if name == "uniform256":
        return uniform(256, 3, seed)
    if name == "mixture4096":
        return gaussian_mixture(4096, 3, k=8, sigma=0.05, center_range=10.0,
                                seed=seed)
    if name == "circles32768":
        return noisy_circles(8192, 4, 16, noise=0.02, center_range=5.0,
                             seed=seed)
    raise KeyError(name)


def stream_clouds(count: int, seed: int = DEFAULT_SEED, n_min: int = 64,
                  n_max: int = 8192, dims=(2, 3, 8, 32)):
    """Serving workload: `count` clouds with N log-uniform in [n_min, n_max],
    d uniform in `dims`, Gaussian mixtures with k ~ U{1..16} and
    sigma ~ U[0.05, 0.5], centres ~ U[0,10)^d.  Returns a list of fp32 arrays.
    """
    rng = _rng(seed)
    clouds = []
    for _ in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        d = int(dims[rng.integers(len(dims))])
        k = int(rng.integers(1, 17))
        sigma = float(rng.uniform(0.05, 0.5))
        sub = int(rng.integers(2**31))
        clouds.append(gaussian_mixture(n, d, k=k, sigma=sigma,
                                       center_range=10.0, seed=sub))
    return clouds


def poisson_arrivals(count: int, rate_per_s: float,
                     seed: int = DEFAULT_SEED) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson stream: exponential gaps."""
    rng = _rng(seed ^ 0x5EED)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


# ---------------------------------------------------------------------------
# Adversarial and degenerate inputs
# ---------------------------------------------------------------------------

def lattice(k: int, d: int = 2, spacing: float = 1.0) -> np.ndarray:
    """k^d integer lattice points (many exactly equal distances)."""
    axes = [np.arange(k, dtype=np.float64) * spacing] * d
    grid = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, d)
    return grid.astype(np.float32)


def with_duplicates(n: int, d: int, n_unique: int,
                    seed: int = DEFAULT_SEED) -> np.ndarray:
    """n points drawn (with repetition) from n_unique distinct points, so
    that many squared distances are exactly +0."""
    rng = _rng(seed)
    base = rng.random((n_unique, d))
    return base[rng.integers(n_unique, size=n)].astype(np.float32)


def exponent_gaps(n: int, d: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """Coordinates spanning many binades (1e-30 .. 1e3), signed, with some
    exact zeros and negative zeros: fp32->fp64 differences that must round."""
    rng = _rng(seed)
    mag = 10.0 ** rng.uniform(-30, 3, size=(n, d))
    sign = np.where(rng.random((n, d)) < 0.5, -1.0, 1.0)
    pts = (mag * sign).astype(np.float32)
    z = rng.random((n, d))
    pts[z < 0.05] = np.float32(0.0)
    pts[(z >= 0.05) & (z < 0.1)] = np.float32(-0.0)
    return pts


def negative_zero_mix(n: int, d: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """Small integers with signed zeros: +0 and -0 must give identical keys."""
    rng = _rng(seed)
    pts = rng.integers(-3, 4, size=(n, d)).astype(np.float32)
    flip = rng.random((n, d)) < 0.5
    pts[(pts == 0) & flip] = np.float32(-0.0)
    return pts
