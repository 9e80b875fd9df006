"""The seeded synthetic inputs follow their stated recipes (CPU).

The generators hold none of the method's arithmetic; these checks pin the
shapes, sizes and value distributions the workloads are described with:
the jittered grid with dropped cells, the cluster/uniform mixture, the gaps
of the large uniform set, the theta designs, and the covariance of the
circulant-embedding GP draws.
"""
import math

import numpy as np
import pytest

from paper_1905_00141_gb300 import synth


def test_grid_recipe():
    """n = 131,072 jittered points, at most one per cell of a 382 x 382 grid,
    10% of the cells left empty or more, values of variance near
    sigma2 + tau2, the same draw for the same seed."""
    d = synth.grid()
    x, y, z = d["x"], d["y"], d["z"]
    G = 382
    assert len(x) == 131072 and (d["M"], d["J"], d["r"]) == (7, 4, 32)
    assert x.min() >= 0 and x.max() <= 1 and y.min() >= 0 and y.max() <= 1
    cells = np.floor(x * G).astype(np.int64) * G + np.floor(y * G).astype(np.int64)
    assert len(np.unique(cells)) == len(x)
    assert len(x) <= 0.9 * G * G
    assert 0.8 < np.var(z) < 1.25
    d2 = synth.grid()
    assert np.array_equal(d2["x"], x) and np.array_equal(d2["z"], z)


def test_clustered_recipe_scaled_down():
    """70% of the points in 8 tight clusters: on a 64 x 64 histogram, the
    densest cells hold far more than a uniform share."""
    d = synth.clustered(n=100000, grid_n=128)
    x, y = d["x"], d["y"]
    assert len(x) == 100000 and (d["M"], d["J"], d["r"]) == (9, 4, 32)
    assert d["theta"].shape == (64, 3)
    h, _, _ = np.histogram2d(x, y, bins=64)
    top = np.sort(h.ravel())[::-1]
    # 8 clusters of sd 0.03 cover ~ 8 * pi * (2 sd)^2 = 9% of the area with ~95% of 70% of the points
    assert top[: int(0.09 * h.size)].sum() > 0.6 * len(x)


def test_massive_recipe_scaled_down():
    """Uniform points with 200 empty discs covering 5% of the square: the
    share of empty cells on a fine grid is the gap fraction plus the Poisson
    share of a uniform set."""
    n = 400000
    d = synth.massive(n=n, grid_n=256)
    x, y = d["x"], d["y"]
    assert len(x) == n and (d["M"], d["J"], d["r"]) == (12, 4, 16)
    B = 200
    h, _, _ = np.histogram2d(x, y, bins=B, range=[[0, 1], [0, 1]])
    lam = n / (B * B) / 0.95
    expected = 0.05 + 0.95 * math.exp(-lam)
    empty = np.mean(h == 0)
    assert 0.5 * expected < empty < 1.6 * expected, (empty, expected)


def test_sparse_clusters_recipe():
    """n points in the unit square with its corners, all but the sprinkle
    within a few sd of k centres, a smooth field of variance near
    sigma2 + tau2; the same draw for the same seed."""
    x, y, z = synth.sparse_clusters(30000, 81, k=6, sd=0.006, sprinkle=200, grid_n=256)
    assert len(x) == len(y) == len(z) == 30000
    assert x.min() == 0.0 and y.min() == 0.0 and x.max() == 1.0 and y.max() == 1.0
    h, _, _ = np.histogram2d(x, y, bins=100, range=[[0, 1], [0, 1]])
    # 6 clusters of sd 0.006 fit in a few cells each of a 100 x 100 histogram
    assert np.sort(h.ravel())[::-1][:6 * 9].sum() > 0.9 * (30000 - 202)
    assert 0.2 < np.var(z) < 2.5
    x2, _, z2 = synth.sparse_clusters(30000, 81, k=6, sd=0.006, sprinkle=200, grid_n=256)
    assert np.array_equal(x2, x) and np.array_equal(z2, z)


def test_theta_designs():
    th = synth.theta_grid_4x4x4()
    assert th.shape == (64, 3)
    lo, hi = synth.THETA_BOX
    assert np.allclose(th.min(axis=0), lo) and np.allclose(th.max(axis=0), hi)
    s = synth.theta_sobol(2048)
    assert s.shape == (2048, 3)
    assert np.all(s >= lo) and np.all(s <= hi)
    u = (np.log(s) - np.log(lo)) / (np.log(hi) - np.log(lo))
    assert np.all(np.abs(u.mean(axis=0) - 0.5) < 0.02)
    assert np.array_equal(s, synth.theta_sobol(2048))


@pytest.mark.parametrize("beta", [0.05, 0.2])
def test_circulant_embedding_covariance(beta):
    """Empirical covariance of gp_grid draws against sigma2 exp(-d / beta)
    at a few lags (400 draws on a 24 x 24 grid)."""
    rng = np.random.default_rng(11)
    n, h, s2 = 24, 1.0 / 23, 1.3
    F = np.stack([synth.gp_grid(n, n, h, h, s2, beta, rng) for _ in range(400)])
    for lag in (0, 1, 3, 6):
        a = F[:, :n - lag, :].ravel()
        b = F[:, lag:, :].ravel()
        emp = np.mean(a * b)
        ref = s2 * math.exp(-lag * h / beta)
        assert abs(emp - ref) < 0.12 * s2, (lag, emp, ref)


def test_exact_gp_covariance():
    """gp_exact: the empirical covariance of repeated draws at three points."""
    rng = np.random.default_rng(12)
    x = np.array([0.1, 0.15, 0.6])
    y = np.array([0.2, 0.2, 0.7])
    Z = np.stack([synth.gp_exact(x, y, 1.0, 0.1, 0.05, rng) for _ in range(4000)])
    C = np.cov(Z.T)
    d = np.hypot(x[:, None] - x[None, :], y[:, None] - y[None, :])
    ref = np.exp(-d / 0.1) + 0.05 * np.eye(3)
    assert np.max(np.abs(C - ref)) < 0.08
