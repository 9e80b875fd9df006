"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the tests, the benchmark and the oracle checks.  It
draws locations and values only; it holds none of the MRA arithmetic (no
partition, no remainder covariance, no likelihood).  Values z are draws of a
zero-mean Gaussian process with the exponential covariance
sigma2 * exp(-d / beta) plus a N(0, tau2) nugget, made either exactly (dense
Cholesky, small n) or by circulant embedding on a regular grid (large n).

Workloads (sizes follow the configurations the library is measured on):

* ``small``    n=4,096 i.i.d. uniform on [0,1]^2, exact GP (sigma2=1, beta=0.1,
               tau2=0.05); tree M=3, J=4, r=16.
* ``grid``     n=131,072 on a jittered 382x382 grid with 10% of the cells
               dropped at random and a random trim to exactly n; GP by
               circulant embedding on the grid (sigma2=1, beta=0.05,
               tau2=0.01), values carried to the jittered points; M=7, J=4,
               r=32 (30 knots per region).  Stand-in for the paper's small
               MODIS scene (a gridded satellite field with missing cells).
* ``clustered`` n=2,097,152: 70% in 8 Gaussian clusters (sd 0.03, centres
               uniform), 30% uniform; GP by circulant embedding on a 1024^2 grid
               over the bounding box, nearest-cell value; M=9, J=4, r=32; a
               4x4x4 log-spaced theta grid.  Stand-in for the skewed leaf
               counts of the AMSR data.
* ``massive``  n=47,185,920 uniform on [0,1]^2 minus 200 random discs (5% of
               the area); GP by circulant embedding on a 4096^2 grid
               (sigma2=1, beta=0.02, tau2=0.01); M=12, J=4, r=16.  Stand-in
               for the large MODIS scene (gaps where clouds mask pixels).
* ``swaths``   n=2,439,827 uniform on [0,1]^2 inside parallel slanted bands
               (a band of width 0.1 every 0.125 across the direction
               (1, 0.35): 80% coverage, straight gaps between passes); GP by
               circulant embedding on a 2048^2 grid (sigma2=1, beta=0.05,
               tau2=0.01); M=14, J=2, r=49.  Stand-in for the AMSR scene of
               the paper (satellite passes with gaps, its r = 49 binary tree).
* ``modis18``  n=4,194,304 by the swaths recipe (another seed) on the tree
               of the paper's large MODIS run: M=18, J=2, r=49 (35 device
               levels, 131,071 regions).  Its number of points is a tenth
               of that scene's: one GPU holds this tree's prior and leaf
               basis, the upward pass streams subtrees.
"""
from __future__ import annotations

import math

import numpy as np

WORKLOADS = {
    "small": dict(n=4096, M=3, J=4, r=16, theta=(1.0, 0.1, 0.05)),
    "grid": dict(n=131072, M=7, J=4, r=32, theta=(1.0, 0.05, 0.01)),
    "clustered": dict(n=2097152, M=9, J=4, r=32, theta=(1.0, 0.05, 0.01)),
    "massive": dict(n=47185920, M=12, J=4, r=16, theta=(1.0, 0.02, 0.01)),
    "swaths": dict(n=2439827, M=14, J=2, r=49, theta=(1.0, 0.05, 0.01)),
    "modis18": dict(n=4194304, M=18, J=2, r=49, theta=(1.0, 0.05, 0.01)),
}

SEED_BASE = 1905


def _exp_cov(d, sigma2, beta):
    return sigma2 * np.exp(-d / beta)


def gp_exact(x, y, sigma2, beta, tau2, rng):
    """Exact zero-mean GP draw at (x, y) by a dense Cholesky, plus nugget."""
    d = np.sqrt((x[:, None] - x[None, :]) ** 2 + (y[:, None] - y[None, :]) ** 2)
    C = _exp_cov(d, sigma2, beta)
    C[np.diag_indices_from(C)] += 1e-10
    L = np.linalg.cholesky(C)
    return L @ rng.standard_normal(len(x)) + math.sqrt(tau2) * rng.standard_normal(len(x))


def gp_grid(nx, ny, hx, hy, sigma2, beta, rng):
    """GP on an nx x ny grid of spacing (hx, hy) by circulant embedding on the
    2nx x 2ny torus; negative eigenvalues (if any) are clipped to zero."""
    Nx, Ny = 2 * nx, 2 * ny
    ix = np.arange(Nx)
    iy = np.arange(Ny)
    dx = np.minimum(ix, Nx - ix) * hx
    dy = np.minimum(iy, Ny - iy) * hy
    d = np.sqrt(dx[:, None] ** 2 + dy[None, :] ** 2)
    c = _exp_cov(d, sigma2, beta)
    lam = np.fft.fft2(c).real
    lam = np.maximum(lam, 0.0)
    w = rng.standard_normal((Nx, Ny)) + 1j * rng.standard_normal((Nx, Ny))
    f = np.fft.fft2(np.sqrt(lam / (Nx * Ny)) * w)
    return f.real[:nx, :ny]


def small(seed: int = SEED_BASE + 1, n: int = 4096):
    rng = np.random.default_rng(seed)
    x = rng.random(n)
    y = rng.random(n)
    s2, b, t2 = WORKLOADS["small"]["theta"]
    z = gp_exact(x, y, s2, b, t2, rng)
    return dict(x=x, y=y, z=z, M=3, J=4, r=16, theta=np.array([[s2, b, t2]]))


def grid(seed: int = SEED_BASE + 2, n: int = 131072):
    rng = np.random.default_rng(seed)
    G = int(math.ceil(math.sqrt(n / 0.9)))
    h = 1.0 / G
    s2, b, t2 = WORKLOADS["grid"]["theta"]
    field = gp_grid(G, G, h, h, s2, b, rng)
    cells = np.arange(G * G)
    kept = rng.permutation(cells)[: int(round(0.9 * G * G))]
    if len(kept) < n:
        raise ValueError("grid too small for n")
    kept = np.sort(rng.permutation(kept)[:n])
    i, j = kept // G, kept % G
    x = (i + 0.5 + rng.uniform(-0.5, 0.5, n)) * h
    y = (j + 0.5 + rng.uniform(-0.5, 0.5, n)) * h
    z = field[i, j] + math.sqrt(t2) * rng.standard_normal(n)
    return dict(x=x, y=y, z=z, M=7, J=4, r=32, theta=np.array([[s2, b, t2]]))


def theta_grid_4x4x4():
    """64 theta on a log-spaced 4x4x4 grid: sigma2 in [0.5, 2], beta in
    [0.02, 0.2], tau2 in [0.005, 0.05]."""
    s = np.geomspace(0.5, 2.0, 4)
    b = np.geomspace(0.02, 0.2, 4)
    t = np.geomspace(0.005, 0.05, 4)
    S, B, T = np.meshgrid(s, b, t, indexing="ij")
    return np.stack([S.ravel(), B.ravel(), T.ravel()], axis=1)


# theta box of the surrogate and of the batched workload: sigma2, beta, tau2
THETA_BOX = (np.array([0.5, 0.02, 0.005]), np.array([2.0, 0.2, 0.05]))


def theta_sobol(n: int, seed: int = SEED_BASE + 4, box=THETA_BOX):
    """n theta log-uniform over the box from a scrambled Sobol sequence."""
    from scipy.stats import qmc
    u = qmc.Sobol(d=3, scramble=True, seed=seed).random_base2(max(0, math.ceil(math.log2(max(n, 1)))))[:n]
    lo, hi = np.log(box[0]), np.log(box[1])
    return np.exp(lo + u * (hi - lo))


def mlp_init(seed: int = SEED_BASE + 5, hidden: int = 64):
    """Initial FP32 parameters of the 3 -> hidden -> hidden -> 1 network
    (W1, b1, W2, b2, w3, b3 flattened in that order): weights uniform in
    +-sqrt(6 / (fan_in + fan_out)) (Glorot), biases zero."""
    rng = np.random.default_rng(seed)

    def glorot(fo, fi):
        a = math.sqrt(6.0 / (fi + fo))
        return rng.uniform(-a, a, size=(fo, fi))

    parts = [glorot(hidden, 3), np.zeros(hidden), glorot(hidden, hidden), np.zeros(hidden), glorot(1, hidden),
             np.zeros(1)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def clustered(seed: int = SEED_BASE + 3, n: int = 2097152, grid_n: int = 1024):
    rng = np.random.default_rng(seed)
    nc = int(round(0.7 * n))
    centres = rng.random((8, 2))
    lab = rng.integers(0, 8, nc)
    pc = centres[lab] + 0.03 * rng.standard_normal((nc, 2))
    pu = rng.random((n - nc, 2))
    p = np.concatenate([pc, pu])
    p = p[rng.permutation(n)]
    x, y = p[:, 0].copy(), p[:, 1].copy()
    s2, b, t2 = WORKLOADS["clustered"]["theta"]
    x0, x1, y0, y1 = x.min(), x.max(), y.min(), y.max()
    hx = (x1 - x0) / (grid_n - 1)
    hy = (y1 - y0) / (grid_n - 1)
    field = gp_grid(grid_n, grid_n, hx, hy, s2, b, rng)
    ix = np.clip(np.rint((x - x0) / hx).astype(np.int64), 0, grid_n - 1)
    iy = np.clip(np.rint((y - y0) / hy).astype(np.int64), 0, grid_n - 1)
    z = field[ix, iy] + math.sqrt(t2) * rng.standard_normal(n)
    return dict(x=x, y=y, z=z, M=9, J=4, r=32, theta=theta_grid_4x4x4())


def massive(seed: int = SEED_BASE + 6, n: int = 47185920, grid_n: int = 4096, n_discs: int = 200,
            gap_fraction: float = 0.05):
    """n points uniform on [0,1]^2 minus n_discs random discs (gaps) whose
    radius is set so their areas add up to gap_fraction of the square (an
    oversample is drawn and trimmed to n); z from an exponential GP
    (sigma2=1, beta=0.02, tau2=0.01) by circulant embedding on a grid_n^2
    grid, nearest-cell value plus the nugget; M=12, J=4, r=16."""
    rng = np.random.default_rng(seed)
    rad = math.sqrt(gap_fraction / (n_discs * math.pi))
    centres = rng.random((n_discs, 2))
    m = int(n / (1.0 - gap_fraction) * 1.03) + 1024
    x = rng.random(m)
    y = rng.random(m)
    order = np.argsort(x, kind="stable")
    x, y = x[order], y[order]
    keep = np.ones(m, dtype=bool)
    for cx, cy in centres:
        a, b = np.searchsorted(x, [cx - rad, cx + rad])
        keep[a:b] &= (x[a:b] - cx) ** 2 + (y[a:b] - cy) ** 2 > rad * rad
    idx = np.flatnonzero(keep)
    if len(idx) < n:
        raise ValueError("oversample too small")
    idx = np.sort(rng.permutation(idx)[:n])
    x, y = x[idx], y[idx]
    perm = rng.permutation(n)
    x, y = x[perm], y[perm]
    s2, b, t2 = WORKLOADS["massive"]["theta"]
    h = 1.0 / (grid_n - 1)
    field = gp_grid(grid_n, grid_n, h, h, s2, b, rng)
    ix = np.clip(np.rint(x / h).astype(np.int64), 0, grid_n - 1)
    iy = np.clip(np.rint(y / h).astype(np.int64), 0, grid_n - 1)
    z = field[ix, iy] + math.sqrt(t2) * rng.standard_normal(n)
    return dict(x=x, y=y, z=z, M=12, J=4, r=16, theta=np.array([[s2, b, t2]]))


def swaths(seed: int = SEED_BASE + 7, n: int = 2439827, grid_n: int = 2048, period: float = 0.125,
           width: float = 0.1, slant: float = 0.35):
    """n points uniform on [0,1]^2 kept where frac((x + slant y) / period) <
    width / period (parallel slanted bands, the rest a gap), an oversample
    trimmed to n; z from an exponential GP (sigma2=1, beta=0.05, tau2=0.01)
    by circulant embedding on a grid_n^2 grid, nearest-cell value plus the
    nugget; M=14, J=2, r=49."""
    rng = np.random.default_rng(seed)
    cover = width / period
    m = int(n / cover * 1.05) + 1024
    x = rng.random(m)
    y = rng.random(m)
    keep = np.mod((x + slant * y) / period, 1.0) < cover
    idx = np.flatnonzero(keep)
    if len(idx) < n:
        raise ValueError("oversample too small")
    idx = np.sort(rng.permutation(idx)[:n])
    x, y = x[idx], y[idx]
    perm = rng.permutation(n)
    x, y = x[perm], y[perm]
    s2, b, t2 = WORKLOADS["swaths"]["theta"]
    h = 1.0 / (grid_n - 1)
    field = gp_grid(grid_n, grid_n, h, h, s2, b, rng)
    ix = np.clip(np.rint(x / h).astype(np.int64), 0, grid_n - 1)
    iy = np.clip(np.rint(y / h).astype(np.int64), 0, grid_n - 1)
    z = field[ix, iy] + math.sqrt(t2) * rng.standard_normal(n)
    w = WORKLOADS["swaths"]
    return dict(x=x, y=y, z=z, M=w["M"], J=w["J"], r=w["r"], theta=np.array([[s2, b, t2]]))


def modis18(seed: int = SEED_BASE + 8, n: int = 4194304, grid_n: int = 2048):
    """The swaths recipe (slanted passes with gaps, a GP field) at n points on
    the tree shape of the paper's large MODIS run: J=2, M=18, r=49 (131,072
    finest regions, about 32 points each)."""
    d = swaths(seed=seed, n=n, grid_n=grid_n)
    w = WORKLOADS["modis18"]
    d.update(M=w["M"], J=w["J"], r=w["r"])
    return d


def sparse_clusters(n: int, seed: int, k: int = 6, sd: float = 0.015, sprinkle: int = 200, grid_n: int = 1024,
                    sigma2: float = 1.0, beta: float = 0.05, tau2: float = 0.01):
    """n points: k isotropic Gaussian clusters (sd, centres uniform on
    [0.1, 0.9]^2) holding n - sprinkle - 2 points, `sprinkle` uniform points,
    and the corners (0, 0) and (1, 1), which fix the domain to the unit
    square; z from an exponential GP (sigma2, beta) by circulant embedding on
    a grid_n^2 grid, nearest-cell value plus a N(0, tau2) nugget.  On a deep
    tree most subtrees stay empty, which a reference that skips empty
    subtrees evaluates quickly; the device path runs every region all the
    same."""
    rng = np.random.default_rng(seed)
    nc = n - sprinkle - 2
    c = 0.1 + 0.8 * rng.random((k, 2))
    lab = rng.integers(0, k, nc)
    x = np.concatenate([c[lab, 0] + sd * rng.standard_normal(nc), rng.random(sprinkle), [0.0, 1.0]])
    y = np.concatenate([c[lab, 1] + sd * rng.standard_normal(nc), rng.random(sprinkle), [0.0, 1.0]])
    x = np.clip(x, 0.0, 1.0)
    y = np.clip(y, 0.0, 1.0)
    h = 1.0 / (grid_n - 1)
    field = gp_grid(grid_n, grid_n, h, h, sigma2, beta, rng)
    ix = np.clip(np.rint(x / h).astype(np.int64), 0, grid_n - 1)
    iy = np.clip(np.rint(y / h).astype(np.int64), 0, grid_n - 1)
    return x, y, field[ix, iy] + math.sqrt(tau2) * rng.standard_normal(n)


def uniform(n: int, seed: int, sigma2=1.0, beta=0.1, tau2=0.05, exact=True):
    """Small uniform draw for tests (exact GP values when exact=True)."""
    rng = np.random.default_rng(seed)
    x = rng.random(n)
    y = rng.random(n)
    if exact and n <= 6000:
        z = gp_exact(x, y, sigma2, beta, tau2, rng)
    else:
        z = rng.standard_normal(n)
    return x, y, z


def make(name: str, **kw):
    return {"small": small, "grid": grid, "clustered": clustered, "massive": massive, "swaths": swaths,
            "modis18": modis18}[name](**kw)
