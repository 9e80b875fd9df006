"""Brute-force dense MRA covariance for tiny inputs (numpy, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

This module does not use the likelihood recursion at all.  It rebuilds the
partition of Sec. 1.2 with its own code, puts every observation and every knot
of levels 1..M-1 into one point set Z, and evaluates the remainder covariances
of Sec. 1.1 pair by pair:

    C_1 = C,
    C_{m+1}(a, b) = C_m(a, b) - C_m(a, Q) C_m(Q, Q)^{-1} C_m(Q, b)
                    if a and b lie in the same level-(m+1) region, else 0,

with Q the knots of the level-m region holding a and b.  The MRA process is
X = tau_1 + ... + tau_M with tau_m(s) = C_m(s, Q)' eta and
eta ~ N(0, C_m(Q, Q)^{-1}) independent over regions, so

    Sigma_MRA(a, b) = sum_{m<M} [a, b in one level-m region]
                          C_m(a, Q) C_m(Q, Q)^{-1} C_m(Q, b)
                      + [a, b in one leaf] C_M(a, b),

and the log-likelihood is log N(z; 0, Sigma_MRA + tau2 I), evaluated with a
numpy Cholesky.  Cost grows like |Z|^3 per level: use n of a few hundred.
"""
from __future__ import annotations

import math

import numpy as np


def grid_dims(r: int):
    """ceil(sqrt r) bars along x and floor(r / ceil(sqrt r)) along y (Sec. 1.2)."""
    nx = math.isqrt(r)
    if nx * nx < r:
        nx += 1
    return nx, r // nx


def knots_of(x0, x1, y0, y1, r, f):
    """App. A: bar p at x0 + L (f + p (1 - 2f) / (n - 1)); index q*nx + p."""
    nx, ny = grid_dims(r)
    kx, ky = [], []
    for q in range(ny):
        for p in range(nx):
            Lx = x1 - x0
            Ly = y1 - y0
            xs = x0 + Lx * (f + float(p) * (1.0 - 2.0 * f) / float(nx - 1)) if nx > 1 else x0 + 0.5 * Lx
            ys = y0 + Ly * (f + float(q) * (1.0 - 2.0 * f) / float(ny - 1)) if ny > 1 else y0 + 0.5 * Ly
            kx.append(xs)
            ky.append(ys)
    return np.array(kx), np.array(ky)


class Partition:
    """Regions of every level (list per level of (x0, x1, y0, y1)), knots of
    levels 1..M-1, and the kept observations (Sec. 1.2)."""

    def __init__(self, x, y, z, M, J, r, f=math.e / 100.0, dedup=False):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        z = np.asarray(z, dtype=np.float64)
        keep = ~np.isnan(z)
        if dedup:
            seen = set()
            for i in range(len(x)):
                if not keep[i]:
                    continue
                key = (float(x[i]), float(y[i]))
                if key in seen:
                    keep[i] = False
                else:
                    seen.add(key)
        xs, ys = x[keep], y[keep]
        xmin, xmax, ymin, ymax = xs.min(), xs.max(), ys.min(), ys.max()
        root = (xmin, xmax + 0.01 * (xmax - xmin), ymin, ymax + 0.01 * (ymax - ymin))
        self.M, self.J, self.r, self.f = M, J, r, f
        self.levels = [[root]]
        Lx, Ly = root[1] - root[0], root[3] - root[2]
        for m in range(1, M):
            nxt = []
            cut_x = Lx >= Ly
            for (x0, x1, y0, y1) in self.levels[-1]:
                mx, my = 0.5 * (x0 + x1), 0.5 * (y0 + y1)
                if J == 4:
                    nxt += [(x0, mx, y0, my), (mx, x1, y0, my), (x0, mx, my, y1), (mx, x1, my, y1)]
                elif cut_x:
                    nxt += [(x0, mx, y0, y1), (mx, x1, y0, y1)]
                else:
                    nxt += [(x0, x1, y0, my), (x0, x1, my, y1)]
            if J == 4:
                Lx, Ly = Lx / 2, Ly / 2
            elif cut_x:
                Lx = Lx / 2
            else:
                Ly = Ly / 2
            self.levels.append(nxt)
        self.knots = []  # per level m < M: list of (kx, ky)
        allk = set()
        for m in range(M - 1):
            lk = [knots_of(*b, r, f) for b in self.levels[m]]
            self.knots.append(lk)
            for kx, ky in lk:
                allk.update(zip(kx.tolist(), ky.tolist()))
        idx = np.nonzero(keep)[0]
        on_knot = np.array([(float(x[i]), float(y[i])) in allk for i in idx], dtype=bool)
        self.n_knot = int(on_knot.sum())
        idx = idx[~on_knot]
        self.index = idx
        self.x, self.y, self.z = x[idx], y[idx], z[idx]

    def region_of(self, px, py, m):
        """Index at level m (0-based list index) of the region holding each point."""
        out = np.full(len(px), -1, dtype=np.int64)
        for k, (x0, x1, y0, y1) in enumerate(self.levels[m]):
            inside = (px >= x0) & (px < x1) & (py >= y0) & (py < y1)
            out[inside] = k
        return out


def sigma_mra(part: Partition, sigma2: float, beta: float, return_all: bool = False, extra=None,
              first_level: int = 1):
    """Dense Sigma_MRA over the observations (and, with return_all, over the
    point set Z = observations + knots (+ the extra points, last), with the
    knot bookkeeping).  Extra points must lie inside the root region.

    first_level > 1 keeps only the terms of levels first_level..M: the
    covariance of the data given that the basis weights eta of the coarser
    levels are zero (Sec. 1.1: the levels' terms are independent and add up).
    The remainder recursion itself always runs from level 1."""
    M = part.M
    zx = [part.x]
    zy = [part.y]
    knot_ids = []  # per level m < M, per region: indices into Z
    base = len(part.x)
    for m in range(M - 1):
        ids = []
        for kx, ky in part.knots[m]:
            ids.append(np.arange(base, base + len(kx)))
            zx.append(kx)
            zy.append(ky)
            base += len(kx)
        knot_ids.append(ids)
    if extra is not None:
        zx.append(np.asarray(extra[0], dtype=np.float64))
        zy.append(np.asarray(extra[1], dtype=np.float64))
    X = np.concatenate(zx)
    Y = np.concatenate(zy)
    reg = [part.region_of(X, Y, m) for m in range(M)]
    D = np.sqrt((X[:, None] - X[None, :]) ** 2 + (Y[:, None] - Y[None, :]) ** 2)
    Cm = sigma2 * np.exp(-D / beta)
    Sig = np.zeros_like(Cm)
    for m in range(M - 1):
        proj = np.zeros_like(Cm)
        for k, q in enumerate(knot_ids[m]):
            members = np.nonzero(reg[m] == k)[0]
            if len(members) == 0:
                continue
            CaQ = Cm[np.ix_(members, q)]
            CQQ = Cm[np.ix_(q, q)]
            proj[np.ix_(members, members)] = CaQ @ np.linalg.solve(CQQ, CaQ.T)
        if m + 1 >= first_level:
            Sig += proj
        same_next = reg[m + 1][:, None] == reg[m + 1][None, :]
        Cm = np.where(same_next, Cm - proj, 0.0)
    same_leaf = reg[M - 1][:, None] == reg[M - 1][None, :]
    Sig += np.where(same_leaf, Cm, 0.0)
    n = len(part.x)
    if return_all:
        return Sig, dict(X=X, Y=Y, reg=reg, knot_ids=knot_ids, n_obs=n)
    return Sig[:n, :n]


def gauss_loglik(Sigma: np.ndarray, z: np.ndarray) -> float:
    """log N(z; 0, Sigma) by a Cholesky factor."""
    L = np.linalg.cholesky(Sigma)
    w = np.linalg.solve(L, z)
    return float(-0.5 * (2.0 * np.sum(np.log(np.diag(L))) + w @ w + len(z) * math.log(2.0 * math.pi)))


def loglik(x, y, z, M, J, r, theta, f=math.e / 100.0, dedup=False) -> float:
    sigma2, beta, tau2 = [float(v) for v in theta]
    part = Partition(x, y, z, M, J, r, f, dedup)
    S = sigma_mra(part, sigma2, beta)
    return gauss_loglik(S + tau2 * np.eye(len(part.z)), part.z)


def predict(x, y, z, M, J, r, theta, px, py, f=math.e / 100.0, dedup=False):
    """Kriging with Sigma_MRA (the plain definition of the MRA posterior
    predictive of the latent process, Sec. 1.1 model):
        mean = Sigma(P, S) (Sigma(S, S) + tau2 I)^{-1} z,
        var  = diag Sigma(P, P) - diag Sigma(P, S) (Sigma(S, S) + tau2 I)^{-1} Sigma(S, P).
    Points outside the root region give NaN."""
    sigma2, beta, tau2 = [float(v) for v in theta]
    part = Partition(x, y, z, M, J, r, f, dedup)
    px = np.asarray(px, dtype=np.float64)
    py = np.asarray(py, dtype=np.float64)
    x0, x1, y0, y1 = part.levels[0][0]
    inside = (px >= x0) & (px < x1) & (py >= y0) & (py < y1)
    mean = np.full(len(px), np.nan)
    var = np.full(len(px), np.nan)
    if not inside.any():
        return mean, var
    Sig, info = sigma_mra(part, sigma2, beta, return_all=True, extra=(px[inside], py[inside]))
    n = info["n_obs"]
    P = np.arange(len(Sig) - int(inside.sum()), len(Sig))
    K = Sig[:n, :n] + tau2 * np.eye(n)
    L = np.linalg.cholesky(K)
    A = np.linalg.solve(L, Sig[:n][:, P])          # L^{-1} Sigma(S, P)
    w = np.linalg.solve(L, part.z)                 # L^{-1} z
    mean[inside] = A.T @ w
    var[inside] = np.diag(Sig[np.ix_(P, P)]) - np.sum(A * A, axis=0)
    return mean, var
