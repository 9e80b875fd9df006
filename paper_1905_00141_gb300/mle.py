"""Maximum-likelihood search over theta = (sigma2, beta, tau2) above the library.

The paper fits theta with a derivative-free optimiser that calls the exact
log-likelihood once per step ("likelihood" mode, Sec. 2.2.5).  Two searches
are provided, both maximising the exact MRA log-likelihood in the scaled
coordinates u = 2 (log theta - log lo) / (log hi - log lo) - 1 of a theta box:

* :func:`nelder_mead` -- the plain simplex method (Nelder & Mead 1965, with
  the standard coefficients 1, 2, 1/2, 1/2), one exact evaluation at a time.
* :func:`guided_search` -- a batched trust-region search guided by models of
  the exact values seen so far: a weighted quadratic trend in u and the
  learned surrogate (``mlp.Surrogate``, the 3 -> 64 -> 64 -> 1 network trained
  by the library's own kernels) fitted to the trend's residuals.  Each round
  scores a small batch of proposals in one batched library call; the exact
  values decide, the models only choose the next batch, and the initial
  design counts in the budget.  With ``use_network=False`` the same loop runs
  on the trend alone (the method without the learned part).
"""
from __future__ import annotations

import math

import numpy as np


def to_unit(theta, box):
    lo, hi = np.log(np.asarray(box[0], float)), np.log(np.asarray(box[1], float))
    return 2.0 * (np.log(np.asarray(theta, float)) - lo) / (hi - lo) - 1.0


def from_unit(u, box):
    lo, hi = np.log(np.asarray(box[0], float)), np.log(np.asarray(box[1], float))
    return np.exp(lo + (np.asarray(u, float) + 1.0) * 0.5 * (hi - lo))


def sobol_unit(n, seed, d=3):
    """n scrambled Sobol points in [-1, 1]^d."""
    from scipy.stats import qmc
    m = max(0, math.ceil(math.log2(max(n, 1))))
    return 2.0 * qmc.Sobol(d=d, scramble=True, seed=seed).random_base2(m)[:n] - 1.0


class Exact:
    """Exact log-likelihood with an evaluation counter and a record of every
    (theta, loglik) it produced.  ``fn(theta[k][3]) -> loglik[k]`` is a batched
    evaluator (e.g. ``mra.MRA.loglik``); NaN (a failed factor) counts as -inf."""

    def __init__(self, fn, box, n_obs):
        self.fn = fn
        self.box = box
        self.n = n_obs
        self.evals = 0
        self.calls = 0
        self.thetas = []
        self.values = []
        self.trace = []  # (evals so far, best loglik so far)
        self.best = -math.inf
        self.best_theta = None

    def __call__(self, theta):
        th = np.atleast_2d(np.asarray(theta, dtype=np.float64))
        ll = np.asarray(self.fn(th), dtype=np.float64).reshape(-1)
        ll = np.where(np.isfinite(ll), ll, -np.inf)
        self.calls += 1
        for t, v in zip(th, ll):
            self.evals += 1
            self.thetas.append(t.copy())
            self.values.append(v)
            if v > self.best:
                self.best, self.best_theta = v, t.copy()
            self.trace.append((self.evals, self.best))
        return ll

    def evals_to_reach(self, target):
        """Evaluations until the best value first reached `target` (None if never)."""
        for k, b in self.trace:
            if b >= target:
                return k
        return None


def nelder_mead(f, x0, step=0.25, max_evals=400, xtol=1e-4, ftol=1e-3):
    """Minimise f from x0 with an initial simplex of edge `step` along each
    axis.  Stops when the simplex is smaller than xtol (sup norm) and its
    values differ by less than ftol, or after max_evals calls of f."""
    x0 = np.asarray(x0, dtype=np.float64)
    d = x0.size
    pts = [x0.copy()] + [x0 + step * np.eye(d)[i] for i in range(d)]
    vals = [f(p) for p in pts]
    ne = d + 1
    while ne < max_evals:
        order = np.argsort(vals)
        pts = [pts[i] for i in order]
        vals = [vals[i] for i in order]
        if max(np.max(np.abs(p - pts[0])) for p in pts[1:]) < xtol and vals[-1] - vals[0] < ftol:
            break
        c = np.mean(pts[:-1], axis=0)
        xr = c + (c - pts[-1])
        fr = f(xr)
        ne += 1
        if fr < vals[0]:
            xe = c + 2.0 * (c - pts[-1])
            fe = f(xe)
            ne += 1
            pts[-1], vals[-1] = (xe, fe) if fe < fr else (xr, fr)
        elif fr < vals[-2]:
            pts[-1], vals[-1] = xr, fr
        else:
            if fr < vals[-1]:
                xc = c + 0.5 * (xr - c)
            else:
                xc = c + 0.5 * (pts[-1] - c)
            fc = f(xc)
            ne += 1
            if fc < min(fr, vals[-1]):
                pts[-1], vals[-1] = xc, fc
            else:
                for i in range(1, d + 1):
                    pts[i] = pts[0] + 0.5 * (pts[i] - pts[0])
                    vals[i] = f(pts[i])
                    ne += 1
    i = int(np.argmin(vals))
    return pts[i], vals[i], ne


def exact_nelder_mead(exact, u0, step=0.25, max_evals=400, xtol=1e-4, ftol=1e-3):
    """Nelder-Mead on -loglik in scaled coordinates (outside the box: +inf)."""
    def f(u):
        if np.any(np.abs(u) > 1.0 + 1e-12):
            return math.inf
        return -float(exact(from_unit(u, exact.box)[None, :])[0])
    u, fu, ne = nelder_mead(f, u0, step=step, max_evals=max_evals, xtol=xtol, ftol=ftol)
    return u, -fu, ne


def _top_distinct(u, v, k, min_dist, taken=None):
    """Up to k points of u in decreasing order of v, each at least min_dist
    (sup norm) from those already taken (and from the rows of `taken`)."""
    order = np.argsort(-v)
    take = []
    prior = [] if taken is None else list(np.atleast_2d(taken))
    for i in order:
        if len(take) == k:
            break
        if not np.isfinite(v[i]):
            continue
        if all(np.max(np.abs(u[i] - u[j])) >= min_dist for j in take) and \
                all(np.max(np.abs(u[i] - p)) >= min_dist for p in prior):
            take.append(i)
    return u[take]


def _quad_features(u):
    """1, u_i, u_i^2 and u_i u_j (i < j) of points u [k][3]: 10 columns."""
    u = np.atleast_2d(u)
    a, b, c = u[:, 0], u[:, 1], u[:, 2]
    return np.stack([np.ones_like(a), a, b, c, a * a, b * b, c * c, a * b, a * c, b * c], axis=1)


def _fit_trend(u, ll, center, radius):
    """Weighted least-squares quadratic of loglik over scaled coordinates u
    (centred on the incumbent and divided by the trust radius).  Points are
    weighted by exp(-(l_best - l) / s), s the median gap of the points to the
    best, so the fit follows the top of the surface; the weights never fall
    below 1e-3."""
    z = (np.asarray(u, float) - center) / radius
    gap = np.max(ll) - ll
    s = max(float(np.median(gap)), 1.0)
    wt = np.maximum(np.exp(-gap / s), 1e-3)
    X = _quad_features(z) * np.sqrt(wt)[:, None]
    coef, *_ = np.linalg.lstsq(X, ll * np.sqrt(wt), rcond=None)
    return lambda uu: _quad_features((np.asarray(uu, float) - center) / radius) @ coef


def guided_search(exact, new_surrogate=None, n0=16, batch=6, seed=1909, max_evals=160, radius0=1.0,
                  shrink=0.5, min_local=24, cloud=8192, steps=(600, 600), rates=(3e-3, 5e-4), use_network=True,
                  net_share=0.5, log=None):
    """Batched model-based trust-region search for the maximiser of the exact
    loglik, with the design counted in the budget.

    Round 0 scores n0 scrambled-Sobol theta of the box (one batched call).
    Every round then:
      1. takes the exact points near the incumbent (sup-norm distance <= 1.5 r
         in scaled coordinates, at least the min_local nearest);
      2. fits a quadratic trend of loglik to them (weighted least squares, the
         weights favouring the top of the surface: the log-likelihood of a
         smooth covariance model is close to quadratic in log theta near its
         maximum) and, with use_network, the 3 -> 64 -> 64 -> 1 network to the
         trend's residuals (input scaling: the trust region; a few hundred Adam
         steps of the library's own kernels);
      3. scores in one batched exact call `batch` points of a Sobol cloud of
         the trust region (sup-norm radius r around the incumbent), at least
         r/16 apart: a share net_share of them of highest trend + network
         prediction, the rest of highest trend prediction (the network's
         proposals are a hedge: fitted to a few dozen points it can place
         spurious maxima, and the trend alone keeps the search moving);
      4. recentres on the best exact point and halves r (shrink) when it moved
         by less than r/4.
    The exact values decide; the models only choose the next batch.  Stops
    after max_evals exact evaluations or once r < 1e-3.  Returns the best theta
    and loglik, the evaluations and the rounds."""
    if use_network and new_surrogate is None:
        from . import mlp

        def new_surrogate(b):
            return mlp.Surrogate(b, mlp.glorot_init(seed))

    box = exact.box
    exact(from_unit(sobol_unit(n0, seed), box))
    radius = float(radius0)
    rounds = 0
    while exact.evals + batch <= max_evals and radius >= 1e-3:
        rounds += 1
        center = to_unit(exact.best_theta, box)
        u_all = to_unit(np.array(exact.thetas), box)
        ll_all = np.array(exact.values)
        ok = np.isfinite(ll_all)
        dist = np.max(np.abs(u_all - center), axis=1)
        near = ok & (dist <= 1.5 * radius)
        if near.sum() < min_local:
            order = np.argsort(np.where(ok, dist, np.inf))
            near = np.zeros_like(ok)
            near[order[:min(min_local, int(ok.sum()))]] = True
        u_loc, ll_loc = u_all[near], ll_all[near]
        trend = _fit_trend(u_loc, ll_loc, center, radius)
        lo_u, hi_u = np.clip(center - radius, -1, 1), np.clip(center + radius, -1, 1)
        pts = np.clip(center + radius * sobol_unit(cloud, seed + 100 + rounds), -1, 1)
        pred_t = trend(pts)
        k_net = int(round(net_share * batch)) if use_network else 0
        cand = _top_distinct(pts, pred_t, batch - k_net, radius / 16.0)
        if k_net > 0:
            res = ll_loc - trend(u_loc)
            scale = max(float(np.std(res)), 1e-3)
            sur = new_surrogate((from_unit(lo_u, box), from_unit(hi_u, box)))
            try:
                sur.set_target_scaling(0.0, scale)
                th_loc = from_unit(u_loc, box)
                for st, lr in zip(steps, rates):
                    sur.train(th_loc, res, st, lr=lr)
                pred_n = pred_t + sur.predict(from_unit(pts, box))
            finally:
                sur.close()
            cand = np.vstack([cand, _top_distinct(pts, pred_n, k_net, radius / 16.0, taken=cand)])
        before = exact.best
        exact(from_unit(cand, box))
        moved = float(np.max(np.abs(to_unit(exact.best_theta, box) - center)))
        if log is not None:
            log.append(dict(round=rounds, radius=radius, best=float(exact.best), gain=float(exact.best - before),
                            moved=moved, local=int(near.sum())))
        if moved < 0.25 * radius:
            radius *= shrink
    return dict(theta=exact.best_theta, loglik=exact.best, evals=exact.evals, rounds=rounds)
