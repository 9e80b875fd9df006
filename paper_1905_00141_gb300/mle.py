"""Maximum-likelihood search over theta = (sigma2, beta, tau2) above the library.

The paper fits theta with a derivative-free optimiser that calls the exact
log-likelihood once per step ("likelihood" mode, Sec. 2.2.5).  Two searches
are provided, both maximising the exact MRA log-likelihood in the scaled
coordinates u = 2 (log theta - log lo) / (log hi - log lo) - 1 of a theta box:

* :func:`nelder_mead` -- the plain simplex method (Nelder & Mead 1965, with
  the standard coefficients 1, 2, 1/2, 1/2), one exact evaluation at a time.
* :func:`surrogate_search` -- the learned surrogate (``mlp.Surrogate``, the
  3 -> 64 -> 64 -> 1 network trained by the library's own kernels) is fitted
  to exact evaluations on a Sobol design, proposes where to look, and every
  proposal is scored by the exact likelihood in batches of 64 theta (one
  batched library call per round).  The exact values decide; the network
  only chooses the next batch.  If a round brings no improvement the search
  falls back to Nelder-Mead on the exact likelihood from the best point.

With ``use_network=False`` the same batched trust-region loop runs without
the network (each round is centred on the best exact point so far), which is
the method without the learned part.
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


def _cloud(center, radius, n, seed):
    """n Sobol points in the box |u - center| <= radius (sup norm), clipped to [-1, 1]^3."""
    return np.clip(np.asarray(center, float) + float(radius) * sobol_unit(n, seed), -1.0, 1.0)


def _top_distinct(u, v, k, min_dist):
    """Up to k points of u in decreasing order of v, each at least min_dist
    (sup norm) from those already taken."""
    order = np.argsort(-v)
    take = []
    for i in order:
        if not np.isfinite(v[i]):
            continue
        if all(np.max(np.abs(u[i] - u[j])) >= min_dist for j in take):
            take.append(i)
            if len(take) == k:
                break
    return u[take]


DEFAULT_SCHEDULE = ((2500, 3e-3), (2500, 1e-3), (2500, 3e-4), (2500, 1e-4))


def _fit(sur, th, y, schedule):
    sur.set_target_scaling(float(np.mean(y)), float(max(np.std(y), 1e-300)))
    for steps, lr in schedule:
        sur.train(th, y, steps, lr=lr)


class _Gap:
    """Monotone transform of loglik the network is fitted to:
    T(l) = -log(l_ref - l + c), c > 0 in nats.  It spreads the values near the
    best point l_ref over a wide range of T, so the fit's relative precision
    (bounded by the BF16 parameters) turns into a fine absolute precision of
    loglik near the maximum, where it matters; the argmax is unchanged."""

    def __init__(self, l_ref, c):
        self.l_ref, self.c = float(l_ref), float(c)

    def __call__(self, ll):
        return -np.log(self.l_ref - np.asarray(ll, float) + self.c)

    def inverse(self, t):
        return self.l_ref + self.c - np.exp(-np.asarray(t, float))


def surrogate_search(exact, new_surrogate=None, n_train=2048, batch=64, tol=0.5, seed=1909, max_rounds=10,
                     top_fraction=0.25, schedule=DEFAULT_SCHEDULE, radius0=0.2, shrink=0.25, cloud=16384,
                     gap_nats=0.0, use_network=True, nm_fallback_evals=200, log=None):
    """Batched trust-region search for the maximiser of the exact loglik.

    1. Exact loglik on n_train Sobol points of the box (batches of `batch`).
    2. A network over the whole box is fitted on the best `top_fraction` of
       them (full-batch Adam, `schedule` of (steps, rate)) to
       -log(l_best - loglik + gap_nats), a monotone transform of loglik that
       concentrates the fit's precision near the best value (gap_nats = 0:
       loglik/n itself).
    3. Each round proposes `batch` theta: the points of highest predicted
       loglik in a Sobol cloud of the trust region (sup-norm radius r around
       the incumbent, the best exact point), kept at least r/64 apart, and
       scores them exactly in one batched call.  If the incumbent moved by
       less than r/4 the region shrinks by `shrink` (otherwise it follows the
       incumbent at the same size), and a fresh network is fitted to the exact
       values inside the new region, with its inputs scaled to that region,
       for the next round.
    4. The loop ends when a round gains less than tol/4 without moving far
       (or once r <= 0.02).  A round with no gain at all hands over to
       Nelder-Mead on the exact loglik from the incumbent (the fallback).
    Without the network (use_network=False) each round scores a Sobol set of
    the trust region instead.  new_surrogate(box) -> ``mlp.Surrogate``.

    Returns a dict with the best theta and loglik, the exact evaluations of the
    design and of the search, and the rounds used."""
    if use_network and new_surrogate is None:
        from . import mlp

        def new_surrogate(b):
            return mlp.Surrogate(b, mlp.glorot_init(seed))

    box, n = exact.box, exact.n
    th_design = from_unit(sobol_unit(n_train, seed), box)
    for i in range(0, n_train, batch):
        exact(th_design[i:i + batch])
    evals_design = exact.evals
    radius = radius0
    sur, sur_box = None, None
    tf = None

    def targets(ll):
        return tf(ll) if tf is not None else np.asarray(ll, float) / n

    def predicted_ll(th):
        p = sur.predict(th)
        return tf.inverse(p) if tf is not None else p * n

    if use_network:
        th_all = np.array(exact.thetas)
        ll_all = np.array(exact.values)
        good = np.isfinite(ll_all)
        keep = good & (ll_all >= np.quantile(ll_all[good], 1.0 - top_fraction))
        tf = _Gap(exact.best, gap_nats) if gap_nats > 0 else None
        sur_box = box
        sur = new_surrogate(box)
        _fit(sur, th_all[keep], targets(ll_all[keep]), schedule)
    rounds = 0
    fell_back = False
    while rounds < max_rounds:
        rounds += 1
        center = to_unit(exact.best_theta, box)
        pts = _cloud(center, radius, cloud, seed + 100 + rounds)
        if use_network:
            pred = predicted_ll(from_unit(pts, box))
            cand = _top_distinct(pts, pred, batch, radius / 64.0)
        else:
            cand = np.vstack([center[None, :], pts[:batch - 1]])
        before = exact.best
        ll_c = exact(from_unit(cand, box))
        gain = exact.best - before
        moved = float(np.max(np.abs(to_unit(exact.best_theta, box) - center)))
        if log is not None:
            err = None
            if use_network:
                err = float(np.sqrt(np.mean((predicted_ll(from_unit(cand, box)) - ll_c) ** 2)))
            log.append(dict(round=rounds, radius=radius, best=float(exact.best), gain=float(gain), moved=moved,
                            pred_rmse_nats=err))
        if gain < 0.25 * tol and (moved < 0.25 * radius or radius <= 0.02):
            if gain <= 0.0 and radius > 0.01:
                exact_nelder_mead(exact, to_unit(exact.best_theta, box), step=radius, max_evals=nm_fallback_evals,
                                  ftol=0.1 * tol)
                fell_back = True
            break
        if moved < 0.25 * radius:
            radius = max(radius * shrink, 1e-3)  # the optimum is inside: zoom in
        if use_network:
            # fresh local network on the exact values inside the new region
            c = to_unit(exact.best_theta, box)
            lo_u, hi_u = np.clip(c - radius, -1, 1), np.clip(c + radius, -1, 1)
            u_all = to_unit(np.array(exact.thetas), box)
            ll_all = np.array(exact.values)
            inside = np.all((u_all >= lo_u - 1e-12) & (u_all <= hi_u + 1e-12), axis=1) & np.isfinite(ll_all)
            if inside.sum() >= 16:
                sur.close()
                sur_box = (from_unit(lo_u, box), from_unit(hi_u, box))
                sur = new_surrogate(sur_box)
                tf = _Gap(exact.best, gap_nats) if gap_nats > 0 else None
                _fit(sur, np.array(exact.thetas)[inside], targets(ll_all[inside]), schedule)
    if sur is not None:
        sur.close()
    return dict(theta=exact.best_theta, loglik=exact.best, evals_design=evals_design,
                evals_search=exact.evals - evals_design, rounds=rounds, fell_back=fell_back,
                calls=exact.calls)
