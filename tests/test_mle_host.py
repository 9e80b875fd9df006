"""Host logic of the maximum-likelihood search (no GPU): the simplex method,
the evaluation counter, the scaled coordinates, and the batched
trust-region loop without the network on a cheap smooth objective."""
import math

import numpy as np

from paper_1905_00141_gb300 import mle, synth

BOX = synth.THETA_BOX


def test_unit_coordinates_round_trip():
    th = synth.theta_sobol(100, seed=3)
    u = mle.to_unit(th, BOX)
    assert np.all(np.abs(u) <= 1.0)
    assert np.allclose(mle.from_unit(u, BOX), th, rtol=1e-13)
    assert np.allclose(mle.to_unit(np.array(BOX[0]), BOX), -1.0)
    assert np.allclose(mle.to_unit(np.array(BOX[1]), BOX), 1.0)


def test_nelder_mead_quadratic_and_rosenbrock():
    A = np.array([[3.0, 1.0, 0.0], [1.0, 2.0, 0.5], [0.0, 0.5, 1.0]])
    x_star = np.array([0.3, -0.2, 0.5])
    x, f, ne = mle.nelder_mead(lambda x: (x - x_star) @ A @ (x - x_star) + 7.0, np.zeros(3), step=0.25,
                               max_evals=2000, xtol=1e-8, ftol=1e-12)
    assert np.max(np.abs(x - x_star)) < 1e-5 and abs(f - 7.0) < 1e-9 and ne < 2000

    def rosen(x):
        return 100.0 * (x[1] - x[0] ** 2) ** 2 + (1.0 - x[0]) ** 2
    x, f, ne = mle.nelder_mead(rosen, np.array([-1.2, 1.0]), step=0.5, max_evals=5000, xtol=1e-9, ftol=1e-14)
    assert np.max(np.abs(x - 1.0)) < 1e-4


def test_exact_counter_and_trace():
    calls = []

    def fn(th):
        calls.append(len(th))
        return -np.sum(np.log(th) ** 2, axis=1)

    ex = mle.Exact(fn, BOX, 10)
    ex(np.array([[1.0, 0.1, 0.01], [0.5, 0.05, 0.02]]))
    ex(np.array([1.0, 0.05, 0.01]))
    assert ex.evals == 3 and ex.calls == 2 and calls == [2, 1]
    assert ex.best == max(ex.values)
    assert [k for k, _ in ex.trace] == [1, 2, 3]
    assert ex.evals_to_reach(ex.best) == 1 + int(np.argmax(ex.values))
    assert ex.evals_to_reach(ex.best + 1.0) is None


def test_nan_counts_as_minus_infinity():
    ex = mle.Exact(lambda th: np.full(len(th), np.nan), BOX, 1)
    v = ex(np.array([[1.0, 0.1, 0.01]]))
    assert v[0] == -math.inf and ex.best == -math.inf


def test_top_distinct_spacing():
    rng = np.random.default_rng(0)
    u = rng.uniform(-1, 1, (500, 3))
    v = -np.sum(u ** 2, axis=1)
    t = mle._top_distinct(u, v, 20, 0.1)
    assert len(t) == 20
    for i in range(20):
        for j in range(i):
            assert np.max(np.abs(t[i] - t[j])) >= 0.1
    assert np.allclose(t[0], u[np.argmax(v)])


def test_trust_region_without_network_finds_maximum():
    # a smooth, ridge-shaped stand-in for loglik over the box (maximum inside)
    u_star = np.array([0.35, 0.1, -0.4])

    def fn(th):
        u = mle.to_unit(th, BOX) - u_star
        ridge = (u[:, 0] - u[:, 1]) ** 2 * 400.0 + (u[:, 0] + u[:, 1]) ** 2 * 20.0 + u[:, 2] ** 2 * 200.0
        return -ridge
    ex = mle.Exact(fn, BOX, 1)
    log = []
    r = mle.guided_search(ex, use_network=False, n0=16, batch=6, max_evals=160, log=log)
    assert ex.best > -0.5 and r["evals"] == ex.evals <= 160
    assert ex.evals_to_reach(-0.5) <= 100
    # the design is one batched call, then every round one call of `batch` points
    assert ex.calls == 1 + len(log) and ex.evals == 16 + 6 * len(log)


def test_quadratic_trend_is_exact_on_a_quadratic():
    rng = np.random.default_rng(4)
    u = rng.uniform(-1, 1, (30, 3))
    A = np.array([[-3.0, 0.5, 0.2], [0.5, -2.0, 0.1], [0.2, 0.1, -1.0]])
    b = np.array([0.3, -0.2, 0.1])
    f = np.einsum("ij,jk,ik->i", u, A, u) + u @ b + 7.0
    trend = mle._fit_trend(u, f, np.array([0.1, 0.0, -0.1]), 0.5)
    v = rng.uniform(-1, 1, (50, 3))
    assert np.allclose(trend(v), np.einsum("ij,jk,ik->i", v, A, v) + v @ b + 7.0, atol=1e-9)
