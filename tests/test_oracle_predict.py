"""Pins of the prediction oracle (dense kriging with Sigma_MRA, oracle/dense.py)
to things other than itself.

* The Gaussian conditional density: adding the point as an observation of
  value t changes the recursion oracle's log-likelihood (mra_oracle.c, pinned
  in test_oracle.py) by log N(t; mean, var + tau2), so three likelihood
  differences determine mean and var (oracle.predict_by_loglik).  The two
  routes share no code.
* Interpolation: with a tiny nugget the prediction at an observed location
  returns the observation with a vanishing variance.
* Bounds: 0 <= var <= sigma2 (conditioning cannot raise the variance).
* Outside the domain: NaN.
"""
import numpy as np
import pytest

import oracle
from oracle import dense


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _data(n, seed):
    rng = np.random.default_rng(seed)
    return rng.random(n), rng.random(n), rng.standard_normal(n), rng


@pytest.mark.parametrize("M,J,r", [(1, 4, 9), (3, 4, 9), (4, 2, 6), (2, 4, 16)])
def test_dense_prediction_equals_likelihood_differences(M, J, r):
    x, y, z, rng = _data(260, 31 + M)
    th = [1.4, 0.12, 0.04]
    px, py = rng.uniform(0.05, 0.95, 4), rng.uniform(0.05, 0.95, 4)
    mean, var = dense.predict(x, y, z, M, J, r, th, px, py)
    for k in range(4):
        m2, v2 = oracle.predict_by_loglik(x, y, z, M, J, r, th, px[k], py[k])
        assert abs(mean[k] - m2) <= 1e-9 * (1 + abs(m2))
        assert abs(var[k] - v2) <= 1e-9


def test_interpolation_at_observations():
    x, y, z, _ = _data(150, 41)
    th = [1.0, 0.2, 1e-9]
    mean, var = dense.predict(x, y, z, 3, 4, 9, th, x[:10], y[:10])
    assert np.max(np.abs(mean - z[:10])) < 1e-5
    assert np.max(np.abs(var)) < 1e-6


def test_variance_bounds_and_outside_points():
    x, y, z, rng = _data(200, 42)
    th = [2.0, 0.1, 0.05]
    px = np.concatenate([rng.uniform(0, 1, 30), [1.5, -0.2]])
    py = np.concatenate([rng.uniform(0, 1, 30), [0.5, 0.5]])
    mean, var = dense.predict(x, y, z, 3, 4, 9, th, px, py)
    assert np.all(np.isnan(mean[-2:])) and np.all(np.isnan(var[-2:]))
    v = var[:-2][~np.isnan(var[:-2])]
    assert np.all(v >= -1e-12) and np.all(v <= th[0] + 1e-12)


def test_likelihood_difference_route_detects_a_wrong_mean():
    """The identity is sharp: shifting the dense mean by 1e-6 breaks it."""
    x, y, z, rng = _data(200, 43)
    th = [1.0, 0.1, 0.05]
    px, py = np.array([0.4]), np.array([0.6])
    mean, var = dense.predict(x, y, z, 2, 4, 9, th, px, py)
    m2, v2 = oracle.predict_by_loglik(x, y, z, 2, 4, 9, th, px[0], py[0])
    assert abs(mean[0] - m2) < 1e-10
    assert abs(mean[0] + 1e-6 - m2) > 5e-7


PREDICT_MUTATIONS = {
    "no_nugget": ("K = Sig[:n, :n] + tau2 * np.eye(n)", "K = Sig[:n, :n] + 0.5 * tau2 * np.eye(n)"),
    "mean_without_solve": ("mean[inside] = A.T @ w", "mean[inside] = A.T @ part.z"),
    "variance_sign": ("- np.sum(A * A, axis=0)", "+ np.sum(A * A, axis=0)"),
    "nugget_in_variance": ("var[inside] = np.diag(Sig[np.ix_(P, P)])",
                           "var[inside] = tau2 + np.diag(Sig[np.ix_(P, P)])"),
    "prior_instead_of_mra": ("Sig, info = sigma_mra(part, sigma2, beta, return_all=True, extra=(px[inside], py[inside]))",
                             "Sig, info = sigma_mra(part, sigma2, beta, return_all=True, extra=(px[inside], py[inside]))\n"
                             "    Sig = sigma2 * np.exp(-np.hypot(info['X'][:, None] - info['X'][None, :], "
                             "info['Y'][:, None] - info['Y'][None, :]) / beta)"),
}


@pytest.mark.parametrize("name", sorted(PREDICT_MUTATIONS))
def test_prediction_pin_catches_mutation(name):
    """Each plausible mistake planted in a private copy of dense.predict
    breaks the likelihood-difference pin."""
    import inspect
    src = inspect.getsource(dense.predict)
    old, new = PREDICT_MUTATIONS[name]
    assert src.count(old) == 1
    ns = dict(vars(dense))
    exec(src.replace(old, new), ns)
    bad = ns["predict"]
    x, y, z, rng = _data(220, 51)
    th = [1.2, 0.1, 0.05]
    px, py = np.array([0.37, 0.71]), np.array([0.52, 0.26])
    m, v = bad(x, y, z, 3, 4, 9, th, px, py)
    ref = [oracle.predict_by_loglik(x, y, z, 3, 4, 9, th, a, b) for a, b in zip(px, py)]
    err = max(max(abs(m[k] - ref[k][0]), abs(v[k] - ref[k][1])) for k in range(2))
    assert err > 1e-6, (name, err)
