"""GPU prediction (mra_predict: posterior predictive mean and variance of the
latent process) against the oracle, through the C ABI.

References:
* small trees: dense kriging with Sigma_MRA (oracle/dense.py), the plain
  definition;
* the 131,072-point gridded workload: the recursion oracle's likelihood with
  the point added as an observation (oracle.predict_by_loglik), at sampled
  points.

Tolerances.  FP64 path: 1e-9 absolute on the mean and the variance (data and
sigma2 of order one; both sides are FP64 by different routes; measured
<= 4e-13).  Mixed path: the basis values, Y = L^{-1} U and the small leaves'
L^{-1} are stored in FP32 (unit roundoff u = 2^-24 = 6e-8).  The mean is a
sum of n_R + (M-1) r such products weighted by the solution of the leaf's
kriging system, whose condition number is up to (sigma2 + tau2) / tau2
(= 250 at theta = (2.5, 0.3, 0.01)); the rounding errors add up like
sqrt(n_R) (n_R <= 300 here): u * 250 * sqrt(300) = 2.6e-4 bounds the error,
and the tests use 1e-4 (measured at most 1.9e-5, in the 300-point cluster
at the long range and small nugget).
"""
import numpy as np
import pytest

import oracle
from oracle import dense
from paper_1905_00141_gb300 import build as mbuild
from paper_1905_00141_gb300 import mra, synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-9
TOLMIX = 1e-4
THETAS = [[1.0, 0.1, 0.05], [2.5, 0.3, 0.01]]


@pytest.fixture(scope="module", autouse=True)
def _built():
    mbuild.build()
    oracle.build()


def _points(rng, k, lo=0.02, hi=0.98):
    return rng.uniform(lo, hi, k), rng.uniform(lo, hi, k)


def _check(x, y, z, M, J, r, px, py, thetas=THETAS, precisions=("fp64", "mixed")):
    worst = {}
    with mra.MRA(x, y, z, M, J, r) as g:
        for th in thetas:
            ref_m, ref_v = dense.predict(x, y, z, M, J, r, th, px, py)
            for p in precisions:
                g.set_precision(p)
                m, v = g.predict(th, px, py)
                assert np.array_equal(np.isnan(m), np.isnan(ref_m)), p
                ok = ~np.isnan(ref_m)
                em = np.max(np.abs(m[ok] - ref_m[ok]))
                ev = np.max(np.abs(v[ok] - ref_v[ok]))
                tol = TOL64 if p == "fp64" else TOLMIX
                assert em <= tol and ev <= tol, (p, th, em, ev)
                worst[p] = max(worst.get(p, 0.0), em, ev)
    return worst


def test_predict_quadtree_small():
    """n = 1500, M = 3, J = 4, r = 16: mean and variance at 40 points, plus
    points on observations, in the top/right extension of the domain and
    outside it (NaN)."""
    x, y, z = synth.uniform(1500, 11)
    rng = np.random.default_rng(5)
    px, py = _points(rng, 40)
    px = np.concatenate([px, x[:3], [x.max() + 1e-4, 2.0, -1.0]])
    py = np.concatenate([py, y[:3], [0.5, 0.5, np.nan]])
    _check(x, y, z, 3, 4, 16, px, py)


def test_predict_binary_tree_deeper():
    """J = 2, M = 6, r = 9 (odd knot count, padding to 16)."""
    x, y, z = synth.uniform(900, 12)
    rng = np.random.default_rng(6)
    px, py = _points(rng, 30)
    _check(x, y, z, 6, 2, 9, px, py)


def test_predict_wide_regions_r49():
    """r = 49 (J = 2, M = 4; J = 4, M = 3): the kernels run each level's
    knots as two device levels; the predictive distribution is the paper's
    (dense kriging with all 49 knots of a region at once)."""
    rng = np.random.default_rng(8)
    for M, J, seed in [(4, 2, 13), (3, 4, 14)]:
        x, y, z = synth.uniform(1200, seed)
        px, py = _points(rng, 30)
        _check(x, y, z, M, J, 49, px, py)


def test_predict_empty_leaf_and_large_leaf():
    """A tight cluster makes a leaf of more than 64 observations (the tiled
    large-leaf path) and a hole leaves leaves empty; points land in both."""
    rng = np.random.default_rng(7)
    xc = 0.3 + 0.02 * rng.standard_normal(300)
    yc = 0.3 + 0.02 * rng.standard_normal(300)
    xu, yu = rng.random(500), rng.random(500)
    keep = ~((xu > 0.6) & (yu > 0.6))
    x = np.concatenate([xc, xu[keep]])
    y = np.concatenate([yc, yu[keep]])
    z = synth.gp_exact(x, y, 1.0, 0.1, 0.05, rng)
    px = np.concatenate([0.3 + 0.02 * rng.standard_normal(10), [0.8, 0.9, 0.75], rng.uniform(0.05, 0.95, 10)])
    py = np.concatenate([0.3 + 0.02 * rng.standard_normal(10), [0.8, 0.7, 0.95], rng.uniform(0.05, 0.55, 10)])
    with mra.MRA(x, y, z, 3, 4, 16) as g:
        assert g.stats()["max_leaf"] > 64
    _check(x, y, z, 3, 4, 16, px, py)


def test_predict_single_level():
    """M = 1: the prediction is plain kriging with the exponential covariance
    (one small leaf and one large one)."""
    for n, seed in ((50, 13), (200, 14)):
        x, y, z = synth.uniform(n, seed)
        rng = np.random.default_rng(seed)
        px, py = _points(rng, 12)
        _check(x, y, z, 1, 4, 16, px, py)


def test_predict_grid_workload_sampled():
    """The 131,072-point gridded workload (M = 7, J = 4, r = 32) at sampled
    points against the recursion oracle's likelihood differences."""
    d = synth.grid()
    rng = np.random.default_rng(8)
    x, y = d["x"], d["y"]
    px = rng.uniform(x.min() + 0.05, x.max() - 0.05, 4)
    py = rng.uniform(y.min() + 0.05, y.max() - 0.05, 4)
    th = [1.0, 0.05, 0.01]
    ref = np.array([oracle.predict_by_loglik(x, y, d["z"], d["M"], d["J"], d["r"], th, a, b)
                    for a, b in zip(px, py)])
    with mra.MRA(x, y, d["z"], d["M"], d["J"], d["r"]) as g:
        for p in ("fp64", "mixed"):
            g.set_precision(p)
            m, v = g.predict(th, px, py)
            tol = 1e-8 if p == "fp64" else TOLMIX
            assert np.max(np.abs(m - ref[:, 0])) <= tol, (p, m, ref[:, 0])
            assert np.max(np.abs(v - ref[:, 1])) <= tol, (p, v, ref[:, 1])


def test_predict_many_points_consistent():
    """100,000 points in one call: the same values as the points one by one
    (grouping by leaf, chunking and the per-warp scratch do not mix points),
    and 0 <= var <= sigma2."""
    x, y, z = synth.uniform(4096, 15, exact=False)
    rng = np.random.default_rng(9)
    px, py = _points(rng, 100000)
    th = [1.3, 0.08, 0.02]
    with mra.MRA(x, y, z, 4, 4, 16, precision="mixed") as g:
        m, v = g.predict(th, px, py)
        assert np.all(np.isfinite(m)) and np.all(v >= -1e-6) and np.all(v <= th[0] + 1e-6)
        idx = rng.choice(len(px), 20, replace=False)
        for k in idx:
            m1, v1 = g.predict(th, px[k:k + 1], py[k:k + 1])
            assert m1[0] == m[k] and v1[0] == v[k]


def test_predict_errors_and_empty_call():
    """EINVAL for a theta that is not finite and positive (the context stays
    usable), nothing to do for zero points, NaN for non-finite locations."""
    x, y, z = synth.uniform(300, 16)
    with mra.MRA(x, y, z, 3, 4, 9) as g:
        for bad in ([0.0, 0.1, 0.05], [1.0, -0.1, 0.05], [1.0, 0.1, np.inf]):
            with pytest.raises(mra.MRAError) as e:
                g.predict(bad, [0.5], [0.5])
            assert e.value.status == 1
        m, v = g.predict([1.0, 0.1, 0.05], [], [])
        assert m.size == 0 and v.size == 0
        m, v = g.predict([1.0, 0.1, 0.05], [np.nan, 0.5, np.inf], [0.5, 0.5, 0.5])
        assert np.isnan(m[0]) and np.isnan(m[2]) and np.isfinite(m[1]) and np.isfinite(v[1])
        ref_m, ref_v = dense.predict(x, y, z, 3, 4, 9, [1.0, 0.1, 0.05], [0.5], [0.5])
        assert abs(m[1] - ref_m[0]) <= TOL64 and abs(v[1] - ref_v[0]) <= TOL64


def test_predict_reuses_factors_only_while_valid():
    """The factors of the last prediction pass are reused for the same theta
    and recomputed after any other pass or theta: the values stay those of a
    fresh context."""
    x, y, z = synth.uniform(600, 17)
    rng = np.random.default_rng(10)
    px, py = _points(rng, 50)
    t1, t2 = [1.0, 0.1, 0.05], [1.7, 0.2, 0.02]
    with mra.MRA(x, y, z, 4, 4, 9, precision="mixed") as fresh:
        r1 = fresh.predict(t1, px, py)
    with mra.MRA(x, y, z, 4, 4, 9, precision="mixed") as fresh:
        r2 = fresh.predict(t2, px, py)
    with mra.MRA(x, y, z, 4, 4, 9, precision="mixed") as g:
        for th, ref in ((t1, r1), (t1, r1), (t2, r2), (t1, r1)):
            m, v = g.predict(th, px, py)
            assert np.array_equal(m, ref[0]) and np.array_equal(v, ref[1])
        g.loglik([t2])  # another pass: the kept factors of t1 are stale
        m, v = g.predict(t1, px, py)
        assert np.array_equal(m, r1[0]) and np.array_equal(v, r1[1])
        g.set_precision("fp64")
        m, v = g.predict(t1, px, py)
        ref_m, ref_v = dense.predict(x, y, z, 4, 4, 9, t1, px, py)
        assert np.max(np.abs(m - ref_m)) <= TOL64 and np.max(np.abs(v - ref_v)) <= TOL64
