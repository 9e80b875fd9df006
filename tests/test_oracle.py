"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: the checks are the paper's
printed knot counts and toy example (Sec. 1.2, Sec. 3.1.2 table), the exact
dense Gaussian likelihood at M=1 (scipy), a brute-force Sigma_MRA built pair by
pair from the C_m recursion of Sec. 1.1 (oracle/dense.py, its own tree code),
and invariants the MRA must satisfy.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import dense
from paper_1905_00141_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_rows(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([float(v) for v in line.split()])
    return rows


def test_rhat_table_sec312():
    for M, r, rhat in _read_rows("rhat_table.txt"):
        kx, ky = oracle.place_knots(0.0, 1.0, 0.0, 1.0, int(r), 0.1)
        assert len(kx) == int(rhat)
        assert dense.grid_dims(int(r))[0] * dense.grid_dims(int(r))[1] == int(rhat)


def test_knots_toy_example_sec12():
    xb, yb = _read_rows("knots_toy_r32_offset0.1.txt")
    kx, ky = oracle.place_knots(0.0, 1.0, 0.0, 1.0, 32, 0.1)
    assert len(kx) == 30
    assert np.allclose(np.unique(np.round(kx, 12)), xb, atol=1e-12)
    assert np.allclose(np.unique(np.round(ky, 12)), yb, atol=1e-12)
    # x fastest: first 6 knots share the lowest y bar
    assert np.allclose(ky[:6], 0.1) and np.allclose(kx[:6], xb)


def test_knots_non_unit_region_app_a():
    # App. A form: x0 + L (f + p (1-2f)/(n-1)); first bar at f*L from x0, last at f*L from x1
    kx, ky = oracle.place_knots(2.0, 6.0, -1.0, 0.0, 16, 0.05)
    assert np.isclose(kx.min(), 2.0 + 0.05 * 4.0) and np.isclose(kx.max(), 6.0 - 0.05 * 4.0)
    assert np.isclose(ky.min(), -1.0 + 0.05) and np.isclose(ky.max(), -0.05)
    assert len(np.unique(np.round(kx, 12))) == 4 and len(np.unique(np.round(ky, 12))) == 4


def test_partition_rules_sec12():
    rng = np.random.default_rng(3)
    x = rng.random(300) * 3.0  # wider than tall: J=2 cuts x first
    y = rng.random(300)
    z = rng.standard_normal(300)
    t = oracle.Tree(x, y, z, M=3, J=2, r=4)
    b = t.export()["bounds"]
    root = b[0]
    assert root[0] == x.min() and root[2] == y.min()
    assert np.isclose(root[1], x.max() + 0.01 * (x.max() - x.min()))
    assert np.isclose(root[3], y.max() + 0.01 * (y.max() - y.min()))
    # level 2: cut along x (the longer side)
    assert b[1][1] == b[2][0] and b[1][2] == b[2][2] == root[2]
    # level 3: the level-2 regions are 1.5 x 1 wide x tall, cut x again
    assert b[3][1] == b[4][0] and b[3][3] == b[4][3]
    t4 = oracle.Tree(x, y, z, M=2, J=4, r=4)
    b4 = t4.export()["bounds"]
    mx, my = 0.5 * (b4[0][0] + b4[0][1]), 0.5 * (b4[0][2] + b4[0][3])
    assert tuple(b4[1]) == (b4[0][0], mx, b4[0][2], my)
    assert tuple(b4[4]) == (mx, b4[0][1], my, b4[0][3])


def test_half_open_and_extension():
    # points on the maximum edge stay (1% extension); a point on an interior
    # split line goes to the upper/right child
    x = np.array([0.0, 1.0, 0.5, 0.25, 0.9, 0.1])
    y = np.array([0.0, 1.0, 0.5, 0.75, 0.2, 0.6])
    z = np.arange(6.0)
    t = oracle.Tree(x, y, z, M=2, J=4, r=1, offset=0.3)
    e = t.export()
    assert t.n_used == 6
    mid = 0.5 * (0.0 + 1.01)
    leaf = np.repeat(np.arange(4), np.diff(e["leaf_off"]))
    got = dict(zip(e["perm"].tolist(), leaf.tolist()))
    for i in range(6):
        want = (1 if x[i] >= mid else 0) + (2 if y[i] >= mid else 0)
        assert got[i] == want


def test_drops_nan_duplicate_and_knot_coincident():
    x, y, z = synth.uniform(200, 11, exact=False)
    kx, ky = oracle.place_knots(x.min(), x.max() + 0.01 * (x.max() - x.min()),
                                y.min(), y.max() + 0.01 * (y.max() - y.min()), 9, math.e / 100)
    x2 = np.concatenate([x, [x[5], kx[4]]])
    y2 = np.concatenate([y, [y[5], ky[4]]])
    z2 = np.concatenate([z, [0.3, 0.1]])
    z2[7] = np.nan
    t = oracle.Tree(x2, y2, z2, M=2, J=4, r=9, dedup=True)
    assert t.n_nan == 1 and t.n_dup == 1 and t.n_knot == 1 and t.n_used == 199
    t2 = oracle.Tree(x2, y2, z2, M=2, J=4, r=9, dedup=False)
    assert t2.n_dup == 0 and t2.n_used == 200


def test_m1_is_exact_dense_gaussian():
    from scipy.stats import multivariate_normal
    x, y, z = synth.uniform(400, 5)
    th = (1.0, 0.1, 0.05)
    ll, st = oracle.loglik(x, y, z, 1, 4, 16, th)
    d = np.sqrt((x[:, None] - x[None, :]) ** 2 + (y[:, None] - y[None, :]) ** 2)
    S = th[0] * np.exp(-d / th[1]) + th[2] * np.eye(len(x))
    ref = multivariate_normal(mean=np.zeros(len(x)), cov=S).logpdf(z)
    assert st == oracle.OK
    assert abs(ll[0] - ref) <= 1e-10 * abs(ref)


CASES = [
    (90, 2, 4, 9, 1), (150, 3, 4, 9, 2), (200, 3, 4, 16, 3), (120, 3, 2, 4, 4),
    (200, 4, 2, 9, 5), (160, 4, 4, 4, 6), (100, 5, 2, 6, 7), (180, 2, 2, 30, 8),
    (260, 3, 2, 49, 9), (220, 2, 4, 64, 10),
]


@pytest.mark.parametrize("n,M,J,r,seed", CASES)
def test_matches_brute_force_sigma_mra(n, M, J, r, seed):
    x, y, z = synth.uniform(n, seed)
    for th in [(1.0, 0.1, 0.05), (2.5, 0.3, 0.01), (0.7, 0.02, 0.2)]:
        ll, st = oracle.loglik(x, y, z, M, J, r, th)
        ref = dense.loglik(x, y, z, M, J, r, th)
        assert st == oracle.OK
        assert abs(ll[0] - ref) <= 1e-10 * abs(ref), (th, ll[0], ref)


def test_brute_force_is_exact_within_a_leaf_and_at_knots():
    x, y, z = synth.uniform(150, 21)
    part = dense.Partition(x, y, z, 3, 4, 9)
    S, info = dense.sigma_mra(part, 1.3, 0.2, return_all=True)
    X, Y, reg = info["X"], info["Y"], info["reg"]
    C = 1.3 * np.exp(-np.sqrt((X[:, None] - X[None, :]) ** 2 + (Y[:, None] - Y[None, :]) ** 2) / 0.2)
    n = info["n_obs"]
    same_leaf = reg[-1][:n, None] == reg[-1][None, :n]
    assert np.allclose(S[:n, :n][same_leaf], C[:n, :n][same_leaf], rtol=0, atol=1e-12)
    assert np.allclose(np.diag(S)[:n], 1.3, atol=1e-12)
    # a knot q of a level-m region and any point s of that region: Sigma(q, s) = C(q, s)
    for m, regions in enumerate(info["knot_ids"]):
        for k, q in enumerate(regions):
            members = np.nonzero(reg[m] == k)[0]
            assert np.allclose(S[np.ix_(q, members)], C[np.ix_(q, members)], atol=1e-10)
    # Sigma_MRA is symmetric positive definite
    assert np.allclose(S, S.T, atol=1e-13)
    assert np.linalg.eigvalsh(S[:n, :n]).min() > -1e-10


def test_permutation_invariance():
    x, y, z = synth.uniform(500, 9)
    th = (1.0, 0.1, 0.05)
    a, _ = oracle.loglik(x, y, z, 3, 4, 16, th)
    p = np.random.default_rng(1).permutation(len(x))
    b, _ = oracle.loglik(x[p], y[p], z[p], 3, 4, 16, th)
    assert abs(a[0] - b[0]) <= 1e-11 * abs(a[0])


def test_scaling_identity():
    # l(c s2, b, c t2; sqrt(c) z) = l(s2, b, t2; z) - (n/2) log c
    x, y, z = synth.uniform(600, 13)
    c = 3.7
    a, _ = oracle.loglik(x, y, z, 3, 4, 16, (1.1, 0.08, 0.03))
    b, _ = oracle.loglik(x, y, math.sqrt(c) * z, 3, 4, 16, (1.1 * c, 0.08, 0.03 * c))
    assert abs(b[0] - (a[0] - 0.5 * len(x) * math.log(c))) <= 1e-10 * abs(a[0])


def test_empty_leaves_and_subtree_match_brute_force():
    x, y, z = synth.uniform(260, 17)
    # keep the bounding box, empty the lower-left quarter except the corner
    # extremes so the tree stays the same, leaving an empty level-2 subtree
    hole = (x < 0.45) & (y < 0.45)
    keep = ~hole
    keep[np.argmin(x)] = keep[np.argmin(y)] = True
    keep[np.argmax(x)] = keep[np.argmax(y)] = True
    x, y, z = x[keep], y[keep], z[keep]
    t = oracle.Tree(x, y, z, 4, 4, 9)
    counts = np.diff(t.export()["leaf_off"])
    assert (counts == 0).sum() >= 8
    for th in [(1.0, 0.1, 0.05), (1.0, 0.4, 0.02)]:
        ll, st = t.loglik(th)
        ref = dense.loglik(x, y, z, 4, 4, 9, th)
        assert st == oracle.OK and abs(ll[0] - ref) <= 1e-10 * abs(ref)


def test_region_terms_sum_to_loglik():
    x, y, z = synth.uniform(700, 23)
    t = oracle.Tree(x, y, z, 3, 4, 16)
    rt = t.region_terms(np.array([1.0, 0.1, 0.05]))
    ll = -0.5 * (rt["d"][0] + rt["u"][0] + t.n_used * math.log(2 * math.pi))
    assert abs(ll - rt["loglik"]) < 1e-9 * abs(ll)
    lo = 1 + 4  # leaves start after levels 1 and 2
    assert np.all(np.isnan(rt["logdetW"][lo:])) and np.all(np.isfinite(rt["logdetW"][:lo]))


def test_bad_theta_and_not_pd():
    x, y, z = synth.uniform(200, 29)
    t = oracle.Tree(x, y, z, 3, 4, 9)
    ll, st = t.loglik(np.array([[1.0, 0.1, 0.05], [-1.0, 0.1, 0.05], [1.0, 0.1, 0.0]]))
    assert st == oracle.EINVAL and np.isfinite(ll[0]) and np.isnan(ll[1]) and np.isnan(ll[2])
    # a range so long that the exponential kernel is numerically rank one
    ll, st = t.loglik(np.array([[1.0, 1e8, 0.05]]))
    assert st == oracle.ENOTPD and np.isnan(ll[0])


def test_invalid_and_empty_inputs():
    x, y, z = synth.uniform(50, 31, exact=False)
    with pytest.raises(oracle.OracleError) as e:
        oracle.Tree(x, y, z, 3, 3, 9)
    assert e.value.status == oracle.EINVAL
    with pytest.raises(oracle.OracleError) as e:
        oracle.Tree(x, y, np.full(50, np.nan), 3, 4, 9)
    assert e.value.status == oracle.EEMPTY
    with pytest.raises(oracle.OracleError) as e:
        oracle.Tree(x[:0], y[:0], z[:0], 3, 4, 9)
    assert e.value.status == oracle.EEMPTY


def test_thread_count_does_not_change_result():
    d = synth.small()
    t = oracle.Tree(d["x"], d["y"], d["z"], d["M"], d["J"], d["r"])
    a, _ = t.loglik(d["theta"], nthreads=1)
    b, _ = t.loglik(d["theta"], nthreads=4)
    assert a[0] == b[0]
