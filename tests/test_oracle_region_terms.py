"""Pin of the oracle's per-region terms below the root (oracle_region_terms).

For a region R of level m holding the observations S_R with values z_R, the
recursion's record after R's step is the log-determinant and the quadratic
form of z_R under the covariance the data of R have once the basis weights of
levels m..M are integrated out and those of the coarser levels are held at
zero (Sec. 1.1: the levels' terms are independent and add up):

    Sigma_R = sum_{l=m}^{M-1} [same level-l region] C_l(a, Q) C_l(Q, Q)^{-1} C_l(Q, b)
              + [same leaf] C_M(a, b) + tau2 [a = b],        a, b in S_R,
    d_R = log |Sigma_R|,   u_R = z_R' Sigma_R^{-1} z_R.

At a leaf Sigma_R is V = C_M(S, S) + tau2 I; at the root it is the whole
Sigma_MRA + tau2 I.  Sigma_R here comes from oracle/dense.py (the brute-force
Sigma_MRA built pair by pair from the C_m recursion, its own tree code), so the
check does not reuse the recursion it tests.  Planted mistakes in the lines
that record the terms (compiled here from a private copy of mra_oracle.c) must
each fail it.
"""
import math
import os
import subprocess

import numpy as np
import pytest

import oracle
from oracle import dense
from paper_1905_00141_gb300 import synth

SRC = os.path.join(os.path.dirname(oracle.__file__), "mra_oracle.c")
REL = 1e-10

# (n, M, J, r, seed, hole): hole empties the lower-left quarter (empty leaves
# and an empty subtree), keeping the extreme points so the domain is unchanged
CASES = [
    (160, 3, 4, 9, 51, False),
    (220, 4, 4, 4, 52, True),
    (180, 4, 2, 9, 53, False),
    (200, 5, 2, 6, 54, True),
    (240, 3, 2, 16, 55, True),
    (150, 5, 4, 2, 56, False),
]
THETA = (1.3, 0.15, 0.04)


def _data(n, seed, hole):
    x, y, z = synth.uniform(n, seed)
    if hole:
        out = (x < 0.45) & (y < 0.45)
        for a in (np.argmin(x), np.argmin(y), np.argmax(x), np.argmax(y)):
            out[a] = False
        x, y, z = x[~out], y[~out], z[~out]
    return x, y, z


def _dense_terms(x, y, z, M, J, r, theta):
    """(d_R, u_R) of every region from the dense definition, by global id
    (level 1 first, children of (m, i) are (m+1, J i + j))."""
    s2, b, t2 = theta
    part = dense.Partition(x, y, z, M, J, r)
    d, u, bounds = [], [], []
    for m in range(1, M + 1):
        S = dense.sigma_mra(part, s2, b, first_level=m)
        reg = part.region_of(part.x, part.y, m - 1)
        for i, bx in enumerate(part.levels[m - 1]):
            bounds.append(bx)
            idx = np.flatnonzero(reg == i)
            if len(idx) == 0:
                d.append(0.0)
                u.append(0.0)
                continue
            K = S[np.ix_(idx, idx)] + t2 * np.eye(len(idx))
            L = np.linalg.cholesky(K)
            w = np.linalg.solve(L, part.z[idx])
            d.append(2.0 * float(np.sum(np.log(np.diag(L)))))
            u.append(float(w @ w))
    return np.array(d), np.array(u), np.array(bounds)


def _check(rt, ref_d, ref_u):
    scale_d = np.maximum(np.abs(ref_d), 1.0)
    scale_u = np.maximum(np.abs(ref_u), 1.0)
    return (np.all(np.abs(rt["d"] - ref_d) <= REL * scale_d) and
            np.all(np.abs(rt["u"] - ref_u) <= REL * scale_u))


@pytest.mark.parametrize("n,M,J,r,seed,hole", CASES)
def test_region_terms_equal_restricted_sigma_mra(n, M, J, r, seed, hole):
    x, y, z = _data(n, seed, hole)
    ref_d, ref_u, bounds = _dense_terms(x, y, z, M, J, r, THETA)
    t = oracle.Tree(x, y, z, M, J, r)
    try:
        # both trees number the regions the same way
        assert np.array_equal(t.export()["bounds"], bounds)
        rt = t.region_terms(np.array(THETA))
    finally:
        t.close()
    assert rt["status"] == oracle.OK
    if hole and M >= 4:
        assert np.sum(ref_u == 0.0) > 0  # empty regions are part of the check
    assert _check(rt, ref_d, ref_u), (np.max(np.abs(rt["d"] - ref_d)), np.max(np.abs(rt["u"] - ref_u)))
    # the root's terms give the likelihood
    ll = -0.5 * (ref_d[0] + ref_u[0] + t.n_used * math.log(2.0 * math.pi))
    assert abs(rt["loglik"] - ll) <= REL * abs(ll)


# mistakes in the recording of the terms only: the likelihood itself stays
# right, so only this pin can catch them
MUTATIONS = {
    "region_d_before_own_step": ("if (c->rd) { c->rd[g] = *d; c->ru[g] = *u; c->rlw[g] = self.logdetW; }",
                                 "if (c->rd) { c->rd[g] = ds; c->ru[g] = *u; c->rlw[g] = self.logdetW; }"),
    "region_u_children_sum": ("if (c->rd) { c->rd[g] = *d; c->ru[g] = *u; c->rlw[g] = self.logdetW; }",
                              "if (c->rd) { c->rd[g] = *d; c->ru[g] = us; c->rlw[g] = self.logdetW; }"),
    "region_d_without_prior_logdet": (
        "if (c->rd) { c->rd[g] = *d; c->ru[g] = *u; c->rlw[g] = self.logdetW; }",
        "if (c->rd) { c->rd[g] = ds + logdetT; c->ru[g] = *u; c->rlw[g] = self.logdetW; }"),
    "leaf_terms_swapped": ("if (c->rd) { c->rd[g] = *d; c->ru[g] = *u; c->rlw[g] = NAN; }\n    free(B);",
                           "if (c->rd) { c->rd[g] = *u; c->ru[g] = *d; c->rlw[g] = NAN; }\n    free(B);"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_recording_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / ("libmut_%s.so" % name)
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so), str(path),
                    "-lm"], check=True)
    lib = oracle.load_variant(str(so))
    n, M, J, r, seed, hole = CASES[1]
    x, y, z = _data(n, seed, hole)
    ref_d, ref_u, _ = _dense_terms(x, y, z, M, J, r, THETA)
    t = oracle.Tree(x, y, z, M, J, r, lib=lib)
    try:
        rt = t.region_terms(np.array(THETA))
        ll, _ = t.loglik(np.array(THETA))
        n_used = t.n_used
    finally:
        t.close()
    # the likelihood is untouched by a recording mistake ...
    lref = -0.5 * (ref_d[0] + ref_u[0] + n_used * math.log(2.0 * math.pi))
    assert abs(ll[0] - lref) <= REL * abs(lref)
    # ... but the per-region pin fails
    assert not _check(rt, ref_d, ref_u)
