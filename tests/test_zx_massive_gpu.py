"""The 47,185,920-observation tree (M=12, J=4, r=16, mixed precision) at full
size on one GPU, checked on sampled outputs the oracle computes one by one.

A leaf's terms (log|V|, z'V^{-1}z) depend only on its own observations and on
the prior of its ancestors, which the knots fix; the knots depend on the data
only through its bounding box.  So the oracle evaluates a reduced data set --
the points that set the bounding box plus the observations of a few sampled
leaves -- on the same M=12 tree (its empty subtrees cost nothing), and those
leaves' terms must equal the GPU's terms from the full data, to the precision
of mixed-mode leaf terms.  The full
likelihood itself is checked for a finite value and an OK status, and the
theta-batched call against single calls."""
import numpy as np
import pytest

import oracle
from paper_1905_00141_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def massive():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    free, _ = torch.cuda.mem_get_info()
    if free < 200e9:
        pytest.skip("needs ~180 GB of free device memory")
    from paper_1905_00141_gb300 import build, mra
    build.build()
    oracle.build()
    d = synth.massive()
    g = mra.MRA(d["x"], d["y"], d["z"], d["M"], d["J"], d["r"], precision="mixed")
    yield d, g
    g.close()


def test_massive_sampled_leaves_match_oracle(massive):
    d, g = massive
    th = d["theta"][0]
    st = g.stats()
    assert st["n_used"] == len(d["x"])
    rg = g.region_terms(th)
    assert rg["status"] == 0 and np.isfinite(rg["loglik"])
    tr = g.tree()
    off, perm = np.asarray(tr["leaf_off"]), np.asarray(tr["perm"])
    nleaf = len(off) - 1
    lvl_leaf = st["n_regions"] - nleaf  # global id of the first leaf
    ext = {int(np.argmin(d["x"])), int(np.argmax(d["x"])), int(np.argmin(d["y"])), int(np.argmax(d["y"]))}
    rng = np.random.default_rng(7)
    counts = np.diff(off)
    cand = np.flatnonzero(counts > 0)
    picks = list(rng.choice(cand, 12, replace=False)) + [int(np.argmax(counts))]
    picks = [c for c in picks if not (set(perm[off[c]:off[c + 1]].tolist()) & ext)]
    assert len(picks) >= 8
    rows = sorted(ext) + [int(k) for c in picks for k in perm[off[c]:off[c + 1]]]
    xr, yr, zr = d["x"][rows], d["y"][rows], d["z"][rows]
    t = oracle.Tree(xr, yr, zr, d["M"], d["J"], d["r"])
    try:
        ro = t.region_terms(th)
        eo = t.export()
    finally:
        t.close()
    assert ro["status"] == 0
    ooff = np.asarray(eo["leaf_off"])
    for c in picks:
        nl = off[c + 1] - off[c]
        assert ooff[c + 1] - ooff[c] == nl  # the same leaf holds the same observations
        gid = lvl_leaf + c
        for key in ("d", "u"):
            # mixed-mode leaf terms are those of the FP32-rounded basis U, a model
            # within ~1e-7 of the exact one, whose log|V| and z'V^{-1}z move by up
            # to ~1e-5 relative on their own (the upward pass cancels most of it);
            # a wrong index or term would move them by O(1)
            assert abs(rg[key][gid] - ro[key][gid]) <= 1e-4 * (abs(ro[key][gid]) + nl), \
                (c, key, rg[key][gid], ro[key][gid])


def test_massive_batch_equals_single_calls(massive):
    d, g = massive
    th = synth.theta_grid_4x4x4()[[0, 21, 42, 63]]
    batch = g.loglik(th)
    single = np.array([g.loglik(th[k])[0] for k in range(len(th))])
    assert np.all(np.isfinite(batch))
    assert np.array_equal(batch, single)
