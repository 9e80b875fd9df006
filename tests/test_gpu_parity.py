"""GPU (sm_103a) likelihood against the FP64 oracle, through the C ABI.

Tolerances (|loglik_gpu - loglik_oracle| / n): FP64 path 1e-10, mixed path
1e-6 (the mixed target of the workload definition).  Both sides evaluate the
same likelihood by different routes: the oracle in the paper's K form, the
GPU in the whitened form, so agreement checks the arithmetic, not a shared
code path.
"""
import numpy as np
import pytest

import oracle
from paper_1905_00141_gb300 import build as mbuild
from paper_1905_00141_gb300 import mra, synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOLMIX = 1e-6
THETAS = np.array([[1.0, 0.1, 0.05], [2.5, 0.3, 0.01], [0.7, 0.02, 0.2]])


@pytest.fixture(scope="module", autouse=True)
def _built():
    mbuild.build()
    oracle.build()


def _parity(x, y, z, M, J, r, thetas=THETAS, precisions=("fp64", "mixed"), build_precision="fp64", **kw):
    ref, st = oracle.loglik(x, y, z, M, J, r, thetas, **kw)
    assert st == 0
    out = {}
    with mra.MRA(x, y, z, M, J, r, precision=build_precision, **kw) as g:
        n = g.stats()["n_used"]
        for p in precisions:
            g.set_precision(p)
            got = g.loglik(thetas)
            err = np.abs(got - ref) / n
            tol = TOL64 if p == "fp64" else TOLMIX  # mixed and mixed_fast
            assert np.all(err <= tol), (p, got, ref, err)
            out[p] = err
    return out


@pytest.mark.parametrize("n,M,J,r,seed", [
    (300, 1, 4, 16, 1),     # the root is one leaf of 300 (large-leaf path)
    (600, 2, 4, 16, 2),
    (2000, 3, 4, 9, 3),     # r_hat = 9, padded to 16
    (3000, 4, 2, 30, 4),    # J = 2, r_hat = 30, padded to 32
    (3000, 5, 4, 32, 5),
    (4000, 6, 2, 16, 6),
    (1500, 4, 4, 2, 7),     # r_hat = 2
    (2300, 4, 4, 32, 8),    # leaves of about 36: the <=32, <=40, <=48 and <=64 buckets
])
def test_parity_small_trees(n, M, J, r, seed):
    x, y, z = synth.uniform(n, seed)
    _parity(x, y, z, M, J, r)


def test_parity_ragged_leaves_and_empty_subtrees():
    x, y, z = synth.uniform(3000, 11)
    hole = (x < 0.5) & (y < 0.5) & ~((x < 0.02) | (y < 0.02))
    x, y, z = x[~hole], y[~hole], z[~hole]
    # a dense cluster makes leaves of > 64 observations next to empty ones
    rng = np.random.default_rng(5)
    cx = 0.8 + 0.01 * rng.standard_normal(400)
    cy = 0.8 + 0.01 * rng.standard_normal(400)
    x, y = np.concatenate([x, cx]), np.concatenate([y, cy])
    z = np.concatenate([z, rng.standard_normal(400)])
    with mra.MRA(x, y, z, 4, 4, 16) as g:
        s = g.stats()
        assert s["empty_leaves"] > 0 and s["max_leaf"] > 64
    _parity(x, y, z, 4, 4, 16)


def test_parity_small_workload():
    d = synth.small()
    _parity(d["x"], d["y"], d["z"], d["M"], d["J"], d["r"], d["theta"])


def test_parity_grid_workload_full_size():
    d = synth.grid()
    th = np.array([[1.0, 0.05, 0.01], [1.3, 0.08, 0.02]])
    err = _parity(d["x"], d["y"], d["z"], d["M"], d["J"], d["r"], th)
    print("grid |dl|/n", {k: v.tolist() for k, v in err.items()})


def _region_counts(t):
    """Observations below every region (global id order) of an oracle tree."""
    e = t.export()
    cnt = np.diff(e["leaf_off"]).astype(np.int64)
    levels = [cnt]
    while len(levels[-1]) > 1:
        levels.append(levels[-1].reshape(-1, t.J).sum(1))
    return np.concatenate(levels[::-1])


# Per-region tolerances.  FP64: 1e-9 relative.  Mixed: the path carries the
# FP32-rounded whitened basis U, a model within ~1e-7 sigma2 of the exact one.  U
# enters a leaf twice -- in V = C - U U' + tau2 I and in the coarse part U U' -- and
# the two perturbations cancel exactly only once all levels are summed, at the root
# (Sigma = U U' + (C - U U') within a leaf).  Below the root, V's small eigenvalues
# (~tau2) carry the rounding of U U' relative to sigma2 / tau2, which moves a
# region's log|.| and quadratic form by up to a few 1e-6 of their size, so
# d_R + u_R is held to 1e-5 of (|d_R| + |u_R| + n_R) and d_R, u_R alone to 1e-5 of
# (|term| + n_R); the root, the likelihood, to the 1e-6 per observation of the
# mixed path.
TOL_REGION_MIX = 1e-5


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("M,J,r", [(4, 4, 16), (4, 2, 49)])
def test_region_terms_match_oracle(precision, M, J, r):
    # r = 49: the GPU runs every level as two device levels of the same
    # regions; its records are mapped back to the partition's regions (d, u of
    # the first half-level, log|W| summed over the halves)
    x, y, z = synth.uniform(3000, 21)
    th = np.array([1.2, 0.15, 0.03])
    t = oracle.Tree(x, y, z, M, J, r)
    ro = t.region_terms(th)
    nr = _region_counts(t).astype(np.float64)
    with mra.MRA(x, y, z, M, J, r, precision=precision) as g:
        rg = g.region_terms(th)
    assert rg["status"] == 0 and ro["status"] == 0
    k = np.isfinite(ro["logdetW"])
    assert np.array_equal(k, np.isfinite(rg["logdetW"]))
    if precision == "fp64":
        scale = np.abs(ro["d"]).max() + np.abs(ro["u"]).max()
        assert np.allclose(rg["d"], ro["d"], rtol=1e-9, atol=1e-10 * scale)
        assert np.allclose(rg["u"], ro["u"], rtol=1e-9, atol=1e-10 * scale)
        assert np.allclose(rg["logdetW"][k], ro["logdetW"][k], rtol=1e-9, atol=1e-9)
        assert abs(rg["loglik"] - ro["loglik"]) <= TOL64 * t.n_used
        return
    # the GPU carries the whitened form: its log|W^m| is the oracle's, to FP32 level
    assert np.allclose(rg["logdetW"][k], ro["logdetW"][k], rtol=1e-5, atol=1e-4)
    err_sum = np.abs((rg["d"] + rg["u"]) - (ro["d"] + ro["u"])) / (np.abs(ro["d"]) + np.abs(ro["u"]) + nr + 1.0)
    err_d = np.abs(rg["d"] - ro["d"]) / (np.abs(ro["d"]) + nr + 1.0)
    err_u = np.abs(rg["u"] - ro["u"]) / (np.abs(ro["u"]) + nr + 1.0)
    print("mixed per-region: max relative |d+u| err %.3g, d %.3g, u %.3g" % (err_sum.max(), err_d.max(), err_u.max()))
    assert np.all(err_sum <= TOL_REGION_MIX), err_sum.max()
    assert np.all(err_d <= 1e-5) and np.all(err_u <= 1e-5), (err_d.max(), err_u.max())
    assert abs(rg["loglik"] - ro["loglik"]) <= TOLMIX * t.n_used


# r_hat > 32: the kernels enter each region's knots in two device levels (the
# first ceil(r_hat/2), then the rest: Sec. 1.1 recursion in two steps); the
# oracle evaluates the paper's tree with all r_hat knots of a region at once.
@pytest.mark.parametrize("n,M,J,r,seed", [
    (3000, 3, 2, 49, 51),   # the paper's r = 49 on a binary tree
    (4000, 4, 2, 49, 52),
    (3000, 3, 4, 49, 53),
    (2500, 2, 4, 64, 54),   # r_hat = 64: two halves of 32
    (3000, 5, 2, 36, 55),   # r_hat = 36: 18 + 18, padded to 32 each
    (600, 1, 4, 49, 56),    # M = 1: no knots, one leaf
    (6000, 7, 2, 49, 57),   # 13 device levels: the deepest r = 49 tree the FP64 kernels fit
])
def test_parity_wide_regions(n, M, J, r, seed):
    x, y, z = synth.uniform(n, seed)
    with mra.MRA(x, y, z, M, J, r, device=-1) as h:
        assert h.stats()["device_levels"] == (2 * (M - 1) + 1 if M > 1 else 1)
    err = _parity(x, y, z, M, J, r)
    print("r=%d M=%d J=%d |dl|/n" % (r, M, J), {k: float(v.max()) for k, v in err.items()})


@pytest.mark.parametrize("n,M,seed", [(60000, 10, 61), (60000, 14, 62)])
def test_parity_deep_binary_trees_r49(n, M, seed):
    """The paper's AMSR tree shape (J = 2, r = 49) at depth 10 and 14: 19 and
    27 device levels, on the swaths generator's data (slanted passes with
    gaps, a GP field) at 60,000 points.  Only the mixed modes fit the
    shared-memory kernels this deep; the FP64 mode is refused with EINVAL."""
    d = synth.swaths(seed=seed, n=n, grid_n=512)
    x, y, z = d["x"], d["y"], d["z"]
    th = np.array([[1.0, 0.05, 0.01], [1.5, 0.15, 0.005]])
    err = _parity(x, y, z, M, 2, 49, th, precisions=("mixed",), build_precision="mixed")
    print("deep r=49 M=%d |dl|/n" % M, float(err["mixed"].max()))
    with mra.MRA(x, y, z, M, 2, 49, precision="mixed") as g:
        # the default leaf basis of this depth streams its ancestor blocks; the
        # 32-row kernel (one CTA per SM here) gives the same U bit for bit
        ll = g.loglik(th)
        g.set_launch(32, 1, 0, True)
        assert np.array_equal(g.loglik(th), ll)
        g.set_launch(0, 0, 0, True)
        with pytest.raises(mra.MRAError) as e:
            g.set_precision("fp64")
        assert e.value.status == mra.EINVAL
    with pytest.raises(mra.MRAError) as e:
        mra.MRA(x, y, z, M, 2, 49, precision="fp64")
    assert e.value.status == mra.EINVAL


def test_parity_m18_binary_tree_r49():
    """The paper's large-MODIS tree shape, J = 2, M = 18, r = 49: 35 device
    levels and 131,071 regions.  This deep, the prior and the upward pass
    stage their blocks in parts, the large-leaf assembly reads its rows in
    two parts, and the ATilde arrays of the whole tree (hundreds of GB) do not
    fit, so the memory plan streams subtrees by itself.  The data (tight
    clusters, a sprinkle of points) leaves most subtrees empty, which the
    oracle skips; the device path runs every region."""
    x, y, z = synth.sparse_clusters(30000, 81, sd=0.006)
    th = np.array([[1.0, 0.05, 0.01], [1.5, 0.15, 0.005]])
    ref, st = oracle.loglik(x, y, z, 18, 2, 49, th)
    assert st == 0
    with mra.MRA(x, y, z, 18, 2, 49, precision="mixed") as g:
        s = g.stats()
        assert s["device_levels"] == 35 and s["n_regions"] == 2 ** 18 - 1
        assert s["subtree_level"] > 0 and s["subtree_chunks"] >= 1
        assert s["max_leaf"] > 64
        ll = g.loglik(th)
        n = s["n_used"]
        print("M=18 r=49: subtree level %d, %d chunks, |dl|/n" % (s["subtree_level"], s["subtree_chunks"]),
              np.abs(ll - ref) / n)
        assert np.all(np.abs(ll - ref) / n <= TOLMIX)
        # another level and chunking (6 chunks of 3 of the 16 real-level-5
        # subtrees) gives the same values bit for bit
        g.set_launch(subtree_level=9, subtree_chunk=3)
        assert g.stats()["subtree_chunks"] == 6
        assert np.array_equal(g.loglik(th), ll)


def test_batch_with_invalid_theta():
    x, y, z = synth.uniform(1200, 31)
    th = np.array([[1.0, 0.1, 0.05], [np.nan, 0.1, 0.05], [1.0, -0.1, 0.05], [1.0, 0.1, 0.0],
                   [0.9, 0.2, 0.04]])
    ref, _ = oracle.loglik(x, y, z, 3, 4, 16, th)
    with mra.MRA(x, y, z, 3, 4, 16) as g:
        got, st = g.loglik_status(th)
    assert st == mra.EINVAL
    ok = np.isfinite(ref)
    assert list(ok) == [True, False, False, False, True]
    assert np.array_equal(ok, np.isfinite(got))
    assert np.all(np.abs(got[ok] - ref[ok]) / 1200 <= TOL64)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_coincident_knots_are_singular(precision):
    # offset = 0 puts a parent's knots on its children's boundary knots: the
    # remainder covariance of those knots is zero and the prior is singular
    # (Sec. 1.2); both sides must report it.
    x, y, z = synth.uniform(1200, 31)
    th = np.array([[1.0, 0.1, 0.05], [2.0, 0.3, 0.01]])
    ref, st_o = oracle.loglik(x, y, z, 3, 4, 16, th, offset=0.0)
    assert st_o == oracle.ENOTPD and np.all(np.isnan(ref))
    with mra.MRA(x, y, z, 3, 4, 16, offset=0.0, precision=precision) as g:
        got, st = g.loglik_status(th)
    assert st == mra.ENOTPD and np.all(np.isnan(got))


def test_device_api_with_torch_stream_and_batches():
    import torch
    d = synth.small()
    th = np.stack([np.geomspace(0.5, 2.0, 7), np.geomspace(0.03, 0.3, 7), np.geomspace(0.01, 0.1, 7)], 1)
    ref, _ = oracle.loglik(d["x"], d["y"], d["z"], d["M"], d["J"], d["r"], th)
    with mra.MRA(d["x"], d["y"], d["z"], d["M"], d["J"], d["r"], max_batch=3) as g:
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            tt = torch.tensor(th, device="cuda", dtype=torch.float64)
            st = torch.full((7,), -1, dtype=torch.int32, device="cuda")
            out = g.loglik_torch(tt, status=st)
        s.synchronize()
        assert np.all(np.abs(out.cpu().numpy() - ref) / 4096 <= TOL64)
        assert st.cpu().tolist() == [0] * 7
        again = g.loglik(th)
        assert np.array_equal(again, out.cpu().numpy())  # deterministic


def test_mixed_is_not_the_fp64_path():
    # the mixed path must actually change the arithmetic (FP32 bulk)
    d = synth.small()
    with mra.MRA(d["x"], d["y"], d["z"], d["M"], d["J"], d["r"]) as g:
        a = g.loglik(d["theta"])
        g.set_precision("mixed")
        b = g.loglik(d["theta"])
    assert a[0] != b[0] and abs(a[0] - b[0]) / 4096 <= TOLMIX


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_streamed_level_gram_matches_whole_level(precision):
    # a budget of one byte forces the level M-1 Gram blocks to be produced and
    # consumed one region at a time; the result must not change at all
    x, y, z = synth.uniform(3000, 21)
    ref, st = oracle.loglik(x, y, z, 4, 4, 16, THETAS)
    assert st == 0
    with mra.MRA(x, y, z, 4, 4, 16, precision=precision) as g, \
            mra.MRA(x, y, z, 4, 4, 16, precision=precision, hbm_budget=1) as gs:
        a = g.loglik(THETAS)
        b = gs.loglik(THETAS)
        n = g.stats()["n_used"]
    assert np.array_equal(a, b)
    assert np.all(np.abs(b - ref) / n <= (TOL64 if precision == "fp64" else TOLMIX))


def _clustered_uniform(n, seed):
    # uniform points plus two tight clusters (leaves beyond the shared-memory
    # buckets, so the large-leaf pipeline runs too)
    x, y, z = synth.uniform(n, seed, exact=False)
    rng = np.random.default_rng(seed + 1)
    cx = np.concatenate([0.31 + 0.004 * rng.standard_normal(400), 0.77 + 0.003 * rng.standard_normal(300)])
    cy = np.concatenate([0.62 + 0.004 * rng.standard_normal(400), 0.18 + 0.003 * rng.standard_normal(300)])
    return np.concatenate([x, cx]), np.concatenate([y, cy]), np.concatenate([z, rng.standard_normal(700)])


@pytest.mark.parametrize("precision,M,J,r,cases", [
    ("fp64", 5, 4, 16, [(1, 0), (2, 1), (3, 5), (3, 0)]),
    ("mixed", 5, 4, 16, [(2, 3), (3, 7), (3, 1)]),
    # r_hat = 49: device levels 2l-1 and 2l hold the same regions (one child)
    ("mixed", 6, 2, 49, [(4, 3), (5, 2), (9, 5), (7, 0)]),
])
def test_subtree_streaming_matches_whole_levels(precision, M, J, r, cases):
    """The leaf Gram and the upward pass of the levels below S run chunk by
    chunk of level-S subtrees, with ATilde arrays that hold one chunk: the
    same log-likelihoods and per-region terms bit for bit, for every level
    and chunk size (uneven last chunks included), batched theta and graph
    replay."""
    x, y, z = _clustered_uniform(20000, 71)
    with mra.MRA(x, y, z, M, J, r, precision=precision) as g:
        st = g.stats()
        assert st["max_leaf"] > 64 and st["subtree_level"] == 0 and st["subtree_chunks"] == 0
        ref = g.loglik(THETAS)
        terms = g.region_terms(THETAS[1])
        lv = st["device_levels"]
        for S, C in cases:
            g.set_launch(subtree_level=S, subtree_chunk=C)
            s2 = g.stats()
            assert s2["subtree_level"] == S
            assert s2["subtree_chunks"] >= 1
            if C > 0:
                k = S if r <= 32 else (S + 1) // 2  # real level of device level S
                assert s2["subtree_chunks"] == -(-(J ** (k - 1)) // C)
            for _ in range(2):  # the second call replays the captured pass
                assert np.array_equal(g.loglik(THETAS), ref)
            t2 = g.region_terms(THETAS[1])
            for key in ("d", "u", "logdetW"):
                assert np.array_equal(t2[key], terms[key], equal_nan=True), (S, C, key)
            assert t2["loglik"] == terms["loglik"]
        if precision == "mixed":
            # the tensor-core Gram's column exponents follow the chunks too
            g.set_launch(gram_tensor_cores=True)
            tc = g.loglik(THETAS)
            g.set_launch(gram_tensor_cores=True, subtree_level=lv - 3, subtree_chunk=2)
            assert np.array_equal(g.loglik(THETAS), tc)
        for bad in (lv - 1, -1):
            with pytest.raises(mra.MRAError) as e:
                g.set_launch(subtree_level=bad)
            assert e.value.status == mra.EINVAL
        g.set_launch()
        assert g.stats()["subtree_level"] == 0
        assert np.array_equal(g.loglik(THETAS), ref)


def test_precision_switch_resizes_scratch():
    x, y, z = synth.uniform(2000, 22)
    ref, _ = oracle.loglik(x, y, z, 3, 4, 16, THETAS)
    with mra.MRA(x, y, z, 3, 4, 16, precision="mixed") as g:
        n = g.stats()["n_used"]
        m1 = g.loglik(THETAS)
        g.set_precision("fp64")
        d1 = g.loglik(THETAS)
        g.set_precision("mixed")
        m2 = g.loglik(THETAS)
    assert np.array_equal(m1, m2)
    assert np.all(np.abs(d1 - ref) / n <= TOL64)
    assert np.all(np.abs(m1 - ref) / n <= TOLMIX)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_equals_direct_launches(precision):
    torch = pytest.importorskip("torch")
    x, y, z = synth.uniform(5000, 23)
    x = np.concatenate([x, 0.3 + 0.005 * np.random.default_rng(1).standard_normal(300)])
    y = np.concatenate([y, 0.7 + 0.005 * np.random.default_rng(2).standard_normal(300)])
    z = np.concatenate([z, np.random.default_rng(3).standard_normal(300)])  # a few large leaves too
    with mra.MRA(x, y, z, 4, 4, 16, precision=precision, graphs=False) as g0, \
            mra.MRA(x, y, z, 4, 4, 16, precision=precision) as g1:
        assert g0.stats()["max_leaf"] > 64
        ref = g0.loglik(THETAS)
        for _ in range(4):  # first run direct, second captured, then replayed
            assert np.array_equal(g1.loglik(THETAS), ref)
        # device entry point with alternating buffers
        th = [torch.tensor(THETAS[k:k + 1], dtype=torch.float64, device="cuda") for k in range(3)]
        out = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in range(3)]
        for _ in range(3):
            for k in range(3):
                g1.loglik_device(th[k].data_ptr(), 1, out[k].data_ptr(), 0, 0)
        torch.cuda.synchronize()
        assert np.array_equal(np.array([o.item() for o in out]), ref)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_launch_configurations_agree_bit_for_bit(precision):
    # leaves of every bucket (<=32, <=40, <=48, <=64) and larger ones
    rng = np.random.default_rng(31)
    x, y, z = synth.uniform(6000, 24)
    cx = 0.25 + 0.01 * rng.standard_normal(500)
    cy = 0.6 + 0.01 * rng.standard_normal(500)
    x, y, z = np.concatenate([x, cx]), np.concatenate([y, cy]), np.concatenate([z, rng.standard_normal(500)])
    with mra.MRA(x, y, z, 4, 4, 16, precision=precision) as g:
        s = g.stats()
        assert s["max_leaf"] > 64
        ref = g.loglik(THETAS)
        # 16 rows: the streaming kernel of deep trees (ancestor blocks staged two
        # at a time; stages do not apply)
        rows = (16, 32, 64) if precision == "mixed" else (16, 32)
        for r in rows:
            for stages in ((1,) if r == 16 else (1, 2)):
                for bset in (0, 1):
                    for conc in (True, False):
                        for queue in (False, True):
                            g.set_launch(r, stages, bset, conc, leaf_queue=queue)
                            assert np.array_equal(g.loglik(THETAS), ref), (r, stages, bset, conc, queue)
                # the regions' short tails in chunks of half the rows (default) or in full chunks
                if r != 16:
                    g.set_launch(r, 0, 0, True, leafbasis_whole_chunks=True)
                    assert np.array_equal(g.loglik(THETAS), ref), (r, "whole chunks")
        # the prior's ancestor blocks in one buffer, in two, two blocks at a time, or by occupancy
        for ps in (1, 2, 3, 0):
            g.set_launch(prior_stages=ps)
            assert np.array_equal(g.loglik(THETAS), ref), ps
        with pytest.raises(mra.MRAError):
            g.set_launch(prior_stages=4)
        rep = g.autotune(THETAS[0], reps=2)
        assert rep["tried"] >= 2 and rep["ms_best"] <= rep["ms_default"]
        assert np.array_equal(g.loglik(THETAS), ref)
        with pytest.raises(mra.MRAError):
            g.set_launch(48, 1, 0, True)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_leaf_buckets_and_leafbasis_tails_r32_bit_for_bit(precision):
    # r = 32: leaves of about 36 observations fill the <=32, <=40, <=48 and
    # <=64 buckets (the 40 cap has a kernel of its own at this padding), and
    # level-3 regions of about 144 rows end in tails of at most half a chunk.
    # Every arrangement computes the same terms in the same order.
    x, y, z = synth.uniform(2300, 8)
    ref, st = oracle.loglik(x, y, z, 4, 4, 32, THETAS)
    assert st == 0
    with mra.MRA(x, y, z, 4, 4, 32, precision=precision) as g:
        n = g.stats()["n_used"]
        sizes = np.diff(g.tree()["leaf_off"])
        assert all(np.any((sizes > lo) & (sizes <= hi)) for lo, hi in ((0, 32), (32, 40), (40, 48), (48, 64)))
        base = g.loglik(THETAS)
        tol = 1e-10 if precision == "fp64" else 1e-6
        assert np.all(np.abs(base - ref) / n <= tol)
        rows = (32, 64) if precision == "mixed" else (32,)
        for r in rows:
            for whole in (False, True):
                for bset in (0, 1):
                    for conc in (True, False):
                        for queue in (False, True):
                            g.set_launch(r, 1, bset, conc, leaf_queue=queue, leafbasis_whole_chunks=whole)
                            assert np.array_equal(g.loglik(THETAS), base), (r, whole, bset, conc, queue)


@pytest.mark.parametrize("n,M,r,seed", [(20000, 14, 16, 41), (30000, 18, 9, 42)])
def test_parity_deep_binary_trees(n, M, r, seed):
    # J = 2 trees as deep as the paper's own runs (M up to 18), at r <= 16: FP64
    # at 1e-10 and the mixed mode at 1e-6.  The fast mixed mode (FP32 remainder
    # recursions) loses accuracy with depth at long range (M = 14, beta = 0.3:
    # |dl|/n ~ 2e-5); it is measured here and bounded loosely
    x, y, z = synth.uniform(n, seed, exact=False)
    _parity(x, y, z, M, 2, r, thetas=THETAS[:2])
    ref, _ = oracle.loglik(x, y, z, M, 2, r, THETAS[:2])
    with mra.MRA(x, y, z, M, 2, r, precision="mixed_fast") as g:
        err = np.abs(g.loglik(THETAS[:2]) - ref) / g.stats()["n_used"]
    print("deep tree M=%d mixed_fast |dl|/n:" % M, err)
    assert np.all(err <= 1e-4)


def test_fast_mixed_mode_on_small_trees():
    x, y, z = synth.uniform(3000, 25)
    _parity(x, y, z, 5, 4, 32, precisions=("mixed_fast",))


# The leaf Gram on the tensor cores (tcgen05 BF16 MMAs of exact fixed-grid slices;
# mra_tune_t.gram_tensor_cores = 1): the same likelihood as the CUDA-core Gram up to
# its last bits, held to the mixed tolerance against the oracle.  The trees cover
# Gram widths from 16 to 272 columns (one to three row chunks of the tile list,
# pieces narrower than the 64-column tile), empty subtrees, and a region of more
# than 320 observations (several exact groups added in FP32).
@pytest.mark.parametrize("n,M,J,r,seed", [
    (600, 2, 4, 16, 2),
    (3000, 4, 2, 30, 4),
    (3000, 5, 4, 32, 5),
    (4000, 6, 2, 16, 6),
    (20000, 14, 2, 16, 41),
    (30000, 18, 2, 9, 42),
])
def test_tensor_core_gram_parity(n, M, J, r, seed):
    x, y, z = synth.uniform(n, seed, exact=n <= 6000)
    th = THETAS[:2]
    ref, st = oracle.loglik(x, y, z, M, J, r, th)
    assert st == 0
    with mra.MRA(x, y, z, M, J, r, precision="mixed") as g:
        nu = g.stats()["n_used"]
        cuda_core = g.loglik(th)
        g.set_launch(gram_tensor_cores=True)
        assert g.autotune(th[0], reps=1)["gram_tensor_cores"] == 1
        tensor = g.loglik(th)
        again = g.loglik(th)
    assert np.array_equal(tensor, again)
    assert not np.array_equal(tensor, cuda_core)
    err = np.abs(tensor - ref) / nu
    print("tensor-core Gram M=%d |dl|/n:" % M, err, "CUDA-core:", np.abs(cuda_core - ref) / nu)
    assert np.all(err <= TOLMIX), err


def test_tensor_core_gram_ragged_and_grid_workload():
    # a 400-point cluster: a level-(M-1) region of more than 320 rows (several groups)
    x, y, z = synth.uniform(3000, 11)
    rng = np.random.default_rng(5)
    x = np.concatenate([x, 0.8 + 0.01 * rng.standard_normal(400)])
    y = np.concatenate([y, 0.8 + 0.01 * rng.standard_normal(400)])
    z = np.concatenate([z, rng.standard_normal(400)])
    d = synth.grid()
    for (xx, yy, zz, M, J, r, th) in [(x, y, z, 4, 4, 16, THETAS),
                                      (d["x"], d["y"], d["z"], d["M"], d["J"], d["r"],
                                       np.array([[1.0, 0.05, 0.01], [1.3, 0.08, 0.02]]))]:
        ref, st = oracle.loglik(xx, yy, zz, M, J, r, th)
        assert st == 0
        with mra.MRA(xx, yy, zz, M, J, r, precision="mixed") as g:
            nu = g.stats()["n_used"]
            g.set_launch(gram_tensor_cores=True)
            got = g.loglik(th)
        err = np.abs(got - ref) / nu
        print("tensor-core Gram n=%d |dl|/n:" % nu, err)
        assert np.all(err <= TOLMIX), err


# The leaf basis with its remainder products on the tensor cores (exact BF16
# slices, MRA_MIXED): trees with (M - 2) x padded r_hat <= 192, padding 16 and
# 32, J = 2 and 4, regions of more than 128 rows (several CTAs), r = 49 on two
# device levels per level, and the gridded workload at full size.
@pytest.mark.parametrize("n,M,J,r,seed", [
    (600, 2, 4, 16, 2),      # one level: no products on the tensor cores
    (3000, 4, 2, 30, 4),
    (3000, 5, 4, 32, 5),
    (4000, 6, 2, 16, 6),
    (20000, 12, 2, 16, 41),  # (M - 2) 16 = 160; a GP field (the swaths generator) at 20,000 points
    (3000, 4, 2, 49, 51),    # 7 device levels, r_hat 25 + 24 (padded 32)
])
def test_tensor_core_leafbasis_parity(n, M, J, r, seed):
    if n <= 6000:
        x, y, z = synth.uniform(n, seed)
    else:
        d = synth.swaths(seed=seed, n=n, grid_n=512)
        x, y, z = d["x"], d["y"], d["z"]
    th = THETAS[:2]
    ref, st = oracle.loglik(x, y, z, M, J, r, th)
    assert st == 0
    with mra.MRA(x, y, z, M, J, r, precision="mixed") as g:
        nu = g.stats()["n_used"]
        cuda_core = g.loglik(th)
        g.set_launch(leafbasis_tensor_cores=True)
        assert g.autotune(th[0], reps=1)["leafbasis_tensor_cores"] == 1
        tensor = g.loglik(th)
        again = g.loglik(th)
        g.set_launch(leafbasis_tensor_cores=False)
        assert np.array_equal(g.loglik(th), cuda_core)
    assert np.array_equal(tensor, again)
    err = np.abs(tensor - ref) / nu
    between = np.abs(tensor - cuda_core) / nu
    print("tensor-core leaf basis M=%d r=%d |dl|/n:" % (M, r), err, "CUDA-core:", np.abs(cuda_core - ref) / nu,
          "between:", between)
    assert np.all(err <= TOLMIX), err
    assert np.all(between <= 1e-7), between


def test_tensor_core_leafbasis_grid_workload_and_limits():
    d = synth.grid()
    th = np.array([[1.0, 0.05, 0.01], [1.3, 0.08, 0.02], [2.0, 0.2, 0.005]])
    ref, st = oracle.loglik(d["x"], d["y"], d["z"], d["M"], d["J"], d["r"], th)
    assert st == 0
    with mra.MRA(d["x"], d["y"], d["z"], d["M"], d["J"], d["r"], precision="mixed") as g:
        nu = g.stats()["n_used"]
        cuda_core = g.loglik(th)
        g.set_launch(leafbasis_tensor_cores=True)
        got = g.loglik(th)
        # the fast mode keeps the CUDA-core kernel (FP32 remainder products)
        g.set_precision("mixed_fast")
        fast = g.loglik(th)
        g.set_launch(leafbasis_tensor_cores=False)
        assert np.array_equal(g.loglik(th), fast)
    err = np.abs(got - ref) / nu
    print("tensor-core leaf basis, grid |dl|/n:", err, "CUDA-core:", np.abs(cuda_core - ref) / nu)
    assert np.all(err <= TOLMIX), err
    # beyond the exactness bound: (M - 2) x 32 > 192
    x, y, z = synth.uniform(3000, 9)
    with mra.MRA(x, y, z, 9, 2, 30, precision="mixed") as g:
        with pytest.raises(mra.MRAError) as e:
            g.set_launch(leafbasis_tensor_cores=True)
        assert e.value.status == mra.EINVAL
