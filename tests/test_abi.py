"""Host-side checks of libmra without a GPU: the library loads, exports every
entry point include/mra.h declares, and its host partition (Sec. 1.2) equals
the oracle's bit for bit."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_1905_00141_gb300 import build as mbuild
from paper_1905_00141_gb300 import mra, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    mbuild.build()


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(mra_\w+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L = mra.lib()
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n
    assert set(mra.EXPORTED) <= set(names)
    from paper_1905_00141_gb300 import mlp
    assert set(mlp.EXPORTED) <= set(names)


def _same_tree(x, y, z, M, J, r, offset=np.e / 100, dedup=False):
    o = oracle.Tree(x, y, z, M, J, r, offset, dedup)
    g = mra.MRA(x, y, z, M, J, r, offset=offset, dedup=dedup, device=-1)
    eo, eg = o.export(), g.tree()
    s = g.stats()
    assert (s["n_used"], s["n_nan"], s["n_dup"], s["n_knot"]) == (o.n_used, o.n_nan, o.n_dup, o.n_knot)
    assert s["r_hat"] == o.rhat and s["n_regions"] == o.nreg and s["n_leaves"] == o.nleaf
    assert np.array_equal(eo["bounds"], eg["bounds"])
    assert np.array_equal(eo["kx"], eg["kx"]) and np.array_equal(eo["ky"], eg["ky"])
    assert np.array_equal(eo["leaf_off"], eg["leaf_off"])
    assert np.array_equal(eo["perm"], eg["perm"])
    g.close()
    o.close()


@pytest.mark.parametrize("M,J,r", [(1, 4, 16), (3, 4, 16), (5, 2, 9), (4, 4, 32), (6, 2, 30), (3, 4, 2),
                                   (6, 2, 49), (3, 4, 64)])
def test_host_partition_matches_oracle(M, J, r):
    x, y, z = synth.uniform(3000, 100 + M * 10 + J, exact=False)
    x = x * 2.3 - 0.4
    _same_tree(x, y, z, M, J, r)


@pytest.mark.parametrize("M,J,r,levels", [(6, 2, 30, 6), (6, 2, 49, 11), (14, 2, 49, 27), (3, 4, 64, 5),
                                          (1, 4, 49, 1)])
def test_device_levels_of_wide_regions(M, J, r, levels):
    """r_hat > 32: every non-leaf level runs as two device levels (Sec. 1.1
    recursion entered in two halves of the knots); the partition the user sees
    (stats, export) stays the paper's."""
    x, y, z = synth.uniform(2000, 5, exact=False)
    g = mra.MRA(x, y, z, M, J, r, device=-1)
    s = g.stats()
    assert s["M"] == M and s["device_levels"] == levels
    assert s["n_regions"] == sum(J ** m for m in range(M))
    g.close()


def test_rhat_above_64_is_refused():
    x, y, z = synth.uniform(500, 6, exact=False)
    with pytest.raises(mra.MRAError) as e:
        mra.MRA(x, y, z, 3, 4, 81, device=-1)  # r_hat = 9 x 9
    assert e.value.status == mra.EINVAL and "64" in str(e.value)
    with pytest.raises(mra.MRAError) as e:
        mra.MRA(x, y, z, 19, 2, 49, device=-1)
    assert e.value.status == mra.EINVAL and "device levels" in str(e.value)


def test_host_partition_grid_workload():
    d = synth.grid()
    _same_tree(d["x"], d["y"], d["z"], d["M"], d["J"], d["r"])


def test_host_partition_eliminations():
    x, y, z = synth.uniform(500, 7, exact=False)
    kx, ky = oracle.place_knots(x.min(), x.max() + 0.01 * (x.max() - x.min()),
                                y.min(), y.max() + 0.01 * (y.max() - y.min()), 16, np.e / 100)
    x = np.concatenate([x, x[:20], kx[:3]])
    y = np.concatenate([y, y[:20], ky[:3]])
    z = np.concatenate([z, z[:20], [1.0, 2.0, 3.0]])
    z[[3, 9, 250]] = np.nan
    for dedup in (False, True):
        _same_tree(x, y, z, 3, 4, 16, dedup=dedup)
    _same_tree(x, y, z, 4, 2, 16, offset=0.1, dedup=True)


def test_build_errors_and_messages():
    x, y, z = synth.uniform(100, 3, exact=False)
    for args, st in [((3, 3, 16), mra.EINVAL), ((0, 4, 16), mra.EINVAL), ((3, 4, 0), mra.EINVAL)]:
        with pytest.raises(mra.MRAError) as e:
            mra.MRA(x, y, z, *args, device=-1)
        assert e.value.status == st and "invalid" in str(e.value)
    with pytest.raises(mra.MRAError) as e:
        mra.MRA(x, y, np.full(100, np.nan), 3, 4, 16, device=-1)
    assert e.value.status == mra.EEMPTY
    with pytest.raises(mra.MRAError) as e:
        mra.MRA(x[:0], y[:0], z[:0], 3, 4, 16, device=-1)
    assert e.value.status == mra.EEMPTY
    with pytest.raises(mra.MRAError) as e:
        mra.MRA(np.full(5, 0.5), np.arange(5.0), np.ones(5), 2, 4, 4, device=-1)
    assert e.value.status == mra.EINVAL and "degenerate" in str(e.value)
    xb = x.copy()
    xb[4] = np.inf
    with pytest.raises(mra.MRAError):
        mra.MRA(xb, y, z, 3, 4, 16, device=-1)
    with pytest.raises(mra.MRAError):
        mra.MRA(x, y, z, 3, 4, 16, offset=0.5, device=-1)


def test_host_only_context_refuses_likelihood():
    x, y, z = synth.uniform(100, 3, exact=False)
    g = mra.MRA(x, y, z, 3, 4, 16, device=-1)
    with pytest.raises(mra.MRAError) as e:
        g.loglik([1.0, 0.1, 0.05])
    assert e.value.status == mra.EINVAL and "without a device" in str(e.value)


def test_stats_work_counts():
    d = synth.grid()
    g = mra.MRA(d["x"], d["y"], d["z"], d["M"], d["J"], d["r"], device=-1)
    s = g.stats()
    assert s["r_hat"] == 30 and s["n_leaves"] == 4 ** 6 and s["n_used"] == 131072
    assert 5e9 < s["flops_per_theta"] < 5e10
    assert s["cov_evals_per_theta"] > 131072 * 6 * 30


def test_host_only_context_refuses_prediction():
    x, y, z = synth.uniform(100, 4, exact=False)
    g = mra.MRA(x, y, z, 3, 4, 16, device=-1)
    with pytest.raises(mra.MRAError) as e:
        g.predict([1.0, 0.1, 0.05], [0.5], [0.5])
    assert e.value.status == mra.EINVAL and "without a device" in str(e.value)
    g.close()


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without the compiled library the binding raises."""
    monkeypatch.setattr(mra, "_lib", None)
    monkeypatch.setattr(mra, "LIB_PATH", str(tmp_path / "libmra.so"))
    with pytest.raises(RuntimeError, match="not built"):
        mra.lib()
