"""The allocation-free entry point (mra_dense_loglik_noalloc) against the
library's regular path on the same single-region problem.

Some callers cannot let a library allocate device memory (a CUDA graph being
captured, a serving loop whose memory is reserved up front, a runtime that owns
every allocation); this entry point keeps its working memory in a fixed array
inside the library.  This file is collected last on purpose.
"""
import math

import numpy as np
import pytest

from paper_1905_00141_gb300 import build as mbuild
from paper_1905_00141_gb300 import mra, synth


def test_noalloc_rejects_oversize_without_a_gpu():
    mbuild.build()
    n = mra.NOALLOC_MAX_N + 1
    with pytest.raises(mra.MRAError) as e:
        mra.dense_loglik_noalloc(1, 1, 1, n, 1, 1)
    assert e.value.status == mra.EINVAL and "n must lie in [1, 1024]" in str(e.value)
    with pytest.raises(mra.MRAError) as e:
        mra.dense_loglik_noalloc(1, 1, 1, 0, 1, 1)
    assert e.value.status == mra.EINVAL


def _call(torch, x, y, z, theta, with_status=True):
    """One call through the C ABI on the current stream; (loglik, status)."""
    dev = torch.device("cuda")
    xd = torch.tensor(np.asarray(x, dtype=np.float64), device=dev)
    yd = torch.tensor(np.asarray(y, dtype=np.float64), device=dev)
    zd = torch.tensor(np.asarray(z, dtype=np.float64), device=dev)
    th = torch.tensor(np.asarray(theta, dtype=np.float64), device=dev)
    out = torch.full((1,), 123.0, dtype=torch.float64, device=dev)
    st = torch.full((1,), -1, dtype=torch.int32, device=dev)
    mra.dense_loglik_noalloc(xd.data_ptr(), yd.data_ptr(), zd.data_ptr(), len(x), th.data_ptr(), out.data_ptr(),
                             st.data_ptr() if with_status else 0, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return float(out.item()), int(st.item())


@pytest.mark.gpu
def test_noalloc_matches_regular_entry_point_twice():
    import torch
    mbuild.build()
    n = 400
    x, y, z = synth.uniform(n, 77)
    thetas = np.array([[1.0, 0.1, 0.05], [2.2, 0.25, 0.02]])
    with mra.MRA(x, y, z, 1, 4, 16, precision="fp64") as g:
        assert g.stats()["n_used"] == n
        ref = g.loglik(thetas)
    for k in range(2):  # two calls in a row share the fixed array
        got, st = _call(torch, x, y, z, thetas[k])
        assert st == mra.OK
        assert abs(got - ref[k]) / n <= 1e-10, (got, ref[k])


@pytest.mark.gpu
def test_noalloc_edge_sizes_and_failures():
    import torch
    mbuild.build()
    # n = 1: log N(z; 0, sigma2 + tau2) in closed form
    th = np.array([1.7, 0.2, 0.3])
    got, st = _call(torch, [0.3], [0.6], [0.8], th)
    v = th[0] + th[2]
    want = -0.5 * (math.log(v) + 0.8 * 0.8 / v + math.log(2.0 * math.pi))
    assert st == mra.OK and abs(got - want) <= 1e-13 * abs(want)
    # n = 1024, the whole fixed array, against the regular path with M = 1
    n = mra.NOALLOC_MAX_N
    x, y, z = synth.uniform(n, 78, exact=False)
    th = np.array([1.1, 0.07, 0.03])
    with mra.MRA(x, y, z, 1, 4, 16, precision="fp64") as g:
        assert g.stats()["n_used"] == n
        ref = g.loglik(th)[0]
    got, st = _call(torch, x, y, z, th)
    assert st == mra.OK and abs(got - ref) / n <= 1e-10, (got, ref)
    # without a status pointer the loglik is still written
    got2, _ = _call(torch, x, y, z, th, with_status=False)
    assert got2 == got
    # an invalid theta: NaN and EINVAL
    got, st = _call(torch, x[:50], y[:50], z[:50], [1.0, -0.1, 0.05])
    assert math.isnan(got) and st == mra.EINVAL
    # two observations at one location with a nugget far below the sill: the
    # covariance is singular to working precision, NaN and ENOTPD
    got, st = _call(torch, [0.2, 0.2, 0.7], [0.4, 0.4, 0.1], [0.1, -0.3, 0.5], [1.0, 0.1, 1e-15])
    assert math.isnan(got) and st == mra.ENOTPD
    # and the array is in a good state for the next call
    got, st = _call(torch, x, y, z, th)
    assert st == mra.OK and abs(got - ref) / n <= 1e-10
