"""The allocation-free entry point (mra_dense_loglik_noalloc) against the
library's regular path on the same single-region problem.

Some callers cannot let a library allocate device memory (a CUDA graph being
captured, a serving loop whose memory is reserved up front, a runtime that owns
every allocation); this entry point keeps its working memory in a fixed array
inside the library.  This file is collected last on purpose.
"""
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
    dev = torch.device("cuda")
    xd = torch.tensor(x, dtype=torch.float64, device=dev)
    yd = torch.tensor(y, dtype=torch.float64, device=dev)
    zd = torch.tensor(z, dtype=torch.float64, device=dev)
    for k in range(2):  # two calls in a row share the fixed array
        th = torch.tensor(thetas[k], dtype=torch.float64, device=dev)
        out = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
        st = torch.full((1,), -1, dtype=torch.int32, device=dev)
        mra.dense_loglik_noalloc(xd.data_ptr(), yd.data_ptr(), zd.data_ptr(), n, th.data_ptr(), out.data_ptr(),
                                 st.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert int(st.item()) == mra.OK
        assert abs(float(out.item()) - ref[k]) / n <= 1e-10, (out.item(), ref[k])
