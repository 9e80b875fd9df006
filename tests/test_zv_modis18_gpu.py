"""The modis18 workload at full size: n = 4,194,304 observations in slanted
passes with gaps on the tree shape of the paper's large MODIS run (J = 2,
M = 18, r = 49 knots per region; 131,072 leaves of about 32 observations),
mixed precision, against the FP64 CPU oracle's stored value.

Every level of r = 49 runs as two device levels (35 in all).  At this depth
the prior stages its ancestor blocks in parts, the upward pass stages the
right-hand blocks of its solve, and the ATilde arrays of one theta (about
370 GB over the whole tree) do not fit one GPU, so the memory plan runs the
leaf Gram and the upward pass of the lower levels chunk by chunk of subtrees.
The oracle evaluates the paper's tree directly, all 49 knots of a region at
once; its value is stored in tests/golden/full_size_oracle.txt by
tests/golden/make_full_size_oracle.py (about half an hour on 8 host
threads, too long to recompute here)."""
import numpy as np
import pytest

from golden_values import fingerprint_matches, golden
from paper_1905_00141_gb300 import synth

pytestmark = pytest.mark.gpu

TOLMIX = 1e-6


@pytest.fixture(scope="module")
def modis18():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1905_00141_gb300 import build, mra
    build.build()
    d = synth.modis18()
    g = mra.MRA(d["x"], d["y"], d["z"], d["M"], d["J"], d["r"], precision="mixed")
    yield d, g, mra
    g.close()


def test_modis18_full_size_mixed_matches_oracle(modis18):
    d, g, _ = modis18
    s = g.stats()
    assert s["r_hat"] == 49 and s["device_levels"] == 35 and s["n_used"] == len(d["x"])
    assert s["n_regions"] == 2 ** 18 - 1
    rows = golden("modis18")
    assert rows, "no stored oracle value for modis18"
    assert all(fingerprint_matches(d, r[3]) for r in rows), "the stored value belongs to another draw of the data"
    th = np.stack([r[0] for r in rows])
    ref = np.array([r[1] for r in rows])
    ll = g.loglik(th)
    err = np.abs(ll - ref) / s["n_used"]
    print("modis18 mixed |dl|/n against the oracle: %s (subtree level %d, %d chunks)" %
          (err.tolist(), s["subtree_level"], s["subtree_chunks"]))
    assert np.all(err <= TOLMIX), err


def test_modis18_fp64_is_refused(modis18):
    _, g, mra = modis18
    with pytest.raises(mra.MRAError) as e:
        g.set_precision("fp64")
    assert e.value.status == mra.EINVAL
