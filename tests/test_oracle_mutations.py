"""The oracle pins are sensitive: each plausible mistake planted in a private
copy of mra_oracle.c (compiled here, on the CPU) makes at least one pin fail.

Pins used: the brute-force Sigma_MRA likelihood on small trees, and the
paper's toy knot example (Sec. 1.2).
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from oracle import dense
from paper_1905_00141_gb300 import synth

SRC = os.path.join(os.path.dirname(oracle.__file__), "mra_oracle.c")

MUTATIONS = {
    "schur_sign": ("At[a * E + b] = A[a * D + b] - s;", "At[a * E + b] = A[a * D + b] + s;"),
    "drop_prior_logdet": ("*d = ds + logdetT - self.logdetW;", "*d = ds + logdetT;"),
    "transposed_ancestor_block": ("s += Gk[i * R + a] * WkA[j * R + a];",
                                  "s += Gk[i * R + a] * WkA[a * R + j];"),
    "drop_nugget": ("V[a * p + a] += c->th.tau2;", "V[a * p + a] += 0.5 * c->th.tau2;"),
    "quadform_sign": ("*u = us - q;", "*u = us + q;"),
    "knot_spacing": ("(f + (double)p * (1.0 - 2.0 * f) / (double)(nx - 1))",
                     "(f + (double)p * (1.0 - f) / (double)(nx - 1))"),
    "wrong_omega_index": ("Z[a * nc + E] = w[E + a];", "Z[a * nc + E] = w[a];"),
    "skip_k_term": ("for (int k = 1; k < l; k++) {\n            const double *Gk",
                    "for (int k = 2; k < l; k++) {\n            const double *Gk"),
}


def _pins_pass(lib):
    kx, ky = np.zeros(40), np.zeros(40)
    import ctypes
    rh = ctypes.c_int(0)
    lib.oracle_place_knots(0.0, 1.0, 0.0, 1.0, 32, 0.1,
                           kx.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           ky.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(rh))
    xs = np.unique(np.round(kx[:rh.value], 12))
    if rh.value != 30 or not np.allclose(xs, [0.1, 0.26, 0.42, 0.58, 0.74, 0.9]):
        return False
    for (n, M, J, r, seed) in [(150, 3, 4, 9, 2), (200, 4, 2, 9, 5)]:
        x, y, z = synth.uniform(n, seed)
        th = (1.0, 0.1, 0.05)
        try:
            t = oracle.Tree(x, y, z, M, J, r, lib=lib)
        except oracle.OracleError:
            return False
        ll, st = t.loglik(th)
        t.close()
        ref = dense.loglik(x, y, z, M, J, r, th)
        if st != 0 or not abs(ll[0] - ref) <= 1e-10 * abs(ref):
            return False
    return True


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / ("libmut_%s.so" % name)
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so),
                    str(path), "-lm"], check=True)
    assert not _pins_pass(oracle.load_variant(str(so)))


def test_unmutated_copy_passes(tmp_path):
    so = tmp_path / "libclean.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so),
                    SRC, "-lm"], check=True)
    assert _pins_pass(oracle.load_variant(str(so)))
