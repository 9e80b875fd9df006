"""Stored FP64 CPU oracle values of the full-size workloads
(tests/golden/full_size_oracle.txt, written by
tests/golden/make_full_size_oracle.py from oracle/ and the seeded generators
only), with the fingerprint of the data each value belongs to."""
import os

import numpy as np

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full_size_oracle.txt")


def golden(name):
    """Stored rows of one workload: (theta, loglik, n_used, fingerprint)."""
    rows = []
    if not os.path.exists(GOLD):
        return rows
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if f[0] != name:
            continue
        rows.append((np.array([float(v) for v in f[1:4]]), float(f[4]), int(f[5]),
                     (int(f[6]),) + tuple(float(v) for v in f[7:11])))
    return rows


def fingerprint_matches(d, fp):
    n, sx, sy, sz, saz = fp
    if len(d["x"]) != n:
        return False
    close = lambda a, b: abs(a - b) <= 1e-9 * max(1.0, abs(b))  # noqa: E731
    return (close(float(np.sum(d["x"])), sx) and close(float(np.sum(d["y"])), sy) and
            close(float(np.sum(np.abs(d["z"]))), saz) and abs(float(np.sum(d["z"])) - sz) <= 1e-9 * saz)
