"""Write full_size_oracle.txt: the FP64 CPU oracle's log-likelihood of the two
largest synthetic workloads at the theta the GPU tests check them on.

The values come from oracle/ alone (the C recursion of Sec. 1.1 on the tree of
Sec. 1.2, all host threads) on the seeded inputs of
paper_1905_00141_gb300/synth.py; nothing here touches the CUDA library.  Each
line also records a fingerprint of the generated data (n, sums of the
coordinates and of the values) so that a test can tell whether its own draw of
the same workload is the one the stored value belongs to.

    python tests/golden/make_full_size_oracle.py [clustered] [massive] [swaths]

The clustered workload (n = 2,097,152, M = 9) takes about 80 s per theta on 8
cores; the 47M-observation tree (M = 12) about 10 minutes for its one theta;
the swaths workload (n = 2,439,827, J = 2, M = 14, r = 49) is checked at two
theta; the modis18 workload (n = 4,194,304 on the J = 2, M = 18, r = 49 tree)
at its generating theta.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1905_00141_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "full_size_oracle.txt")

# theta rows checked per workload: the clustered ones are entries 0, 21, 42 and
# 60 of the 4x4x4 log grid (60 is the corner sigma2 = 2, beta = 0.2,
# tau2 = 0.005); the 47M tree is checked at its generating theta; the swaths
# tree at its generating theta and at a longer range with a smaller nugget
PICKS = {"clustered": [0, 21, 42, 60], "massive": None, "swaths": None, "modis18": None}
SWATHS_EXTRA = [1.5, 0.15, 0.005]


def fingerprint(d):
    return (len(d["x"]), float(np.sum(d["x"])), float(np.sum(d["y"])), float(np.sum(d["z"])),
            float(np.sum(np.abs(d["z"]))))


def thetas_of(name, d):
    if name == "clustered":
        return synth.theta_grid_4x4x4()[PICKS[name]]
    if name == "swaths":
        return np.vstack([np.atleast_2d(d["theta"])[:1], [SWATHS_EXTRA]])
    return np.atleast_2d(d["theta"])[:1]


def main(names):
    oracle.build()
    rows = {}
    if os.path.exists(OUT):
        for line in open(OUT):
            if line.strip() and not line.startswith("#"):
                rows[tuple(line.split()[:4])] = line.rstrip("\n")
    for name in names:
        d = synth.make(name)
        fp = fingerprint(d)
        t = oracle.Tree(d["x"], d["y"], d["z"], d["M"], d["J"], d["r"])
        for th in thetas_of(name, d):
            t0 = time.time()
            ll, st = t.loglik(th)
            dt = time.time() - t0
            assert st == 0, (name, th, st)
            key = (name, "%.17g" % th[0], "%.17g" % th[1], "%.17g" % th[2])
            rows[key] = " ".join(list(key) + ["%.17g" % ll[0], "%d" % t.n_used] + ["%.17g" % v for v in fp] +
                                 ["%.1f" % dt, "%d" % oracle.max_threads()])
            print(rows[key], flush=True)
        t.close()
    with open(OUT, "w") as fh:
        fh.write("# FP64 CPU oracle (oracle/mra_oracle.c) log-likelihood of the full-size synthetic workloads,\n"
                 "# written by tests/golden/make_full_size_oracle.py from oracle/ and synth.py only.\n"
                 "# workload sigma2 beta tau2 loglik n_used | fingerprint: n sum(x) sum(y) sum(z) sum(|z|)"
                 " | seconds threads\n")
        for key in sorted(rows):
            fh.write(rows[key] + "\n")


if __name__ == "__main__":
    main(sys.argv[1:] or ["clustered", "massive"])
