"""The double-float exponential and covariance of ff_math.h (used by the mixed
mode for the leaf covariance) against long-double references, compiled for the
CPU with g++ from the same header."""
import os
import subprocess

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1905_00141_gb300", "csrc")

PROG = r"""
#include <cmath>
#include <cstdio>
#include "ff_math.h"
int main() {
    double x;
    int mode;
    if (scanf("%d", &mode) != 1) return 1;
    if (mode == 0) {
        while (scanf("%lf", &x) == 1) {
            mra::ff r = mra::ff_exp_neg(mra::ff_from_double(x));
            long double ref = expl(-(long double)x);
            printf("%.17g %.21Lg\n", mra::ff_to_double(r), ref);
        }
    } else {
        double s2, beta, ax, ay, bx, by;
        while (scanf("%lf %lf %lf %lf %lf %lf", &s2, &beta, &ax, &ay, &bx, &by) == 6) {
            mra::ff c = mra::ff_cov_exp(mra::ff_from_double(s2), mra::ff_from_double(1.0 / beta),
                                        mra::ff_from_double(ax), mra::ff_from_double(ay),
                                        mra::ff_from_double(bx), mra::ff_from_double(by));
            long double dx = (long double)ax - bx, dy = (long double)ay - by;
            long double ref = (long double)s2 * expl(-sqrtl(dx * dx + dy * dy) / (long double)beta);
            printf("%.17g %.21Lg\n", mra::ff_to_double(c), ref);
        }
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    d = tmp_path_factory.mktemp("ff")
    src = d / "t.cpp"
    src.write_text(PROG)
    exe = d / "t"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, str(src), "-o", str(exe)],
                   check=True)
    return str(exe)


def _run(exe, text):
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout
    a = np.array([[float(v) for v in line.split()] for line in out.strip().splitlines()])
    return a[:, 0], a[:, 1]


def test_exp_neg_relative_error(prog):
    rng = np.random.default_rng(0)
    x = np.concatenate([[0.0, 1e-12, 1e-7, 0.0054, 0.00542, 0.5, 1.0, np.log(2) / 64 * 37, 80.0],
                        rng.uniform(0, 1e-3, 2000), rng.uniform(0, 3, 4000), rng.uniform(0, 86, 4000)])
    got, ref = _run(prog, "0\n" + "\n".join("%.17g" % v for v in x))
    # the float-pair input holds x to ~48 bits, so the relative error grows
    # like x * 3.6e-15 (the conditioning of exp); the absolute error stays tiny
    mid = x <= 60
    rel = np.abs(got - ref) / ref
    assert np.all(rel[mid] <= 1.5e-14 * (1.0 + x[mid])), (rel[mid] / (1 + x[mid])).max()
    assert np.abs(got - ref).max() < 2e-14


def test_cov_exp_relative_error(prog):
    rng = np.random.default_rng(1)
    rows = []
    for _ in range(4000):
        s2 = rng.uniform(0.1, 5)
        beta = 10 ** rng.uniform(-2.5, 1)
        a = rng.uniform(0.0, 0.05, 2)  # coordinates local to a small region, as in the kernels
        b = a + rng.normal(0, 10 ** rng.uniform(-4, -1), 2)
        rows.append("%.17g %.17g %.17g %.17g %.17g %.17g" % (s2, beta, a[0], a[1], b[0], b[1]))
    rows.append("1.3 0.1 0.25 0.5 0.25 0.5")  # zero distance: exactly sigma2
    got, ref = _run(prog, "1\n" + "\n".join(rows))
    s2 = np.array([float(r.split()[0]) for r in rows])
    assert (np.abs(got - ref) / s2).max() < 2e-14
    big = ref > 1e-3 * s2
    assert (np.abs(got - ref) / ref)[big].max() < 5e-14
    assert got[-1] == 1.3 or abs(got[-1] - 1.3) < 1e-15


PROG2 = r"""
#include <cmath>
#include <cstdio>
#include "ff_math.h"
int main() {
    double x;
    while (scanf("%lf", &x) == 1) {
        mra::ff d = mra::ff_from_double(x);
        mra::ff r = mra::ff_rsqrt(d), q = mra::ff_rcp(d);
        printf("%.17g %.17g %.21Lg %.21Lg\n", mra::ff_to_double(r), mra::ff_to_double(q),
               1.0L / sqrtl((long double)x), 1.0L / (long double)x);
    }
    return 0;
}
"""


def test_rsqrt_and_reciprocal(tmp_path):
    src = tmp_path / "t2.cpp"
    src.write_text(PROG2)
    exe = tmp_path / "t2"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, str(src), "-o", str(exe)],
                   check=True)
    x = 10 ** np.random.default_rng(2).uniform(-12, 12, 5000)
    out = subprocess.run([str(exe)], input="\n".join("%.17g" % v for v in x), capture_output=True, text=True,
                         check=True).stdout
    a = np.array([[float(v) for v in line.split()] for line in out.strip().splitlines()])
    assert np.max(np.abs(a[:, 0] - a[:, 2]) / a[:, 2]) < 4e-14
    assert np.max(np.abs(a[:, 1] - a[:, 3]) / a[:, 3]) < 4e-14
