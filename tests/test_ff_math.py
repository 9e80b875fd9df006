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
    } else if (mode == 2) {
        // FP32 coordinates (the overload the remainder recursions use)
        double s2, beta;
        float ax, ay, bx, by;
        while (scanf("%lf %lf %f %f %f %f", &s2, &beta, &ax, &ay, &bx, &by) == 6) {
            mra::ff c = mra::ff_cov_exp(mra::ff_from_double(s2), mra::ff_from_double(1.0 / beta), ax, ay, bx, by);
            long double dx = (long double)ax - bx, dy = (long double)ay - by;
            long double ref = (long double)s2 * expl(-sqrtl(dx * dx + dy * dy) / (long double)beta);
            printf("%.17g %.21Lg\n", mra::ff_to_double(c), ref);
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
    # the covariance enters sums of products carried to ~1e-11 sigma2 (grid
    # accumulation); the float-pair evaluation is held to 2e-13, fifty
    # times below that (sloppy float-pair adds for the coordinate differences
    # and the squared distance, whose terms do not cancel)
    assert (np.abs(got - ref) / s2).max() < 2e-13
    big = ref > 1e-3 * s2
    assert (np.abs(got - ref) / ref)[big].max() < 2e-13
    assert got[-1] == 1.3 or abs(got[-1] - 1.3) < 1e-15


def test_cov_exp_float_coordinates(prog):
    """The FP32-coordinate overload: exact coordinate differences, the same
    2e-13 bound (coordinates rounded to FP32 first, on both sides)."""
    rng = np.random.default_rng(3)
    rows = []
    for _ in range(4000):
        s2 = rng.uniform(0.1, 5)
        beta = 10 ** rng.uniform(-2.5, 1)
        a = rng.uniform(0.0, 0.05, 2).astype(np.float32)
        b = (a + rng.normal(0, 10 ** rng.uniform(-4, -1), 2)).astype(np.float32)
        rows.append("%.17g %.17g %.9g %.9g %.9g %.9g" % (s2, beta, a[0], a[1], b[0], b[1]))
    got, ref = _run(prog, "2\n" + "\n".join(rows))
    s2 = np.array([float(r.split()[0]) for r in rows])
    assert (np.abs(got - ref) / s2).max() < 2e-13


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


PROG3 = r"""
#include <cmath>
#include <cstdio>
#include "ff_math.h"
// mode 0: K, bound, then K pairs (a, b) of floats -> grid sum and the sum in long double
// mode 1: K, bound, then K quadruples (a.hi, a.lo, b.hi, b.lo) -> float-pair operands
// mode 2: a.hi a.lo b.hi b.lo -> ff_sub_sloppy(a, b) and the exact difference
int main() {
    int mode;
    if (scanf("%d", &mode) != 1) return 1;
    if (mode == 2) {
        float ah, al, bh, bl;
        while (scanf("%f %f %f %f", &ah, &al, &bh, &bl) == 4) {
            mra::ff d = mra::ff_sub_sloppy(mra::ff{ah, al}, mra::ff{bh, bl});
            long double ref = ((long double)ah + al) - ((long double)bh + bl);
            printf("%.21Lg %.21Lg\n", (long double)d.hi + d.lo, ref);
        }
        return 0;
    }
    int K;
    double bound;
    while (scanf("%d %lf", &K, &bound) == 2) {
        const float c = mra::grid_constant(bound);
        mra::grid_acc g;
        mra::grid_init(g, c);
        long double ref = 0.0L;
        for (int t = 0; t < K; t++) {
            if (mode == 0) {
                float a, b;
                if (scanf("%f %f", &a, &b) != 2) return 1;
                mra::grid_add(g, a, b);
                ref += (long double)a * b;
            } else {
                float ah, al, bh, bl;
                if (scanf("%f %f %f %f", &ah, &al, &bh, &bl) != 4) return 1;
                mra::grid_add(g, mra::ff{ah, al}, mra::ff{bh, bl});
                ref += ((long double)ah + al) * ((long double)bh + bl);
            }
        }
        const mra::ff v = mra::grid_value(g, c);
        printf("%.21Lg %.21Lg\n", (long double)v.hi + v.lo, ref);
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def prog3(tmp_path_factory):
    d = tmp_path_factory.mktemp("ff3")
    src = d / "t3.cpp"
    src.write_text(PROG3)
    exe = d / "t3"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, str(src), "-o", str(exe)],
                   check=True)
    return str(exe)


def _bounded_rows(rng, K, bound):
    """Two float32 vectors with |a| |b| <= bound (Cauchy-Schwarz bound on
    sum |a_t b_t|), scaled like rows of whitened basis functions."""
    a = rng.standard_normal(K)
    b = rng.standard_normal(K)
    a *= np.sqrt(bound) * rng.uniform(0.3, 0.999) / np.linalg.norm(a)
    b *= np.sqrt(bound) * rng.uniform(0.3, 0.999) / np.linalg.norm(b)
    return a.astype(np.float32), b.astype(np.float32)


def test_grid_accumulation_error(prog3):
    """Sums of products bounded by `bound` come out within 4e-11 * bound of
    the exact sum (long double: the products of floats are exact there), for
    bounds across many binades, lengths 1..600 and a sum that nearly cancels."""
    rng = np.random.default_rng(5)
    cases, lines = [], ["0"]
    for trial in range(400):
        bound = float(10 ** rng.uniform(-6, 6))
        K = int(rng.integers(1, 600))
        a, b = _bounded_rows(rng, K, bound)
        if trial % 4 == 0:  # nearly cancelling: b orthogonalised against a
            bb = b.astype(np.float64) - a * (a.astype(np.float64) @ b) / (a.astype(np.float64) @ a)
            b = bb.astype(np.float32)
        cases.append(bound)
        lines.append("%d %.17g" % (K, bound))
        lines.extend("%.9g %.9g" % (x, y) for x, y in zip(a, b))
    got, ref = _run(prog3, "\n".join(lines))
    err = np.abs(got - ref) / np.array(cases)
    assert np.max(err) < 4e-11


def test_grid_accumulation_float_pairs(prog3):
    """The float-pair form (leading products on the grid, cross terms in
    FP32) stays within float-pair accuracy of the exact sum of the pairs."""
    rng = np.random.default_rng(6)
    cases, lines = [], ["1"]
    for trial in range(200):
        bound = float(10 ** rng.uniform(-3, 3))
        K = int(rng.integers(1, 64))
        a, b = _bounded_rows(rng, K, 0.98 * bound)
        al = (a * rng.uniform(-2 ** -24, 2 ** -24, K)).astype(np.float32)
        bl = (b * rng.uniform(-2 ** -24, 2 ** -24, K)).astype(np.float32)
        cases.append(bound)
        lines.append("%d %.17g" % (K, bound))
        lines.extend("%.9g %.9g %.9g %.9g" % q for q in zip(a, al, b, bl))
    got, ref = _run(prog3, "\n".join(lines))
    assert np.max(np.abs(got - ref) / np.array(cases)) < 4e-11


def test_sloppy_subtraction(prog3):
    """ff_sub_sloppy: absolute error below 2^-44 (|a| + |b|), including
    differences that cancel to a few ulps of the leading floats."""
    rng = np.random.default_rng(7)
    n = 4000
    ah = (10 ** rng.uniform(-8, 8, n) * rng.choice([-1, 1], n)).astype(np.float32)
    bh = np.where(rng.random(n) < 0.5, ah * (1 + rng.uniform(-1e-6, 1e-6, n)),
                  10 ** rng.uniform(-8, 8, n)).astype(np.float32)
    al = (ah * rng.uniform(-2 ** -24, 2 ** -24, n)).astype(np.float32)
    bl = (bh * rng.uniform(-2 ** -24, 2 ** -24, n)).astype(np.float32)
    text = "2\n" + "\n".join("%.9g %.9g %.9g %.9g" % q for q in zip(ah, al, bh, bl))
    got, ref = _run(prog3, text)
    scale = np.abs(ah.astype(np.float64)) + np.abs(bh.astype(np.float64))
    assert np.max(np.abs(got - ref) / scale) < 2.0 ** -44
