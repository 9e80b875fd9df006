"""FP64 CPU oracle of the MRA Gaussian-process log-likelihood.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the library under
``paper_1905_00141_gb300`` never does, and this package never imports it.

Two independent references live here:

* ``mra_oracle.c`` (loaded through ctypes): the tree of Sec. 1.2 and the
  likelihood recursion derived from the remainder covariances of Sec. 1.1
  (prior W/K blocks, leaf posterior, Woodbury upward pass, root), plain FP64.
* ``dense.py``: a brute-force dense Sigma_MRA built pair by pair from the
  C_m recursion of Sec. 1.1, then the textbook Gaussian log-density, and
  kriging with it (posterior predictive mean and variance at new points).
  It has its own tree code and is only meant for tiny inputs.
* ``predict_by_loglik``: the posterior predictive at one point from three
  likelihood evaluations of the recursion oracle with the point added as an
  observation, l(S + {s*: z*}) - l(S) = log N(z*; mean, var + tau2): an
  independent route to the prediction at any data size.
* ``mlp.py``: the surrogate network (an addition to the paper's method: a
  3 -> 64 -> 64 -> 1 SiLU perceptron of loglik/n over log theta) in FP64
  numpy -- BF16 rounding of the parameters, forward pass, hand-derived
  gradient of the squared-error loss, and the Adam update.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mra_oracle.c")
_LIB = os.path.join(_HERE, "libmra_oracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ENOTPD, EEMPTY = 0, 1, 2, 3, 6


def build(force: bool = False) -> str:
    """Compile mra_oracle.c with gcc (FP contraction off, OpenMP on)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _bind(path):
    lib = ctypes.CDLL(path)
    D = ctypes.POINTER(ctypes.c_double)
    I64 = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_tree_new.restype = ctypes.c_void_p
    lib.oracle_tree_new.argtypes = [D, D, D, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int)]
    lib.oracle_tree_free.argtypes = [ctypes.c_void_p]
    lib.oracle_tree_counts.argtypes = [ctypes.c_void_p, I64]
    lib.oracle_tree_export.argtypes = [ctypes.c_void_p, D, D, I64, I64, D]
    lib.oracle_loglik.restype = ctypes.c_int
    lib.oracle_loglik.argtypes = [ctypes.c_void_p, D, ctypes.c_int, D, ctypes.c_int]
    lib.oracle_region_terms.restype = ctypes.c_int
    lib.oracle_region_terms.argtypes = [ctypes.c_void_p, D, D, D, D, D, ctypes.c_int]
    lib.oracle_place_knots.argtypes = [ctypes.c_double] * 4 + [ctypes.c_int, ctypes.c_double,
                                                               D, D, ctypes.POINTER(ctypes.c_int)]
    lib.oracle_max_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(_LIB)
    return _lib


def load_variant(path):
    """Bind another build of mra_oracle.c (used by the mutation test)."""
    return _bind(path)


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def place_knots(x0, x1, y0, y1, r, offset):
    """Knot grid of one region (Sec. 1.2, App. A): returns (kx, ky)."""
    lib = _load()
    cap = r + 8
    kx = np.zeros(cap)
    ky = np.zeros(cap)
    rh = ctypes.c_int(0)
    lib.oracle_place_knots(x0, x1, y0, y1, int(r), float(offset), _dp(kx), _dp(ky), ctypes.byref(rh))
    return kx[:rh.value].copy(), ky[:rh.value].copy()


class Tree:
    """Partition of Sec. 1.2 built by the C oracle (an opaque handle)."""

    def __init__(self, x, y, z, M, J, r, offset=np.e / 100.0, dedup=False, lib=None):
        lib = lib or _load()
        self._lib = lib
        self._x = np.ascontiguousarray(x, dtype=np.float64)
        self._y = np.ascontiguousarray(y, dtype=np.float64)
        self._z = np.ascontiguousarray(z, dtype=np.float64)
        n = self._x.shape[0]
        st = ctypes.c_int(0)
        h = lib.oracle_tree_new(_dp(self._x), _dp(self._y), _dp(self._z), n, int(M), int(J), int(r),
                                float(offset), int(bool(dedup)), ctypes.byref(st))
        self.status = st.value
        self._h = h
        self.M, self.J, self.r = int(M), int(J), int(r)
        if not h:
            raise OracleError(self.status)
        c = np.zeros(10, dtype=np.int64)
        lib.oracle_tree_counts(h, _ip(c))
        (self.n_in, self.n_used, self.n_nan, self.n_dup, self.n_knot, self.nreg, self.nleaf,
         self.rhat, self.nx, self.ny) = [int(v) for v in c]

    def close(self):
        if self._h:
            self._lib.oracle_tree_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def export(self):
        nk = (self.nreg - self.nleaf) * self.rhat
        kx = np.zeros(max(nk, 1))
        ky = np.zeros(max(nk, 1))
        lo = np.zeros(self.nleaf + 1, dtype=np.int64)
        perm = np.zeros(max(self.n_used, 1), dtype=np.int64)
        b = np.zeros(4 * self.nreg)
        self._lib.oracle_tree_export(self._h, _dp(kx), _dp(ky), _ip(lo), _ip(perm), _dp(b))
        return dict(kx=kx[:nk], ky=ky[:nk], leaf_off=lo, perm=perm[:self.n_used],
                    bounds=b.reshape(self.nreg, 4))

    def loglik(self, theta, nthreads: int = 0):
        """loglik at each row (sigma2, beta, tau2) of theta; NaN where it fails."""
        th = np.ascontiguousarray(np.atleast_2d(theta), dtype=np.float64)
        out = np.zeros(th.shape[0])
        st = self._lib.oracle_loglik(self._h, _dp(th), th.shape[0], _dp(out), int(nthreads))
        return out, int(st)

    def region_terms(self, theta, nthreads: int = 0):
        """Per-region (d_R, u_R, log|W^m_R|) at one theta, by global region id."""
        th = np.ascontiguousarray(theta, dtype=np.float64).reshape(3)
        d = np.zeros(self.nreg)
        u = np.zeros(self.nreg)
        lw = np.zeros(self.nreg)
        ll = np.zeros(1)
        st = self._lib.oracle_region_terms(self._h, _dp(th), _dp(d), _dp(u), _dp(lw), _dp(ll),
                                         int(nthreads))
        return dict(d=d, u=u, logdetW=lw, loglik=float(ll[0]), status=int(st))


class OracleError(RuntimeError):
    def __init__(self, status):
        super().__init__("oracle status %d" % status)
        self.status = status


def loglik(x, y, z, M, J, r, theta, offset=np.e / 100.0, dedup=False, nthreads: int = 0):
    t = Tree(x, y, z, M, J, r, offset, dedup)
    try:
        return t.loglik(theta, nthreads)
    finally:
        t.close()


def predict_by_loglik(x, y, z, M, J, r, theta, px, py, scale=1.0, nthreads: int = 0):
    """Posterior predictive mean and variance of the latent process at
    (px, py) through the Gaussian conditional density: with the point added
    as an observation of value t, D(t) = l(S + {s*: t}) - l(S) is
    -1/2 log(2 pi s) - (t - mean)^2 / (2 s), s = var + tau2, so three values
    t in {-h, 0, h} give s = -h^2 / (D(h) + D(-h) - 2 D(0)) and
    mean = s (D(h) - D(-h)) / (2 h).  The point must lie strictly inside the
    bounding box of the data (the tree stays the same) and off every knot."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    th = np.asarray(theta, dtype=np.float64).reshape(1, 3)
    if not (x.min() < px < x.max() and y.min() < py < y.max()):
        raise ValueError("the point must lie strictly inside the data's bounding box")
    base, st = loglik(x, y, z, M, J, r, th, nthreads=nthreads)
    if st != OK:
        raise OracleError(st)
    h = float(scale)
    D = []
    for t in (-h, 0.0, h):
        v, st = loglik(np.append(x, px), np.append(y, py), np.append(z, t), M, J, r, th, nthreads=nthreads)
        if st != OK:
            raise OracleError(st)
        D.append(float(v[0] - base[0]))
    s = -h * h / (D[2] + D[0] - 2.0 * D[1])
    mean = s * (D[2] - D[0]) / (2.0 * h)
    return mean, s - float(th[0, 2])
