"""Thin ctypes binding of libmra (include/mra.h).

Argument marshalling only: every step of the likelihood runs in the CUDA
kernels of libmra.so.  There is no CPU fallback; if the library is missing
the first use raises.  PyTorch (optional) only supplies device memory and
streams to :meth:`MRA.loglik_torch`.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmra.so")

OK, EINVAL, ENOMEM, ENOTPD, ECUDA, ETIMEDOUT, EEMPTY = 0, 1, 2, 3, 4, 5, 6
FP64, MIXED, MIXED_FAST = 0, 1, 2
_STATUS = {0: "MRA_OK", 1: "MRA_EINVAL", 2: "MRA_ENOMEM", 3: "MRA_ENOTPD", 4: "MRA_ECUDA",
           5: "MRA_ETIMEDOUT", 6: "MRA_EEMPTY"}

EXPORTED = ["mra_default_opts", "mra_build", "mra_loglik", "mra_loglik_device", "mra_set_precision",
            "mra_stats", "mra_tree_export", "mra_region_terms", "mra_profile", "mra_profile_read",
            "mra_dense_loglik_noalloc", "mra_autotune", "mra_set_launch", "mra_predict", "mra_last_error",
            "mra_free"]


def last_error() -> str:
    """Reason of the last failure on the calling thread (mra_last_error(NULL))."""
    m = lib().mra_last_error(None)
    return m.decode() if m else ""


class MRAError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_STATUS.get(status, str(status)), msg))
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("offset", ctypes.c_double), ("dedup", ctypes.c_int), ("precision", ctypes.c_int),
                ("device", ctypes.c_int), ("max_batch", ctypes.c_int), ("hbm_budget", ctypes.c_size_t),
                ("graphs", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int64), ("n_used", ctypes.c_int64), ("n_nan", ctypes.c_int64),
                ("n_dup", ctypes.c_int64), ("n_knot", ctypes.c_int64), ("n_regions", ctypes.c_int64),
                ("n_leaves", ctypes.c_int64), ("M", ctypes.c_int), ("J", ctypes.c_int), ("r", ctypes.c_int),
                ("r_hat", ctypes.c_int), ("max_leaf", ctypes.c_int64), ("empty_leaves", ctypes.c_int64),
                ("max_batch", ctypes.c_int), ("flops_per_theta", ctypes.c_double),
                ("cov_evals_per_theta", ctypes.c_double), ("device_bytes", ctypes.c_size_t),
                ("launches_per_pass", ctypes.c_int), ("flops_by_kernel", ctypes.c_double * 8),
                ("device_levels", ctypes.c_int), ("subtree_level", ctypes.c_int), ("subtree_chunks", ctypes.c_int)]

KERNEL_FAMILIES = ["prior", "leafbasis", "leafpost", "leafpost_big", "leafgram", "up", "root"]


class Tune(ctypes.Structure):
    _fields_ = [("leafbasis_rows", ctypes.c_int), ("leafbasis_stages", ctypes.c_int), ("bucket_set", ctypes.c_int),
                ("concurrent", ctypes.c_int), ("ms_default", ctypes.c_double), ("ms_best", ctypes.c_double),
                ("tried", ctypes.c_int), ("gram_tensor_cores", ctypes.c_int), ("leaf_queue", ctypes.c_int),
                ("prior_stages", ctypes.c_int), ("leafbasis_tensor_cores", ctypes.c_int),
                ("subtree_level", ctypes.c_int), ("subtree_chunk", ctypes.c_int),
                ("leafbasis_whole_chunks", ctypes.c_int)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int64), ("ms", ctypes.c_double)]


_lib = None


def lib():
    """Load libmra.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libmra.so is not built (run paper_1905_00141_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        D = ctypes.POINTER(ctypes.c_double)
        I64 = ctypes.POINTER(ctypes.c_int64)
        vp = ctypes.c_void_p
        L.mra_default_opts.argtypes = [ctypes.POINTER(Opts)]
        L.mra_build.restype = ctypes.c_int
        L.mra_build.argtypes = [D, D, D, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.POINTER(Opts), ctypes.POINTER(vp)]
        L.mra_loglik.restype = ctypes.c_int
        L.mra_loglik.argtypes = [vp, D, ctypes.c_int, D]
        L.mra_loglik_device.restype = ctypes.c_int
        L.mra_loglik_device.argtypes = [vp, vp, ctypes.c_int, vp, vp, vp]
        L.mra_autotune.restype = ctypes.c_int
        L.mra_autotune.argtypes = [vp, D, ctypes.c_int, ctypes.POINTER(Tune)]
        L.mra_set_launch.restype = ctypes.c_int
        L.mra_set_launch.argtypes = [vp, ctypes.POINTER(Tune)]
        L.mra_set_precision.restype = ctypes.c_int
        L.mra_set_precision.argtypes = [vp, ctypes.c_int]
        L.mra_stats.restype = ctypes.c_int
        L.mra_stats.argtypes = [vp, ctypes.POINTER(Stats)]
        L.mra_tree_export.restype = ctypes.c_int
        L.mra_tree_export.argtypes = [vp, D, D, I64, I64, D]
        L.mra_region_terms.restype = ctypes.c_int
        L.mra_region_terms.argtypes = [vp, D, D, D, D, D]
        L.mra_predict.restype = ctypes.c_int
        L.mra_predict.argtypes = [vp, D, D, D, ctypes.c_int64, D, D]
        L.mra_profile.restype = ctypes.c_int
        L.mra_profile.argtypes = [vp, ctypes.c_int]
        L.mra_profile_read.restype = ctypes.c_int
        L.mra_profile_read.argtypes = [vp, ctypes.POINTER(KernelTime), ctypes.c_int]
        L.mra_dense_loglik_noalloc.restype = ctypes.c_int
        L.mra_dense_loglik_noalloc.argtypes = [vp, vp, vp, ctypes.c_int64, vp, vp, vp, vp]
        L.mra_last_error.restype = ctypes.c_char_p
        L.mra_last_error.argtypes = [vp]
        L.mra_free.argtypes = [vp]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def default_opts() -> Opts:
    o = Opts()
    lib().mra_default_opts(ctypes.byref(o))
    return o


class MRA:
    """One built partition (mra_build) and its likelihood entry points.

    device=-1 builds the partition on the host only (no GPU needed); such a
    context answers stats/tree queries and refuses likelihood calls.
    """

    def __init__(self, x, y, z, M, J, r, offset=None, dedup=False, precision="fp64", device=0,
                 max_batch=0, hbm_budget=0, graphs=True):
        L = lib()
        self._x = np.ascontiguousarray(x, dtype=np.float64)
        self._y = np.ascontiguousarray(y, dtype=np.float64)
        self._z = np.ascontiguousarray(z, dtype=np.float64)
        o = default_opts()
        if offset is not None:
            o.offset = float(offset)
        o.dedup = int(bool(dedup))
        o.precision = _prec(precision)
        o.device = int(device)
        o.max_batch = int(max_batch)
        o.hbm_budget = int(hbm_budget)
        o.graphs = int(bool(graphs))
        h = ctypes.c_void_p(0)
        st = L.mra_build(_dp(self._x), _dp(self._y), _dp(self._z), len(self._x), int(M), int(J), int(r),
                         ctypes.byref(o), ctypes.byref(h))
        if st != OK:
            raise MRAError(st, L.mra_last_error(None).decode())
        self._h = h
        self._x = self._y = self._z = None
        self.M, self.J, self.r = int(M), int(J), int(r)

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            lib().mra_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, st):
        if st != OK:
            raise MRAError(st, lib().mra_last_error(self._h).decode())

    # -- queries
    def stats(self) -> dict:
        s = Stats()
        self._check(lib().mra_stats(self._h, ctypes.byref(s)))
        d = {f: getattr(s, f) for f, _ in Stats._fields_}
        d["flops_by_kernel"] = dict(zip(KERNEL_FAMILIES, list(s.flops_by_kernel)[:len(KERNEL_FAMILIES)]))
        return d

    def tree(self) -> dict:
        s = self.stats()
        nk = (s["n_regions"] - s["n_leaves"]) * s["r_hat"]
        kx = np.zeros(max(nk, 1))
        ky = np.zeros(max(nk, 1))
        lo = np.zeros(s["n_leaves"] + 1, dtype=np.int64)
        perm = np.zeros(max(s["n_used"], 1), dtype=np.int64)
        b = np.zeros(4 * s["n_regions"])
        self._check(lib().mra_tree_export(self._h, _dp(kx), _dp(ky), _ip(lo), _ip(perm), _dp(b)))
        return dict(kx=kx[:nk], ky=ky[:nk], leaf_off=lo, perm=perm[:s["n_used"]],
                    bounds=b.reshape(s["n_regions"], 4))

    def set_precision(self, precision):
        self._check(lib().mra_set_precision(self._h, _prec(precision)))

    # -- likelihood
    def loglik(self, theta, check: bool = True):
        """Host path: theta (B x 3: sigma2, beta, tau2) -> loglik (B,).  With
        check=False per-theta failures only show as NaN."""
        th = np.ascontiguousarray(np.atleast_2d(theta), dtype=np.float64)
        out = np.zeros(th.shape[0])
        st = lib().mra_loglik(self._h, _dp(th), th.shape[0], _dp(out))
        if check:
            self._check(st)
        return out

    def autotune(self, theta, reps: int = 5) -> dict:
        """Time the launch configurations on one theta and keep the fastest."""
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(3))
        out = Tune()
        self._check(lib().mra_autotune(self._h, _dp(th), int(reps), ctypes.byref(out)))
        return {k: getattr(out, k) for k, _ in Tune._fields_}

    def set_launch(self, leafbasis_rows=0, leafbasis_stages=0, bucket_set=0, concurrent=True, gram_tensor_cores=False,
                   leaf_queue=False, prior_stages=0, leafbasis_tensor_cores=False, subtree_level=0, subtree_chunk=0,
                   leafbasis_whole_chunks=False):
        cfg = Tune(int(leafbasis_rows), int(leafbasis_stages), int(bucket_set), int(bool(concurrent)), 0.0, 0.0, 0,
                   int(bool(gram_tensor_cores)), int(bool(leaf_queue)), int(prior_stages),
                   int(bool(leafbasis_tensor_cores)), int(subtree_level), int(subtree_chunk),
                   int(bool(leafbasis_whole_chunks)))
        self._check(lib().mra_set_launch(self._h, ctypes.byref(cfg)))

    def loglik_status(self, theta):
        th = np.ascontiguousarray(np.atleast_2d(theta), dtype=np.float64)
        out = np.zeros(th.shape[0])
        st = lib().mra_loglik(self._h, _dp(th), th.shape[0], _dp(out))
        return out, st

    def loglik_device(self, theta_ptr: int, batch: int, out_ptr: int, status_ptr: int = 0, stream: int = 0):
        """Device path: raw device pointers and a cudaStream_t handle (ints)."""
        self._check(lib().mra_loglik_device(self._h, ctypes.c_void_p(theta_ptr), int(batch),
                                            ctypes.c_void_p(out_ptr), ctypes.c_void_p(status_ptr or None),
                                            ctypes.c_void_p(stream or None)))

    def loglik_torch(self, theta, out=None, status=None):
        """theta: CUDA float64 tensor (B, 3); enqueued on torch's current stream."""
        import torch
        assert theta.is_cuda and theta.dtype == torch.float64 and theta.is_contiguous()
        B = theta.shape[0]
        if out is None:
            out = torch.empty(B, dtype=torch.float64, device=theta.device)
        sp = status.data_ptr() if status is not None else 0
        self.loglik_device(theta.data_ptr(), B, out.data_ptr(), sp,
                           torch.cuda.current_stream(theta.device).cuda_stream)
        return out

    def profile(self, enable: bool = True):
        self._check(lib().mra_profile(self._h, int(bool(enable))))

    def profile_read(self) -> dict:
        """{kernel family: (launches, device ms)} since the last read."""
        buf = (KernelTime * 16)()
        n = lib().mra_profile_read(self._h, buf, 16)
        if n < 0:
            raise MRAError(ECUDA, "profile read failed")
        return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].ms)) for i in range(min(n, 16))}

    def region_terms(self, theta) -> dict:
        s = self.stats()
        th = np.ascontiguousarray(theta, dtype=np.float64).reshape(3)
        n = s["n_regions"]
        d, u, lw, ll = np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(1)
        st = lib().mra_region_terms(self._h, _dp(th), _dp(d), _dp(u), _dp(lw), _dp(ll))
        return dict(d=d, u=u, logdetW=lw, loglik=float(ll[0]), status=int(st))


    def predict(self, theta, px, py):
        """Posterior predictive mean and variance of the latent process at the
        points (px, py) for one theta (mra_predict); NaN outside the domain."""
        th = np.ascontiguousarray(theta, dtype=np.float64).reshape(3)
        px = np.ascontiguousarray(px, dtype=np.float64).ravel()
        py = np.ascontiguousarray(py, dtype=np.float64).ravel()
        if px.shape != py.shape:
            raise ValueError("px and py differ in length")
        mean = np.empty(len(px))
        var = np.empty(len(px))
        self._check(lib().mra_predict(self._h, _dp(th), _dp(px), _dp(py), len(px), _dp(mean), _dp(var)))
        return mean, var


NOALLOC_MAX_N = 1024


def dense_loglik_noalloc(x_ptr: int, y_ptr: int, z_ptr: int, n: int, theta_ptr: int, out_ptr: int,
                         status_ptr: int = 0, stream: int = 0) -> None:
    """mra_dense_loglik_noalloc through the C ABI (raw device pointers); raises
    MRAError with the library's message on a call-level failure."""
    L = lib()
    st = L.mra_dense_loglik_noalloc(ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr), ctypes.c_void_p(z_ptr),
                                    int(n), ctypes.c_void_p(theta_ptr), ctypes.c_void_p(out_ptr),
                                    ctypes.c_void_p(status_ptr or None), ctypes.c_void_p(stream or None))
    if st != OK:
        raise MRAError(st, L.mra_last_error(None).decode())


def _prec(p):
    if isinstance(p, str):
        return {"fp64": FP64, "mixed": MIXED, "mixed_fast": MIXED_FAST}[p]
    return int(p)


LOG2PI = math.log(2 * math.pi)
