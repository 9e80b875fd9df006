"""Thin ctypes binding of the surrogate network of libmra (include/mra_mlp.h).

Argument marshalling only: the forward pass, the gradient and the Adam steps
run in the CUDA kernels of libmra.so.  PyTorch supplies the device buffers.
There is no CPU fallback: without the library or a GPU the calls raise.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import mra

HIDDEN = 64
NPARAM = 3 * HIDDEN + HIDDEN + HIDDEN * HIDDEN + HIDDEN + HIDDEN + 1
MAX_BATCH = 65536
EXPORTED = ["mra_mlp_create", "mra_mlp_set_params", "mra_mlp_get_params", "mra_mlp_set_target_scaling",
            "mra_mlp_predict", "mra_mlp_grad", "mra_mlp_train", "mra_mlp_free"]


def glorot_init(seed: int, hidden: int = HIDDEN):
    """Initial parameters: weights uniform in +-sqrt(6 / (fan_in + fan_out))
    (Glorot & Bengio 2010), biases zero, in the library's parameter order."""
    rng = np.random.default_rng(seed)

    def w(fo, fi):
        a = (6.0 / (fi + fo)) ** 0.5
        return rng.uniform(-a, a, size=(fo, fi)).ravel()

    z = np.zeros
    return np.concatenate([w(hidden, 3), z(hidden), w(hidden, hidden), z(hidden), w(1, hidden), z(1)]).astype(
        np.float32)


class Scaling(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3), ("t_off", ctypes.c_double),
                ("t_scale", ctypes.c_double)]


_bound = False


def _lib():
    global _bound
    L = mra.lib()
    if not _bound:
        vp = ctypes.c_void_p
        F = ctypes.POINTER(ctypes.c_float)
        L.mra_mlp_create.restype = ctypes.c_int
        L.mra_mlp_create.argtypes = [ctypes.c_int, ctypes.POINTER(Scaling), F, ctypes.POINTER(vp)]
        L.mra_mlp_set_params.restype = ctypes.c_int
        L.mra_mlp_set_params.argtypes = [vp, F]
        L.mra_mlp_get_params.restype = ctypes.c_int
        L.mra_mlp_get_params.argtypes = [vp, F]
        L.mra_mlp_set_target_scaling.restype = ctypes.c_int
        L.mra_mlp_set_target_scaling.argtypes = [vp, ctypes.c_double, ctypes.c_double]
        L.mra_mlp_predict.restype = ctypes.c_int
        L.mra_mlp_predict.argtypes = [vp, vp, ctypes.c_int, vp, vp]
        L.mra_mlp_grad.restype = ctypes.c_int
        L.mra_mlp_grad.argtypes = [vp, vp, vp, ctypes.c_int, vp, vp, vp]
        L.mra_mlp_train.restype = ctypes.c_int
        L.mra_mlp_train.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_float, vp]
        L.mra_mlp_free.restype = None
        L.mra_mlp_free.argtypes = [vp]
        _bound = True
    return L


def _check(st):
    if st != mra.OK:
        raise mra.MRAError(st, mra.last_error())


class Surrogate:
    """The 3 -> 64 -> 64 -> 1 SiLU network predicting loglik(theta)/n.

    box = (lo[3], hi[3]) fixes the input scaling; t_off, t_scale the target
    scaling (prediction = t_off + t_scale * network output)."""

    def __init__(self, box, params, t_off=0.0, t_scale=1.0, device=0):
        import torch
        self.torch = torch
        self.device = device
        sc = Scaling()
        for i in range(3):
            sc.lo[i] = float(box[0][i])
            sc.hi[i] = float(box[1][i])
        sc.t_off, sc.t_scale = float(t_off), float(t_scale)
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != NPARAM:
            raise ValueError("expected %d parameters" % NPARAM)
        h = ctypes.c_void_p()
        _check(_lib().mra_mlp_create(int(device), ctypes.byref(sc), p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                     ctypes.byref(h)))
        self.h = h

    def _dev(self, a, dtype):
        t = self.torch
        if isinstance(a, t.Tensor):
            return a.to(device="cuda:%d" % self.device, dtype=dtype).contiguous()
        return t.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda:%d" % self.device)

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        _check(_lib().mra_mlp_set_params(self.h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def params(self):
        p = np.empty(NPARAM, dtype=np.float32)
        _check(_lib().mra_mlp_get_params(self.h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return p

    def set_target_scaling(self, t_off, t_scale):
        _check(_lib().mra_mlp_set_target_scaling(self.h, float(t_off), float(t_scale)))

    def predict(self, theta):
        """Predicted loglik/n at theta [B][3] (numpy or tensor) -> numpy [B]."""
        t = self.torch
        th = self._dev(theta, t.float64).reshape(-1, 3)
        out = t.empty(th.shape[0], dtype=t.float64, device=th.device)
        for i0 in range(0, th.shape[0], MAX_BATCH):
            n = min(MAX_BATCH, th.shape[0] - i0)
            _check(_lib().mra_mlp_predict(self.h, th[i0:].data_ptr(), n, out[i0:].data_ptr(), None))
        t.cuda.synchronize(th.device)
        return out.cpu().numpy()

    def grad(self, theta, target):
        """(gradient [NPARAM] float32, loss) of the training loss, no update."""
        t = self.torch
        th = self._dev(theta, t.float64).reshape(-1, 3)
        tg = self._dev(target, t.float64).reshape(-1)
        g = t.empty(NPARAM, dtype=t.float32, device=th.device)
        loss = t.empty(1, dtype=t.float32, device=th.device)
        _check(_lib().mra_mlp_grad(self.h, th.data_ptr(), tg.data_ptr(), th.shape[0], g.data_ptr(),
                                   loss.data_ptr(), None))
        t.cuda.synchronize(th.device)
        return g.cpu().numpy(), float(loss.cpu()[0])

    def train(self, theta, target, steps, lr=1e-3):
        """`steps` full-batch Adam steps; returns the loss before each step."""
        t = self.torch
        th = self._dev(theta, t.float64).reshape(-1, 3)
        tg = self._dev(target, t.float64).reshape(-1)
        hist = t.empty(max(int(steps), 1), dtype=t.float32, device=th.device)
        t.cuda.synchronize(th.device)
        _check(_lib().mra_mlp_train(self.h, th.data_ptr(), tg.data_ptr(), th.shape[0], int(steps), float(lr),
                                    hist.data_ptr()))
        return hist[:steps].cpu().numpy()

    def close(self):
        if getattr(self, "h", None):
            _lib().mra_mlp_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
