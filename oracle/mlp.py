"""FP64 reference of the surrogate network of loglik(theta)/n.

TEST INFRASTRUCTURE ONLY (see the package docstring): imported by the tests,
never by the library.  The network is an addition to the paper's method (the
paper's own search, Sec. 2.2.5, calls the exact likelihood at every step):

    x    = 2 (log theta - log lo) / (log hi - log lo) - 1        (3 inputs)
    h1   = SiLU(W1 x + b1),  h2 = SiLU(W2 h1 + b2)               (64, 64)
    yhat = w3 . h2 + b3,     prediction = t_off + t_scale * yhat
    SiLU(z) = z * sigma(z),  sigma(z) = 1 / (1 + exp(-z))

Parameters (flat, this order): W1 [64][3] row-major, b1, W2 [64][64]
row-major, b2, w3, b3.  Before use they are rounded to BF16 (round to
nearest, ties to even, applied to the FP32 value); all other arithmetic here
is FP64.  Loss over B samples: L = (1/2B) sum_s (yhat_s - tau_s)^2 with
tau_s = (target_s - t_off) / t_scale.  The gradient is the chain rule written
out layer by layer (no automatic differentiation); Adam is Kingma & Ba
(ICLR 2015), Algorithm 1, with bias correction.
"""
from __future__ import annotations

import numpy as np

H = 64
NPARAM = 3 * H + H + H * H + H + H + 1
O_W1, O_B1 = 0, 3 * H
O_W2 = O_B1 + H
O_B2 = O_W2 + H * H
O_W3 = O_B2 + H
O_B3 = O_W3 + H


def bf16_round(p):
    """FP32 value of each parameter rounded to the nearest BF16 (ties to even)."""
    bits = np.ascontiguousarray(np.asarray(p, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    lsb = (bits >> np.uint64(16)) & np.uint64(1)
    r = (bits + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return (p[O_W1:O_B1].reshape(H, 3), p[O_B1:O_W2], p[O_W2:O_B2].reshape(H, H), p[O_B2:O_W3], p[O_W3:O_B3],
            p[O_B3])


def features(theta, box):
    th = np.asarray(theta, dtype=np.float64).reshape(-1, 3)
    lo, hi = np.log(np.asarray(box[0], float)), np.log(np.asarray(box[1], float))
    return 2.0 * (np.log(th) - lo) / (hi - lo) - 1.0


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * sigmoid(z)


def dsilu(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def _net(params, X, round_params=True):
    W1, b1, W2, b2, w3, b3 = unpack(bf16_round(params) if round_params else params)
    Z1 = X @ W1.T + b1
    A1 = silu(Z1)
    Z2 = A1 @ W2.T + b2
    A2 = silu(Z2)
    y = A2 @ w3 + b3
    return y, (W1, b1, W2, b2, w3, b3, Z1, A1, Z2, A2)


def forward(params, theta, box, t_off=0.0, t_scale=1.0, round_params=True):
    """Predicted loglik/n at each theta."""
    y, _ = _net(params, features(theta, box), round_params)
    return t_off + t_scale * y


def loss_grad(params, theta, target, box, t_off=0.0, t_scale=1.0, round_params=True):
    """(L, dL/dparams) at the BF16-rounded parameters (or at the parameters
    as given, round_params=False); the gradient is with respect to the
    parameter values the network uses."""
    X = features(theta, box)
    tau = (np.asarray(target, dtype=np.float64).reshape(-1) - t_off) / t_scale
    B = X.shape[0]
    y, (W1, b1, W2, b2, w3, b3, Z1, A1, Z2, A2) = _net(params, X, round_params)
    r = y - tau
    L = 0.5 * np.dot(r, r) / B
    e = r / B                                  # dL/dyhat
    g_w3 = A2.T @ e
    g_b3 = e.sum()
    D2 = np.outer(e, w3) * dsilu(Z2)           # dL/dZ2
    g_W2 = D2.T @ A1
    g_b2 = D2.sum(axis=0)
    D1 = (D2 @ W2) * dsilu(Z1)                 # dL/dZ1
    g_W1 = D1.T @ X
    g_b1 = D1.sum(axis=0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return L, g


def adam(params, m, v, g, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (step number t >= 1) on FP64 copies."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m, v


def train(params, theta, target, box, t_off, t_scale, steps, lr):
    """Full-batch Adam from `params` (moments at zero); returns (params, loss
    before each step)."""
    p = np.asarray(params, dtype=np.float64).copy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    hist = []
    for t in range(1, steps + 1):
        L, g = loss_grad(p, theta, target, box, t_off, t_scale)
        hist.append(L)
        p, m, v = adam(p, m, v, g, t, lr)
    return p, np.array(hist)
