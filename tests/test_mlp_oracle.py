"""Pins of the FP64 reference of the surrogate network (oracle/mlp.py).

The reference's backward pass is hand-written; it is pinned to central finite
differences and to PyTorch autograd (an independent differentiation of a
network built from torch.nn layers), its BF16 rounding to PyTorch's
bfloat16 conversion, and its Adam step to torch.optim.Adam.
"""
import numpy as np
import pytest

from oracle import mlp as om
from paper_1905_00141_gb300 import synth

BOX = synth.THETA_BOX


def _data(n, seed):
    rng = np.random.default_rng(seed)
    th = synth.theta_sobol(n, seed=seed)
    u = om.features(th, BOX)
    target = -1.3 + 0.2 * u[:, 0] - 0.1 * u[:, 1] ** 2 + 0.05 * u[:, 2] + 0.01 * rng.standard_normal(n)
    return th, target


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = rng.standard_normal(20000).astype(np.float32) * np.float32(10.0) ** rng.integers(-8, 8, 20000)
    # exact ties: lower 16 bits 0x8000, both parities of the kept part
    bits = rng.integers(0, 2 ** 31, 4000, dtype=np.uint64).astype(np.uint32)
    ties = ((bits & np.uint32(0xFFFF0000)) | np.uint32(0x8000)).view(np.float32)
    ties = ties[np.isfinite(ties)]
    x = np.concatenate([x, ties, np.array([0.0, -0.0, 1.0, -3.5], np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(om.bf16_round(x), ref)


def test_dsilu_is_derivative_of_silu():
    z = np.linspace(-12, 12, 241)
    h = 1e-6
    fd = (om.silu(z + h) - om.silu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - om.dsilu(z))) < 1e-8


def test_gradient_matches_finite_differences():
    p = synth.mlp_init(seed=3).astype(np.float64)
    p += 0.05 * np.random.default_rng(1).standard_normal(p.size)  # nonzero biases
    th, target = _data(40, 11)
    L, g = om.loss_grad(p, th, target, BOX, t_off=-1.3, t_scale=0.2, round_params=False)
    rng = np.random.default_rng(2)
    idx = np.concatenate([np.arange(0, 5), [om.O_B1, om.O_B1 + 7, om.O_W2, om.O_W2 + 123, om.O_B2 + 3,
                                            om.O_W3, om.O_W3 + 63, om.O_B3], rng.integers(0, om.NPARAM, 20)])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        Lp, _ = om.loss_grad(p + e, th, target, BOX, -1.3, 0.2, round_params=False)
        Lm, _ = om.loss_grad(p - e, th, target, BOX, -1.3, 0.2, round_params=False)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_forward_and_gradient_match_torch_autograd():
    torch = pytest.importorskip("torch")
    p = om.bf16_round(synth.mlp_init(seed=4))
    p = p + 0.0  # rounded values used as-is below
    th, target = _data(100, 12)
    W1, b1, W2, b2, w3, b3 = om.unpack(p)
    net = torch.nn.Sequential(torch.nn.Linear(3, 64), torch.nn.SiLU(), torch.nn.Linear(64, 64), torch.nn.SiLU(),
                              torch.nn.Linear(64, 1)).double()
    with torch.no_grad():
        net[0].weight.copy_(torch.from_numpy(W1))
        net[0].bias.copy_(torch.from_numpy(b1))
        net[2].weight.copy_(torch.from_numpy(W2))
        net[2].bias.copy_(torch.from_numpy(b2))
        net[4].weight.copy_(torch.from_numpy(w3[None, :]))
        net[4].bias.copy_(torch.tensor([float(b3)]))
    X = torch.from_numpy(om.features(th, BOX))
    tau = torch.from_numpy((target - (-1.3)) / 0.2)
    y = net(X)[:, 0]
    loss = 0.5 * ((y - tau) ** 2).mean()
    loss.backward()
    L, g = om.loss_grad(p, th, target, BOX, -1.3, 0.2)
    assert abs(L - loss.item()) <= 1e-12 * max(1.0, L)
    pred = om.forward(p, th, BOX, -1.3, 0.2)
    assert np.allclose(pred, -1.3 + 0.2 * y.detach().numpy(), rtol=0, atol=1e-12)
    tg = np.concatenate([net[0].weight.grad.numpy().ravel(), net[0].bias.grad.numpy(),
                         net[2].weight.grad.numpy().ravel(), net[2].bias.grad.numpy(),
                         net[4].weight.grad.numpy().ravel(), net[4].bias.grad.numpy()])
    assert np.allclose(g, tg, rtol=1e-10, atol=1e-13)


def test_constant_network_closed_form():
    # W1 = W2 = 0: every sample gets c = w3 . silu(b2) + b3, and dL/db3 = c - mean(tau)
    p = np.zeros(om.NPARAM)
    p[om.O_B2:om.O_W3] = 0.5
    p[om.O_W3:om.O_B3] = 0.25
    p[om.O_B3] = -0.125
    th, target = _data(30, 13)
    c = 64 * 0.25 * 0.5 / (1.0 + np.exp(-0.5)) - 0.125
    L, g = om.loss_grad(p, th, target, BOX)
    assert np.allclose(om.forward(p, th, BOX), c, atol=1e-14)
    assert abs(g[om.O_B3] - (c - np.mean(target))) < 1e-14
    assert abs(L - 0.5 * np.mean((c - target) ** 2)) < 1e-14
    # W2 = 0 stops the gradient at layer 2: nothing reaches W1, b1
    assert np.all(g[om.O_W1:om.O_W2] == 0.0)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    p0 = rng.standard_normal(50)
    grads = [rng.standard_normal(50) for _ in range(4)]
    tp = torch.nn.Parameter(torch.from_numpy(p0.copy()))
    opt = torch.optim.Adam([tp], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for t, g in enumerate(grads, start=1):
        tp.grad = torch.from_numpy(g.copy())
        opt.step()
        p, m, v = om.adam(p, m, v, g, t, 3e-3)
    assert np.allclose(p, tp.detach().numpy(), rtol=0, atol=1e-12)


def test_training_reduces_loss():
    th, target = _data(256, 14)
    p0 = synth.mlp_init(seed=6)
    _, hist = om.train(p0, th, target, BOX, float(np.mean(target)), float(np.std(target)), 200, 3e-3)
    assert hist[-1] < 0.2 * hist[0]
