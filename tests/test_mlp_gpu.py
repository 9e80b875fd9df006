"""GPU kernels of the surrogate network against the FP64 reference.

Forward pass, gradient (relative error <= 1e-3, BF16 parameters with FP32
accumulation against FP64 arithmetic on the same BF16 values), Adam steps,
the CUDA-graph replay of training, and that training fits a smooth target.
"""
import numpy as np
import pytest

from oracle import mlp as om
from paper_1905_00141_gb300 import synth

pytestmark = pytest.mark.gpu
BOX = synth.THETA_BOX


@pytest.fixture(scope="module")
def mlp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1905_00141_gb300 import build
    build.build()
    from paper_1905_00141_gb300 import mlp as m
    return m


def _data(n, seed):
    th = synth.theta_sobol(n, seed=seed)
    u = om.features(th, BOX)
    target = -1.3 + 0.2 * u[:, 0] - 0.1 * u[:, 1] ** 2 + 0.05 * u[:, 2] * u[:, 0]
    return th, target


def _params(seed):
    p = synth.mlp_init(seed=seed)
    p[om.O_B1:om.O_W2] = np.random.default_rng(seed).normal(0, 0.1, om.H).astype(np.float32)
    p[om.O_B3] = 0.3
    return p


@pytest.mark.parametrize("n", [1, 63, 64, 1000])
def test_predict_matches_reference(mlp, n):
    p = _params(21)
    th, _ = _data(n, 22)
    s = mlp.Surrogate(BOX, p, t_off=-1.3, t_scale=0.2)
    try:
        got = s.predict(th)
    finally:
        s.close()
    ref = om.forward(p, th, BOX, -1.3, 0.2)
    assert got.shape == (n,)
    assert np.allclose(got, ref, rtol=0, atol=2e-6 * 0.2 * (1 + np.max(np.abs((ref + 1.3) / 0.2))))


@pytest.mark.parametrize("n", [37, 2048])
def test_gradient_matches_reference(mlp, n):
    p = _params(31)
    th, target = _data(n, 32)
    s = mlp.Surrogate(BOX, p, t_off=-1.25, t_scale=0.15)
    try:
        g, L = s.grad(th, target)
        assert np.array_equal(s.params(), p)  # no update
    finally:
        s.close()
    Lr, gr = om.loss_grad(p, th, target, BOX, -1.25, 0.15)
    assert abs(L - Lr) <= 1e-5 * Lr
    assert np.linalg.norm(g - gr) <= 1e-3 * np.linalg.norm(gr)
    assert np.max(np.abs(g - gr)) <= 1e-3 * np.max(np.abs(gr))


def test_adam_steps_match_reference(mlp):
    p = _params(41)
    th, target = _data(512, 42)
    s = mlp.Surrogate(BOX, p, t_off=-1.3, t_scale=0.2)
    try:
        hist = s.train(th, target, 5, lr=1e-3)
        got = s.params()
    finally:
        s.close()
    ref, rh = om.train(p, th, target, BOX, -1.3, 0.2, 5, 1e-3)
    assert np.allclose(hist, rh, rtol=1e-4, atol=0)
    # Adam moves each parameter by about lr per step, whatever the gradient's size
    assert np.max(np.abs(got - ref)) <= 5 * 2e-3
    assert np.median(np.abs(got - ref)) <= 1e-5


def test_graph_replay_is_deterministic(mlp):
    p = _params(51)
    th, target = _data(700, 52)
    out = []
    for split in ([70], [64, 6], [1] * 6 + [64]):
        s = mlp.Surrogate(BOX, p, t_off=-1.3, t_scale=0.2)
        try:
            h = np.concatenate([s.train(th, target, k, lr=2e-3) for k in split])
            out.append((s.params(), h))
        finally:
            s.close()
    for q, h in out[1:]:
        assert np.array_equal(q, out[0][0])
        assert np.array_equal(h, out[0][1])


def test_training_fits_smooth_target(mlp):
    th, target = _data(2048, 61)
    s = mlp.Surrogate(BOX, synth.mlp_init(seed=62), t_off=float(np.mean(target)), t_scale=float(np.std(target)))
    try:
        hist = s.train(th, target, 3000, lr=3e-3)
        th2, t2 = _data(512, 63)
        pred = s.predict(th2)
    finally:
        s.close()
    assert hist[-1] < 1e-3 * hist[0]
    assert np.max(np.abs(pred - t2)) < 0.02 * np.std(target) * 10
