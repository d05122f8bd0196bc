"""Pins of the CPU FP64 seed-network reference (oracle/mlp.py): the analytic gradient
against central finite differences of the loss, SiLU's derivative against finite
differences, closed forms of degenerate networks, and bf16 rounding against torch's
own conversion."""
import numpy as np
import pytest

from oracle import mlp


def _rand(seed=0, B=7):
    g = np.random.default_rng(seed)
    theta = g.normal(0.0, 0.3, mlp.n_params())
    x = g.normal(0.0, 1.0, (B, mlp.N_IN))
    y = g.normal(0.0, 1.0, (B, mlp.N_OUT))
    return theta, x, y


def test_param_count_and_layout():
    assert mlp.n_params() == 64 * 13 + 64 + 2 * (64 * 64 + 64) + 3 * 64 + 3
    theta, _, _ = _rand()
    assert np.array_equal(mlp.flatten(mlp.unflatten(theta)), theta)


def test_gradient_matches_central_differences():
    theta, x, y = _rand(1)
    w = (1.0, 2.0, 0.5)
    g = mlp.grad(theta, x, y, w)
    rng = np.random.default_rng(2)
    idx = rng.choice(theta.size, 200, replace=False)
    h = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        fd = (mlp.loss(tp, x, y, w) - mlp.loss(tm, x, y, w)) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-8)


def test_silu_derivative():
    z = np.linspace(-8, 8, 101)
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.silu_grad(z), fd, rtol=1e-7, atol=1e-9)
    assert mlp.silu(0.0) == 0.0 and mlp.silu_grad(0.0) == 0.5


def test_degenerate_networks():
    # all weights zero: output = b4 whatever the input
    W = [np.zeros(s) for s in mlp.SHAPES]
    W[7] = np.array([0.3, -0.2, 1.5])
    theta = mlp.flatten(W)
    x = np.random.default_rng(3).normal(size=(5, mlp.N_IN))
    o, _, _ = mlp.forward(theta, x)
    np.testing.assert_allclose(o, np.tile(W[7], (5, 1)), rtol=0, atol=0)
    # with zero hidden biases and zero W1 every hidden unit is silu(0) = 0, so the
    # gradient of the output layer weights vanishes and the bias gradient is 2(o - y)/B
    y = np.zeros((5, 3))
    g = mlp.unflatten(mlp.grad(theta, x, y))
    assert np.all(g[6] == 0.0)
    np.testing.assert_allclose(g[7], 2.0 * W[7], rtol=1e-15)


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    a = np.random.default_rng(4).normal(0, 10, 10000) * 10.0 ** np.random.default_rng(5).uniform(-20, 20, 10000)
    ref = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(a), ref)
