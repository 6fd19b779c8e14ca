"""Oracle pins: MLP forward/backward by finite differences, GELU closed values,
Adam closed-form first step."""
import math

import numpy as np

from oracle import mlp


def test_gelu_values():
    assert mlp.gelu(np.array(0.0)) == 0.0
    assert abs(mlp.gelu_grad(np.array(0.0)) - 0.5) < 1e-15
    z = np.array([8.0, -8.0])
    assert np.allclose(mlp.gelu(z), [8.0, 0.0], atol=1e-12)
    # gelu(1) = Phi(1) = 0.8413447460685429 (standard normal CDF at 1)
    assert abs(mlp.gelu(np.array(1.0)) - 0.8413447460685429) < 1e-15
    zz = np.linspace(-4, 4, 41)
    h = 1e-6
    fd = (mlp.gelu(zz + h) - mlp.gelu(zz - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_grad(zz))) < 1e-9


def test_backward_matches_finite_differences():
    sizes = [7, 12, 10, 5]
    params = mlp.init_params(sizes, seed=3)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((6, 7))
    T = rng.standard_normal((6, 5))
    Y, cache = mlp.forward(params, X)
    grads = mlp.backward(params, cache, Y, T)
    h = 1e-6
    for l in range(3):
        for k in range(2):
            p = params[l][k]
            g = grads[l][k]
            for idx in [tuple(rng.integers(0, s) for s in p.shape) for _ in range(4)]:
                def loss(delta):
                    q = [tuple(x.copy() for x in pr) for pr in params]
                    q[l][k][idx] += delta
                    return mlp.mse(mlp.forward(q, X)[0], T)
                fd = (loss(h) - loss(-h)) / (2 * h)
                assert abs(fd - g[idx]) < 1e-7 * (1 + abs(fd)), (l, k, idx, fd, g[idx])


def test_init_bounds_and_shapes():
    params = mlp.init_params([100, 64, 3], seed=1)
    W, b = params[0]
    assert W.shape == (64, 100) and b.shape == (64,)
    assert np.all(np.abs(W) <= 0.1) and np.all(np.abs(b) <= 0.1)
    assert abs(W.std() - 0.1 / math.sqrt(3)) < 0.01       # uniform std = bound / sqrt(3)


def test_adam_first_step_is_lr_sign():
    params = [(np.array([[1.0, -2.0]]), np.array([0.5]))]
    grads = [(np.array([[0.3, -7.0]]), np.array([-1e-3]))]
    opt = mlp.Adam(params, lr=1e-3)
    new = opt.step(params, grads)
    # m_hat = g, v_hat = g^2: the first step is lr * g / (|g| + eps)
    assert np.allclose(new[0][0], [[1.0 - 1e-3, -2.0 + 1e-3]], atol=1e-10)
    assert np.allclose(new[0][1], [0.5 + 1e-3 * 1e-3 / (1e-3 + 1e-8)], atol=1e-12)


def test_training_reduces_loss():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((64, 8))
    T = np.tanh(X[:, :3] * 1.5)
    params = mlp.init_params([8, 32, 32, 3], seed=2)
    opt = mlp.Adam(params, lr=1e-2)
    l0 = mlp.mse(mlp.forward(params, X)[0], T)
    for _ in range(200):
        Y, cache = mlp.forward(params, X)
        params = opt.step(params, mlp.backward(params, cache, Y, T))
    assert mlp.mse(mlp.forward(params, X)[0], T) < 0.1 * l0
