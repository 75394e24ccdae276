"""Pins of the FP64 MLP oracle: GELU values and identities, finite-difference gradients, Adam."""
import math

import numpy as np

from oracle import mlp
from paper_2502_14148_gb300 import inputs


def test_gelu_values_and_identities():
    # gelu(1) = Phi(1) (standard normal table), gelu(0) = 0, gelu(x) - gelu(-x) = x
    assert abs(mlp.gelu(np.array(1.0)) - 0.8413447460685429) < 1e-15
    assert mlp.gelu(np.array(0.0)) == 0.0
    x = np.linspace(-5, 5, 41)
    np.testing.assert_allclose(mlp.gelu(x) - mlp.gelu(-x), x, atol=1e-14)
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_prime(x), (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h), atol=1e-8)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    sizes = (6, 7, 5, 4, 3)
    params = [(rng.standard_normal((sizes[l + 1], sizes[l])) * 0.7, rng.standard_normal(sizes[l + 1]) * 0.1)
              for l in range(4)]
    X = rng.standard_normal((9, 6)); T = rng.standard_normal((9, 3)); mask = np.array([1.0, 1.0, 0.0])
    y, cache = mlp.forward(params, X)
    grads = mlp.backward(params, cache, y, T, mask)
    h = 1e-6
    for l in range(4):
        for which in (0, 1):
            P = params[l][which]
            G = grads[l][which]
            for idx in list(np.ndindex(P.shape))[:12]:
                old = P[idx]
                P[idx] = old + h; lp = mlp.loss(mlp.forward(params, X)[0], T, mask)
                P[idx] = old - h; lm = mlp.loss(mlp.forward(params, X)[0], T, mask)
                P[idx] = old
                assert abs((lp - lm) / (2 * h) - G[idx]) < 1e-7 * max(1.0, abs(G[idx])), (l, which, idx)


def test_masked_outputs_do_not_contribute():
    params = inputs.mlp_init(seed=3, sizes=(8, 6, 6, 6, 4))
    X = np.random.default_rng(1).standard_normal((5, 8))
    T1 = np.random.default_rng(2).standard_normal((5, 4)); T2 = T1.copy(); T2[:, 2:] += 5.0
    mask = np.array([1.0, 1.0, 0.0, 0.0])
    y, cache = mlp.forward(params, X)
    g1, g2 = mlp.backward(params, cache, y, T1, mask), mlp.backward(params, cache, y, T2, mask)
    for a, b in zip(g1, g2):
        np.testing.assert_array_equal(a[0], b[0]); np.testing.assert_array_equal(a[1], b[1])


def test_adam_first_step_is_lr_times_sign():
    """With bias correction, Adam's first step is lr * g/(|g| + eps'), i.e. lr * sign(g) for |g| >> eps."""
    params = [(np.array([[1.0, -2.0]]), np.array([0.5]))]
    grads = [(np.array([[3.0, -0.25]]), np.array([1e-3]))]
    st = {}
    new = mlp.adam_step(params, grads, st, lr=0.01)
    np.testing.assert_allclose(new[0][0] - params[0][0], -0.01 * np.sign(grads[0][0]), rtol=1e-6)
    np.testing.assert_allclose(new[0][1] - params[0][1], -0.01 * np.sign(grads[0][1]), rtol=1e-4)


def test_adam_reduces_a_regression_loss():
    X, T, mask = inputs.mlp_batch(seed=4, M=64, n_in=8, n_out=4, n_real_in=8, n_real_out=2)
    T[:, :2] = np.tanh(X[:, :2])
    params = inputs.mlp_init(seed=4, sizes=(8, 16, 16, 16, 4))
    st = {}
    l0 = mlp.loss(mlp.forward(params, X)[0], T, mask)
    for _ in range(200):
        y, cache = mlp.forward(params, X)
        params = mlp.adam_step(params, mlp.backward(params, cache, y, T, mask), st, lr=3e-3)
    assert mlp.loss(mlp.forward(params, X)[0], T, mask) < 0.2 * l0
