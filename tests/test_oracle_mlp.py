"""Pins of the oracle surrogate network: GELU, manual backward against central
finite differences, Adam against its closed form, the shuffle, training."""
import math

import numpy as np
import pytest

from oracle import mlp
from workloads import mlp_init


def test_gelu_values_and_derivative():
    assert mlp.gelu(0.0) == 0.0
    # gelu(z) = z Phi(z): Phi(1) = 0.841344746..., Phi(-1) = 0.158655253...
    assert abs(mlp.gelu(1.0) - 0.8413447460685429) < 1e-15
    assert abs(mlp.gelu(-1.0) + 0.15865525393145707) < 1e-15
    assert abs(mlp.gelu_grad(0.0) - 0.5) < 1e-16
    z = np.linspace(-4, 4, 33)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.abs(fd - mlp.gelu_grad(z)).max() < 1e-9


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    params = [(rng.standard_normal((5, 2)), rng.standard_normal(5)),
              (rng.standard_normal((5, 5)), rng.standard_normal(5)),
              (rng.standard_normal((3, 5)), rng.standard_normal(3))]
    X = rng.standard_normal((4, 2))
    T = rng.standard_normal((4, 3))
    loss, grads = mlp.loss_and_grads(params, X, T)
    h = 1e-6
    for li in range(3):
        for pi in range(2):
            p = params[li][pi]
            g = grads[li][pi]
            for idx in np.ndindex(p.shape):
                old = p[idx]
                p[idx] = old + h
                lp, _ = mlp.loss_and_grads(params, X, T)
                p[idx] = old - h
                lm, _ = mlp.loss_and_grads(params, X, T)
                p[idx] = old
                assert abs((lp - lm) / (2 * h) - g[idx]) < 1e-7 * max(1.0, abs(g[idx]))


def test_adam_closed_form():
    # scalar parameter, gradients g1 then g2: m_t, v_t with bias correction
    params = [(np.array([[1.0]]), np.array([0.0]))]
    state = mlp.adam_init(params)
    g1, g2, lr = 0.5, -2.0, 0.1
    params, state = mlp.adam_step(params, [(np.array([[g1]]), np.array([0.0]))], state, lr)
    assert abs(params[0][0][0, 0] - (1.0 - lr * g1 / (abs(g1) + 1e-8))) < 1e-15
    params, state = mlp.adam_step(params, [(np.array([[g2]]), np.array([0.0]))], state, lr)
    m = 0.9 * 0.1 * g1 + 0.1 * g2
    v = 0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2
    step2 = lr * (m / (1 - 0.81)) / (math.sqrt(v / (1 - 0.999 ** 2)) + 1e-8)
    assert abs(params[0][0][0, 0] - (1.0 - lr * g1 / (abs(g1) + 1e-8) - step2)) < 1e-14


def test_shuffle_is_permutation():
    for n in (8192, 1000, 7):
        for e in range(3):
            p = mlp.epoch_permutation(n, 5, e)
            assert np.array_equal(np.sort(p), np.arange(n))
    assert not np.array_equal(mlp.epoch_permutation(1000, 5, 0), mlp.epoch_permutation(1000, 5, 1))
    assert mlp.splitmix64(0) == 0xE220A8397B1DCDAF   # first output of SplitMix64 seeded with 0


def test_training_fits_a_smooth_map():
    rng = np.random.default_rng(1)
    X = rng.uniform(-1, 1, (256, 2))
    T = np.stack([np.sin(X[:, 0]) * np.cos(X[:, 1]), X[:, 0] * X[:, 1], np.exp(0.5 * X[:, 0])], 1)
    mean, std = mlp.target_stats(T)
    params = [(W[:, :], b) for W, b in mlp_init(3, hidden=32)]
    _, losses = mlp.train(params, X, (T - mean) / std, epochs=60, batch=64, lr0=3e-3, seed=5)
    assert losses[-1] < 0.05 * losses[0]
