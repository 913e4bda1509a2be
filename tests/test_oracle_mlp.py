"""Pins of the predictor oracle: backpropagation vs finite differences, Adam, POD."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as P
from paper_2508_06302_gb300 import inputs as I


def _small():
    params = I.mlp_init(3, 16, 5, seed=1)
    rng = np.random.default_rng(2)
    for k in ("b1", "b2", "b3"):
        params[k] = 0.1 * rng.standard_normal(params[k].shape)
    X = rng.uniform(-1, 1, (7, 3))
    T = rng.standard_normal((7, 5))
    return params, X, T


def test_gelu_matches_definition():
    z = np.linspace(-4, 4, 17)
    from scipy.stats import norm
    np.testing.assert_allclose(P.gelu(z), z * norm.cdf(z), rtol=1e-13, atol=1e-15)
    h = 1e-6
    np.testing.assert_allclose(P.gelu_grad(z), (P.gelu(z + h) - P.gelu(z - h)) / (2 * h), rtol=1e-7, atol=1e-9)


def test_backprop_matches_finite_differences():
    params, X, T = _small()
    L, g = P.loss_and_grads(params, X, T)
    h = 1e-6
    for k in P.PARAM_ORDER:
        flat = params[k].reshape(-1)
        fd = np.zeros_like(flat)
        for i in range(flat.size):
            old = flat[i]
            flat[i] = old + h
            Lp, _ = P.loss_and_grads(params, X, T)
            flat[i] = old - h
            Lm, _ = P.loss_and_grads(params, X, T)
            flat[i] = old
            fd[i] = (Lp - Lm) / (2 * h)
        np.testing.assert_allclose(g[k].reshape(-1), fd, rtol=1e-6, atol=1e-9)


def test_adam_first_step_is_signed_lr():
    params, X, T = _small()
    L, g = P.loss_and_grads(params, X, T)
    before = {k: v.copy() for k, v in params.items()}
    st = {}
    P.adam_step(params, g, st, lr=1e-3)
    for k in P.PARAM_ORDER:
        np.testing.assert_allclose(params[k] - before[k], -1e-3 * g[k] / (np.abs(g[k]) + 1e-8), rtol=1e-9, atol=1e-15)


def test_training_reduces_loss():
    params, X, T = _small()
    st = {}
    L0, _ = P.loss_and_grads(params, X, T)
    for _ in range(200):
        L, g = P.loss_and_grads(params, X, T)
        P.adam_step(params, g, st, lr=1e-2)
    assert L < 0.1 * L0


def test_pod_basis():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((50, 4)) @ rng.standard_normal((4, 9))   # rank 4 snapshots
    mean, U, s = P.pod_basis(A, 4)
    np.testing.assert_allclose(U.T @ U, np.eye(4), atol=1e-12)
    C = U.T @ (A - mean[:, None])
    np.testing.assert_allclose(mean[:, None] + U @ C, A, atol=1e-10)
