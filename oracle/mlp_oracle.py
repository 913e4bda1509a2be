"""FP64 CPU oracle of the learned continuation predictor (test infrastructure only).

The predictor is not part of the paper: it maps the normalised point
parameters x = (w_1, w_2, F_1) to the coefficients c of the torus in a POD
basis of converged solutions, Z ~ Zbar + Phi_pod c, and is trained on the
solutions the shooting method itself produces.

* MLP: x -> gelu(W1 x + b1) -> gelu(W2 h1 + b2) -> W3 h2 + b3, with the exact
  GELU gelu(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2.
* loss L = 1/(2B) sum_b sum_o (y_bo - t_bo)^2 over a batch of B samples.
* Adam (Kingma and Ba 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
  p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
* POD: thin SVD of the mean-centred snapshot matrix; the first r left
  singular vectors form Phi_pod.

The gradients are pinned by central finite differences of the loss
(tests/test_oracle_mlp.py).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

PARAM_ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(params, X):
    """Returns the output (B x n_out) and the cache of pre-activations/activations."""
    z1 = X @ params["W1"].T + params["b1"]
    h1 = gelu(z1)
    z2 = h1 @ params["W2"].T + params["b2"]
    h2 = gelu(z2)
    y = h2 @ params["W3"].T + params["b3"]
    return y, (X, z1, h1, z2, h2)


def loss_and_grads(params, X, T):
    """L = 1/(2B) sum (y - t)^2 and dL/dparams by backpropagation."""
    B = X.shape[0]
    y, (X_, z1, h1, z2, h2) = forward(params, X)
    r = y - T
    L = 0.5 * float(np.sum(r * r)) / B
    dy = r / B
    g = {}
    g["W3"] = dy.T @ h2
    g["b3"] = dy.sum(axis=0)
    dh2 = dy @ params["W3"]
    dz2 = dh2 * gelu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ params["W2"]
    dz1 = dh1 * gelu_grad(z1)
    g["W1"] = dz1.T @ X_
    g["b1"] = dz1.sum(axis=0)
    return L, g


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; state holds m, v and the step count t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in PARAM_ORDER:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m[...] = beta1 * m + (1 - beta1) * grads[k]
        v[...] = beta2 * v + (1 - beta2) * grads[k] ** 2
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return params


def flatten(params):
    return np.concatenate([params[k].reshape(-1) for k in PARAM_ORDER])


def pod_basis(snapshots, r):
    """Mean and the r leading left singular vectors of the centred snapshots (columns)."""
    mean = snapshots.mean(axis=1)
    U, s, _ = np.linalg.svd(snapshots - mean[:, None], full_matrices=False)
    return mean, U[:, :r], s[:r]
