"""GPU predictor kernels vs the FP64 oracle: forward, gradients (BF16 operands,
FP32 accumulation: per-element error ~1e-2 of the scale, cosine > 0.999),
Adam training, and the POD basis (subspace equal to 1e-10)."""
import numpy as np
import pytest

from oracle import mlp_oracle as P
from paper_2508_06302_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _net(n_in=3, n_h=256, n_out=64, seed=0):
    from paper_2508_06302_gb300 import fse
    params = I.mlp_init(n_in, n_h, n_out, seed=seed)
    rng = np.random.default_rng(seed + 1)
    for k in ("b1", "b2", "b3"):
        params[k] = 0.05 * rng.standard_normal(params[k].shape)
    net = fse.Mlp(n_in, n_h, n_out, max_batch=256)
    net.set_params(params)
    return net, params, rng


def test_forward_and_gradients_match_oracle():
    net, params, rng = _net()
    X = rng.uniform(-1, 1, (40, 3))
    T = 0.3 * rng.standard_normal((40, 64))
    Y = net.forward(X)
    Yr, _ = P.forward(params, X)
    assert np.abs(Y - Yr).max() <= 2e-2 * np.abs(Yr).max()
    loss, g = net.grad(X, T)
    Lr, gr = P.loss_and_grads(params, X, T)
    assert abs(loss - Lr) <= 2e-2 * Lr
    gref = P.flatten(gr)
    cos = float(g @ gref / (np.linalg.norm(g) * np.linalg.norm(gref)))
    assert cos > 0.999, cos
    off = 0
    for k in P.PARAM_ORDER:
        sz = gr[k].size
        blk = g[off:off + sz]
        ref = gr[k].reshape(-1)
        assert np.abs(blk - ref).max() <= 2e-2 * np.abs(ref).max() + 1e-7, k
        off += sz
    net.close()


def test_training_reduces_loss_like_oracle():
    net, params, rng = _net(seed=3)
    X = rng.uniform(-1, 1, (32, 3))
    T = 0.5 * np.sin(X @ rng.standard_normal((3, 64)))
    L0, _ = P.loss_and_grads(params, X, T)
    L = net.train(X, T, steps=300, lr=1e-3)
    ref = {k: v.copy() for k, v in params.items()}
    st = {}
    for _ in range(300):
        _, g = P.loss_and_grads(ref, X, T)
        P.adam_step(ref, g, st, lr=1e-3)
    Lref, _ = P.loss_and_grads(ref, X, T)
    assert L < 0.2 * L0 and Lref < 0.2 * L0
    assert abs(L - Lref) <= 0.3 * Lref + 1e-6
    net.close()


def test_pod_basis_matches_oracle():
    from paper_2508_06302_gb300 import fse
    rng = np.random.default_rng(5)
    S = rng.standard_normal((12, 6)) @ rng.standard_normal((6, 3000)) + 0.01 * rng.standard_normal((12, 3000))
    mean, B, sing = fse.fse_pod_build(S, 5)
    mref, U, sref = P.pod_basis(S.T, 5)
    np.testing.assert_allclose(mean, mref, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(sing, sref, rtol=1e-9)
    # same subspace: the projector difference vanishes
    assert np.abs(B.T @ B - U @ U.T).max() < 1e-10
    np.testing.assert_allclose(B @ B.T, np.eye(5), atol=1e-10)
