"""Continuation (App. C, natural parameter in w_1) through the C ABI: every
accepted torus equals the oracle's torus at the same w_1 (1e-9 relative), and
the learned predictor is compared with the secant predictor on the same sweep."""
import numpy as np
import pytest

from oracle import fse_oracle as O
from paper_2508_06302_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _setup(S1=64):
    from paper_2508_06302_gb300 import fse
    m = I.eb_beam()
    ctx = fse.Context(m, 2, [16], [7], [I.GOLDEN], S1, newton_tol=0, newton_maxit=6)
    return fse, m, ctx


def test_secant_continuation_matches_oracle():
    fse, m, ctx = _setup()
    omegas = m.omega_n1 * np.linspace(1.05, 1.15, 6)
    Z, pts, rc = fse.fse_continue(ctx, omegas, np.zeros(ctx.n_unknowns), rel_tol=1e-11, max_newton=8)
    assert rc == 0 and all(p["status"] == 0 for p in pts)
    prob = O.FSEProblem(m, [16], [7], 64, [I.GOLDEN])
    # the oracle runs its own sweep (zeros, then its own previous solution): no GPU result seeds it
    Zr = np.zeros(ctx.n_unknowns)
    for j, w in enumerate(omegas):
        Zr, hist, ok = O.solve_torus(prob, Zr, w, rel_tol=1e-13, tol=0, maxit=6)
        assert ok
        assert np.linalg.norm(Z[j] - Zr) <= 1e-9 * np.linalg.norm(Zr)
    # the secant predictor is better than the previous point once two points exist
    assert all(p["pred_err"] < 0.5 for p in pts[2:])
    ctx.close()


def test_learned_predictor_vs_secant():
    """The network, trained online on the secant's errors at the accepted points,
    corrects the secant prediction: same tori, a smaller prediction error and no
    more Newton updates than the secant alone on the same sweep."""
    fse, m, ctx = _setup(S1=64)
    omegas = m.omega_n1 * np.linspace(1.06, 1.16, 24)
    Zs, ps, rc1 = fse.fse_continue(ctx, omegas, np.zeros(ctx.n_unknowns), rel_tol=1e-10, max_newton=10)
    net = fse.Mlp(3, 256, 32, max_batch=64)
    net.set_params(I.mlp_init(3, 256, 32, seed=0))
    Zm, pm, rc2 = fse.fse_continue(ctx, omegas, np.zeros(ctx.n_unknowns), predictor="mlp", mlp=net,
                                   rel_tol=1e-10, max_newton=10, warmup=6, pod_modes=32, pod_every=1,
                                   train_steps=300, lr=2e-3)
    assert rc1 == 0 and rc2 == 0
    # both sweeps land on the same tori
    assert np.abs(Zs - Zm).max() <= 1e-8 * np.abs(Zs).max()
    used = [j for j, p in enumerate(pm) if p["predictor"] == fse.FSE_PRED_MLP]
    assert len(used) >= 15
    e_mlp = np.array([pm[j]["pred_err"] for j in used])
    e_sec = np.array([ps[j]["pred_err"] for j in used])
    it_mlp = sum(pm[j]["newton_iters"] for j in used)
    it_sec = sum(ps[j]["newton_iters"] for j in used)
    print("learned correction: median rel. prediction error %.2e, Newton updates %d; secant: %.2e, %d"
          % (np.median(e_mlp), it_mlp, np.median(e_sec), it_sec))
    assert np.median(e_mlp) < np.median(e_sec) / 3
    assert it_mlp <= it_sec
    net.close()
    ctx.close()
