"""The benchmarked form -- FP64 state and residual, FP32 sensitivities, chord or full
Newton with a dense or GMRES outer solve, secant or learned predictor -- converges
to the FP64 oracle's tori (Sec. 3.3 step 6, App. C acceptance at ||R|| <= eps ||Z||).

The oracle solves every torus from its own start (zeros, then its own previous
solution): nothing computed by the GPU seeds it.  Required:
||Z_gpu - Z_oracle|| / ||Z_oracle|| <= 1e-9 with both converged to ||R|| / ||Z|| <= 1e-12.
"""
import numpy as np
import pytest

from oracle import fse_oracle as O
from paper_2508_06302_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-9


def _fse():
    from paper_2508_06302_gb300 import fse
    fse.load()
    return fse


def _oracle_sweep(prob, omegas, maxit):
    """The oracle's own natural-parameter continuation: point 0 from zeros, later points
    from the secant of its own last two solutions."""
    out = []
    for j, w in enumerate(omegas):
        if j == 0:
            Z0 = np.zeros(2 * prob.n * prob.U)
        elif j == 1:
            Z0 = out[0]
        else:
            t = (w - omegas[j - 1]) / (omegas[j - 1] - omegas[j - 2])
            Z0 = out[j - 1] + t * (out[j - 1] - out[j - 2])
        Z, _, ok = O.solve_torus(prob, Z0, w, rel_tol=1e-13, tol=0, maxit=maxit)
        assert ok
        out.append(Z)
    return np.array(out)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("solver", ["dense", "gmres"])
def test_mixed_newton_from_zero_reaches_the_oracle_torus(solver):
    fse = _fse()
    m = I.eb_beam()
    w1 = 1.1 * m.omega_n1
    prob = O.FSEProblem(m, [16], [7], 64, [I.GOLDEN])
    Zref = _oracle_sweep(prob, [w1], 6)[0]
    ctx = fse.Context(m, 2, [16], [7], [I.GOLDEN], 64, newton_tol=0, newton_maxit=6, precision="mixed_fp32")
    if solver == "gmres":
        ctx.set_linear_solver("gmres", rel_tol=1e-10, restart=30, max_iters=300)
    Z = np.zeros_like(Zref)
    hist = []
    for _ in range(12):
        Z, rn, rc = ctx.newton_step(Z, w1)
        hist.append(rn / max(np.linalg.norm(Z), 1e-300))
        if hist[-1] <= 1e-13:
            break
    R, st, it, rc = ctx.residual_jacobian(Z, w1, want_jacobian=False)
    print("mixed %s Newton: ||R||/||Z|| history %s, error vs oracle %.2e"
          % (solver, ["%.1e" % h for h in hist], _rel(Z, Zref)))
    assert np.linalg.norm(R) <= 1e-12 * np.linalg.norm(Z)
    assert _rel(Z, Zref) <= TOL
    ctx.close()


def test_mixed_learned_continuation_matches_oracle_beam():
    """Beam sweep in the benchmarked precision with the learned predictor: every point
    the oracle solves on its own equals the GPU's."""
    fse = _fse()
    m = I.eb_beam()
    ctx = fse.Context(m, 2, [16], [7], [I.GOLDEN], 64, newton_tol=0, newton_maxit=6, precision="mixed_fp32")
    omegas = m.omega_n1 * np.linspace(1.06, 1.14, 12)
    net = fse.Mlp(3, 256, 16, max_batch=64)
    net.set_params(I.mlp_init(3, 256, 16, seed=0))
    Z, pts, rc = fse.fse_continue(ctx, omegas, np.zeros(ctx.n_unknowns), predictor="mlp", mlp=net,
                                  rel_tol=1e-12, max_newton=16, warmup=4, pod_modes=16, pod_every=1,
                                  train_steps=200, lr=2e-3)
    assert rc == 0 and all(p["status"] == 0 for p in pts)
    assert sum(p["predictor"] == fse.FSE_PRED_MLP for p in pts) >= 6
    prob = O.FSEProblem(m, [16], [7], 64, [I.GOLDEN])
    Zr = _oracle_sweep(prob, omegas, 6)
    errs = [_rel(Z[j], Zr[j]) for j in range(len(omegas))]
    print("beam mixed + learned: max error vs oracle %.2e" % max(errs))
    assert max(errs) <= TOL
    net.close()
    ctx.close()


def test_mixed_chord_gmres_learned_continuation_matches_oracle_shell90():
    """The 90-dof flat shell (Q4 membrane + ACM plate, cubic springs between neighbours),
    converged the way the benchmark does it: FP32 tangents, chord corrector, GMRES outer
    solve, learned predictor."""
    fse = _fse()
    m = I.flat_shell(nx=6, ny=4)
    S, H, S1 = [5], [2], 20
    ctx = fse.Context(m, 2, S, H, [I.GOLDEN], S1, newton_tol=0, newton_maxit=8, precision="mixed_fp32")
    ctx.set_linear_solver("gmres", rel_tol=1e-10, restart=40, max_iters=400)
    omegas = m.omega_n1 * np.linspace(0.95, 1.03, 9)
    net = fse.Mlp(3, 256, 8, max_batch=64)
    net.set_params(I.mlp_init(3, 256, 8, seed=0))
    Z, pts, rc = fse.fse_continue(ctx, omegas, np.zeros(ctx.n_unknowns), predictor="mlp", mlp=net,
                                  rel_tol=1e-12, max_newton=40, warmup=4, pod_modes=8, pod_every=1,
                                  train_steps=200, lr=2e-3, chord=True)
    assert rc == 0 and all(p["status"] == 0 for p in pts)
    prob = O.FSEProblem(m, S, H, S1, [I.GOLDEN])
    Zr = _oracle_sweep(prob, omegas, 8)
    errs = [_rel(Z[j], Zr[j]) for j in range(len(omegas))]
    print("shell90 mixed + chord + GMRES + learned: max error vs oracle %.2e, updates %s"
          % (max(errs), [p["newton_iters"] for p in pts]))
    assert max(errs) <= TOL
    net.close()
    ctx.close()
