"""FSE-Shooting in the hyper-time domain (Sec. 3.4, Eq. FSES_T) through the C ABI, against the
FP64 oracle: the residual R_T and the products J_T v at the same start points (1e-10
relative), and a Newton solve from zero start points that lands on Gamma times the oracle's
Eq. (16) torus (1e-9 relative), with more samples than coefficients (S~ = 11 > U~ = 7)."""
import numpy as np
import pytest

from oracle import fse_oracle as O
from oracle import hypertime as HT
from paper_2508_06302_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _fse():
    from paper_2508_06302_gb300 import fse
    fse.load()
    return fse


def _beam():
    m = I.eb_beam()
    return m, O.FSEProblem(m, [11], [3], 48, [I.GOLDEN]), 1.1 * m.omega_n1


def _to_samples(prob, Z):
    return (np.asarray(Z).reshape(2 * prob.n, prob.U) @ prob.G.T).T


@pytest.mark.parametrize("precision,tol_j", [("fp64", 1e-10), ("mixed_fp32", 1e-3)])
def test_hypertime_residual_and_products_match_oracle(precision, tol_j):
    m, prob, w1 = _beam()
    assert prob.N > prob.U
    rng = np.random.default_rng(3)
    zb = 1e-3 * rng.standard_normal((prob.N, 2 * m.n))
    RT_ref, JT_ref = HT.residual_jacobian_hypertime(prob, zb, w1, True, tol=0, maxit=8)
    fse = _fse()
    ctx = fse.Context(m, 2, [11], [3], [I.GOLDEN], 48, newton_tol=0, newton_maxit=8, precision=precision)
    RT, st, it, rc = ctx.residual_jacobian_hypertime(zb, w1, want_jacobian=True)
    assert rc == 0
    e_R = np.linalg.norm(RT - RT_ref) / (np.linalg.norm(zb) + np.linalg.norm(RT_ref))
    V = rng.standard_normal((3, prob.N, 2 * m.n))
    JV = ctx.jacobian_apply_hypertime(V)
    JV_ref = np.array([(JT_ref @ v.reshape(-1)).reshape(prob.N, 2 * m.n) for v in V])
    e_J = np.linalg.norm(JV - JV_ref) / np.linalg.norm(JV_ref)
    print("hyper-time %s: R_T %.2e, J_T v %.2e" % (precision, e_R, e_J))
    assert e_R <= 1e-10
    assert e_J <= tol_j
    # the Eq. (16) form of the same context: R_T(Gamma Z) = Gamma R(Z)
    Z = I.random_coeffs(m.n, prob.U, 1e-3, seed=2)
    R16, _, _, _ = ctx.residual_jacobian(Z, w1, want_jacobian=False)
    RT2, _, _, _ = ctx.residual_jacobian_hypertime(_to_samples(prob, Z), w1, want_jacobian=False)
    GR = _to_samples(prob, R16)
    assert np.abs(RT2 - GR).max() <= 1e-12 * np.abs(GR).max()
    ctx.close()


@pytest.mark.parametrize("precision,solver", [("fp64", "dense"), ("mixed_fp32", "dense"), ("mixed_fp32", "gmres")])
def test_hypertime_newton_lands_on_the_eq16_torus(precision, solver):
    m, prob, w1 = _beam()
    Zref, hist, ok = O.solve_torus(prob, np.zeros(2 * m.n * prob.U), w1, rel_tol=1e-13, tol=0, maxit=8)
    assert ok
    ref = _to_samples(prob, Zref)
    fse = _fse()
    ctx = fse.Context(m, 2, [11], [3], [I.GOLDEN], 48, newton_tol=0, newton_maxit=8, precision=precision)
    if solver == "gmres":
        ctx.set_linear_solver("gmres", rel_tol=1e-11, restart=60, max_iters=600)
    zb = np.zeros((prob.N, 2 * m.n))
    norms = []
    for _ in range(12):
        zb, rn, rc = ctx.newton_step_hypertime(zb, w1)
        norms.append(rn)
        if rn <= 1e-13 * np.linalg.norm(zb):
            break
    err = np.linalg.norm(zb - ref) / np.linalg.norm(ref)
    print("hyper-time Newton %s/%s: ||R_T|| %s, error vs Gamma Z_oracle %.2e"
          % (precision, solver, ["%.1e" % x for x in norms], err))
    assert err <= 1e-9
    ctx.close()
