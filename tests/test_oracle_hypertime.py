"""Pins of the hyper-time oracle (Sec. 3.4, Eq. FSES_T) against the multi-frequency form
(Eq. 16, 22), with more samples than coefficients (S~ > U~, the case the hyper-time form admits)."""
import numpy as np

from oracle import fse_oracle as O
from oracle import hypertime as HT
from paper_2508_06302_gb300 import inputs as I


def _beam_problem():
    m = I.eb_beam()
    return m, O.FSEProblem(m, [11], [3], 48, [I.GOLDEN]), 1.1 * m.omega_n1


def _to_samples(prob, Z):
    """(I_2n (x) Gamma) Z in the (S~, 2n) layout of the hyper-time unknowns (Eq. 20)."""
    return (np.asarray(Z).reshape(2 * prob.n, prob.U) @ prob.G.T).T


def test_hypertime_residual_and_jacobian_are_gamma_images_of_eq16():
    """R_T(Gamma Z) = Gamma R(Z), and J_T (I (x) Gamma) = (I (x) Gamma) J (chain rule)."""
    m, prob, w1 = _beam_problem()
    assert prob.N > prob.U
    Z = I.random_coeffs(m.n, prob.U, 1e-3, seed=2)
    rj = O.residual_jacobian(prob, Z, w1, want_jacobian=True, dense=True, tol=0, maxit=8)
    RT, JT = HT.residual_jacobian_hypertime(prob, _to_samples(prob, Z), w1, True, tol=0, maxit=8)
    GR = _to_samples(prob, rj.R)
    np.testing.assert_allclose(RT, GR, rtol=0, atol=1e-12 * np.abs(GR).max())
    V = np.random.default_rng(4).standard_normal(Z.size)
    lhs = (JT @ _to_samples(prob, V).reshape(-1)).reshape(prob.N, 2 * m.n)
    rhs = _to_samples(prob, rj.J @ V)
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-11 * np.abs(rhs).max())


def test_hypertime_newton_lands_on_the_eq16_torus():
    m, prob, w1 = _beam_problem()
    Zref, hist, ok = O.solve_torus(prob, np.zeros(2 * m.n * prob.U), w1, rel_tol=1e-12, tol=1e-13, maxit=30)
    assert ok
    zb, hist_t, ok_t = HT.solve_hypertime(prob, np.zeros((prob.N, 2 * m.n)), w1, rel_tol=1e-12)
    assert ok_t and len(hist_t) <= 8, hist_t
    ref = _to_samples(prob, Zref)
    np.testing.assert_allclose(zb, ref, rtol=0, atol=1e-9 * np.abs(ref).max())
