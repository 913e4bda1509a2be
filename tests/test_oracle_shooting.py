"""Pins of the oracle's shooting residual, Jacobian (Eq. 16, 22, 23), Newton and Lyapunov (App. F)."""
import math

import numpy as np
import pytest

from oracle import fse_oracle as O
from paper_2508_06302_gb300 import inputs as I


def _small_problem(d=2):
    m = I.chain(4)
    if d == 2:
        return O.FSEProblem(m, [5], [2], 16, [I.GOLDEN]), 1.15 * m.omega_n1
    m3 = I.chain(3, F=(1.0, 0.5, 0.4))
    return O.FSEProblem(m3, [3, 3], [1, 1], 12, [math.sqrt(2), math.sqrt(3)]), 1.1 * m3.omega_n1


@pytest.mark.parametrize("d", [2, 3])
def test_dense_jacobian_matches_fd(d):
    prob, w1 = _small_problem(d)
    rng = np.random.default_rng(0)
    Z = 1e-3 * rng.standard_normal(2 * prob.n * prob.U)
    rj = O.residual_jacobian(prob, Z, w1, tol=0, maxit=8)
    h = 1e-7
    Jfd = np.zeros_like(rj.J)
    for j in range(Z.size):
        e = np.zeros_like(Z)
        e[j] = h
        rp = O.residual_jacobian(prob, Z + e, w1, want_jacobian=False, tol=0, maxit=8).R
        rm = O.residual_jacobian(prob, Z - e, w1, want_jacobian=False, tol=0, maxit=8).R
        Jfd[:, j] = (rp - rm) / (2 * h)
    np.testing.assert_allclose(rj.J, Jfd, rtol=1e-5, atol=1e-6 * np.abs(rj.J).max())
    hw = 1e-6 * w1
    rp = O.residual_jacobian(prob, Z, w1 + hw, want_jacobian=False, tol=0, maxit=8).R
    rm = O.residual_jacobian(prob, Z, w1 - hw, want_jacobian=False, tol=0, maxit=8).R
    np.testing.assert_allclose(rj.dR_dw, (rp - rm) / (2 * hw), rtol=1e-5,
                               atol=1e-6 * np.abs(rj.dR_dw).max())
    v = rng.standard_normal(Z.size)
    np.testing.assert_allclose(O.jacobian_apply(prob, rj.Phi, v), rj.J @ v, rtol=1e-11, atol=1e-11)


def test_linear_jacobian_is_kronecker():
    """f_nl = 0: Phi_s = Phi for all s, so J = Phi (x) R - I in state-major order."""
    m = I.chain(3).linear_only()
    prob = O.FSEProblem(m, [5], [2], 16, [0.41])
    rj = O.residual_jacobian(prob, np.zeros(2 * 3 * 5), 1.1 * m.omega_n1, tol=0, maxit=2)
    np.testing.assert_allclose(rj.J, np.kron(rj.Phi[0], prob.R) - np.eye(30), atol=1e-12)


def test_periodic_special_case_is_classical_shooting():
    """F_2 = 0 (Sec. 3.1, d = 1 reduction): only the constant harmonic survives, and it is the
    fixed point of the one-period Newmark map, i.e. the steady state of a long run."""
    m = I.chain(4, F=(2.0, 0.0), c=3.0)
    w1 = 1.2 * m.omega_n1
    prob = O.FSEProblem(m, [5], [2], 32, [I.GOLDEN])
    Z, hist, ok = O.solve_torus(prob, np.zeros(2 * 4 * 5), w1, rel_tol=1e-12)
    assert ok
    C = Z.reshape(8, 5)
    assert np.abs(C[:, 1:]).max() <= 1e-10 * np.abs(C[:, 0]).max()
    tr = O.integrate_trajectory(m, w1, prob.rho, np.array([0.0]), np.zeros(4), np.zeros(4), 32,
                                tol=0, maxit=6, sens=False, n_steps=32 * 400)
    np.testing.assert_allclose(tr.zT, C[:, 0], rtol=1e-7, atol=1e-9 * np.abs(C[:, 0]).max())


def test_nonlinear_torus_brute_force():
    """A long Newmark run started on the computed torus at an off-grid phase stays on it:
    after m periods the state equals H(phi0 + 2 pi m rho) Z (Eq. 7, Eq. 12)."""
    m = I.eb_beam()
    w1 = 1.1 * m.omega_n1
    prob = O.FSEProblem(m, [16], [7], 128, [I.GOLDEN])
    Z, hist, ok = O.solve_torus(prob, np.zeros(2 * m.n * prob.U), w1, rel_tol=1e-12)
    assert ok
    C = Z.reshape(2 * m.n, prob.U)
    phi0 = 0.123
    z0 = C @ O.basis_row(prob.ktab, np.array([phi0]))
    for periods in (1, 5):
        tr = O.integrate_trajectory(m, w1, prob.rho, np.array([phi0]), z0[:m.n], z0[m.n:], 128,
                                    tol=0, maxit=6, sens=False, n_steps=128 * periods)
        zt = C @ O.basis_row(prob.ktab, np.array([phi0 + 2 * math.pi * periods * prob.rho[0]]))
        assert np.linalg.norm(tr.zT - zt) <= 1e-8 * np.linalg.norm(zt)
    # a nearby non-solution drifts off the torus by far more
    Cb = C.copy()
    Cb[:, 1] *= 1.01
    z0b = Cb @ O.basis_row(prob.ktab, np.array([phi0]))
    tr = O.integrate_trajectory(m, w1, prob.rho, np.array([phi0]), z0b[:m.n], z0b[m.n:], 128,
                                tol=0, maxit=6, sens=False)
    zt = Cb @ O.basis_row(prob.ktab, np.array([phi0 + 2 * math.pi * prob.rho[0]]))
    assert np.linalg.norm(tr.zT - zt) > 1e-5 * np.linalg.norm(zt)


def test_newton_quadratic_convergence():
    m = I.eb_beam()
    w1 = 1.1 * m.omega_n1
    prob = O.FSEProblem(m, [16], [7], 128, [I.GOLDEN])
    Z, hist, ok = O.solve_torus(prob, np.zeros(2 * m.n * prob.U), w1, rel_tol=1e-12)
    assert ok and len(hist) <= 5
    assert hist[2] <= 1e-2 * hist[1] ** 1.5 / hist[0] ** 0.5 or hist[2] < 1e-14


def _linear_lyap_setup(damped=True):
    m = I.chain(3).linear_only()
    if not damped:
        m.D = np.zeros_like(m.D)
    prob = O.FSEProblem(m, [5], [2], 16, [0.3819660112501051])
    w1 = 1.1 * m.omega_n1
    rj = O.residual_jacobian(prob, np.zeros(30), w1, tol=0, maxit=2, dense=False)
    return prob, w1, rj


def test_lyapunov_linear_equals_floquet():
    """f_nl = 0: exponents are (1/T1) ln|mu_j(Phi)|, sorted descending (App. F)."""
    prob, w1, rj = _linear_lyap_setup()
    T1 = 2 * math.pi / w1
    mu = np.sort(np.log(np.abs(np.linalg.eigvals(rj.Phi[0]))))[::-1] / T1
    # equal-modulus pairs make the finite-time values converge like 1/N_Ly
    sig = O.lyapunov(prob, rj.Phi, w1, N_Ly=20000, h=6)
    np.testing.assert_allclose(sig, mu, atol=0.03 * np.abs(mu).max())
    assert sig.sum() == pytest.approx(mu.sum(), rel=1e-9)


def test_lyapunov_undamped_linear_is_zero():
    """Undamped trapezoid map has |mu| = 1, so every exponent vanishes."""
    prob, w1, rj = _linear_lyap_setup(damped=False)
    s1 = O.lyapunov(prob, rj.Phi, w1, N_Ly=400, h=6)
    s2 = O.lyapunov(prob, rj.Phi, w1, N_Ly=4000, h=6)
    assert abs(s1.sum()) < 1e-9 and abs(s2.sum()) < 1e-9
    assert np.abs(s2).max() < 0.2 * np.abs(s1).max()      # O(1/N_Ly) finite-time bias


def test_lyapunov_sum_is_log_det():
    """sum_h sigma_h = (1 / (N_Ly T1)) sum_i ln|det Psi(phi~^{i-1})| for h = 2n."""
    m = I.chain(3)
    prob = O.FSEProblem(m, [5], [2], 16, [I.GOLDEN])
    w1 = 1.1 * m.omega_n1
    rng = np.random.default_rng(1)
    rj = O.residual_jacobian(prob, 1e-2 * rng.standard_normal(30), w1, tol=0, maxit=8, dense=False)
    NL = 50
    sig = O.lyapunov(prob, rj.Phi, w1, N_Ly=NL, h=6)
    dvec = np.concatenate([np.ones(3), w1 * np.ones(3)])
    Psi = rj.Phi * dvec[None, :, None] / dvec[None, None, :]
    coef = np.einsum('us,sij->uij', prob.Gi, Psi)
    tot = 0.0
    for i in range(1, NL + 1):
        Hrow = O.basis_row(prob.ktab, 2 * (i - 1) * math.pi * prob.rho)
        tot += math.log(abs(np.linalg.det(np.einsum('u,uij->ij', Hrow, coef))))
    assert sig.sum() == pytest.approx(tot / (NL * 2 * math.pi / w1), rel=1e-10, abs=1e-10)
