"""Pins of the unknown-base-frequency oracle (Sec. 3.2: Eq. Cont1, Eq. 18, 19, 23, 24) and of the
self-excited (van der Pol) test element it is exercised on."""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import fse_oracle as O
from oracle import unknown_freq as UF
from paper_2508_06302_gb300 import inputs as I

WN = 10.0                  # natural frequency of the van der Pol test model [rad/s]
W1 = WN / 2.7              # forcing frequency: rotation number near 2.7, no low-order locking


def _random_problem(H, n=2, seed=0):
    m = I.chain(n)
    S = [2 * h + 1 + 2 for h in H]
    prob = O.FSEProblem(m, S, H, 16, [0.3] * len(H))
    Z = np.random.default_rng(seed).standard_normal(2 * n * prob.U)
    return prob, Z


@pytest.mark.parametrize("H", [[3], [2, 1]])
def test_nabla_is_the_phase_derivative(H):
    """(I (x) grad_i) Z of Eq. (19) holds the coefficients of dz/dphi_i: central differences of
    the trigonometric interpolant along phi_i."""
    prob, Z = _random_problem(H)
    phi = np.array([0.7, -1.9][:len(H)])
    h = 1e-5
    for j in range(len(H)):
        e = np.zeros(len(H))
        e[j] = h
        fd = (UF.torus_point(prob, Z, phi + e) - UF.torus_point(prob, Z, phi - e)) / (2 * h)
        an = UF.torus_point(prob, UF.phase_gradient(prob, Z, j), phi)
        np.testing.assert_allclose(an, fd, rtol=0, atol=1e-8 * np.abs(an).max())


@pytest.mark.parametrize("H", [[3], [2, 1]])
def test_rotation_derivative_matches_fd(H):
    """dR(rho)/dw_i of Eq. (24) with rho_i = w_i / w_1: central differences of R(rho)."""
    ktab = O.harmonic_table(H)
    rho = np.array([0.61, 1.37][:len(H)])
    w1 = 3.3
    h = 1e-6
    for j in range(len(H)):
        e = np.zeros(len(H))
        e[j] = h / w1                      # d rho_j = d w_{j+2} / w_1
        fd = (O.rotation(ktab, rho + e) - O.rotation(ktab, rho - e)) / (2 * h)
        np.testing.assert_allclose(UF.drotation_domega(ktab, rho, w1, j), fd, rtol=0, atol=1e-8)


def test_vdp_force_and_tangents_fd():
    m = I.van_der_pol(omega_n=WN, eps=0.3)
    q, qd = np.array([1.3]), np.array([-4.1])
    f, Kt, Ct = O.fnl_and_tangent(m, q, qd)
    c = 0.3 * WN
    assert abs(f[0] - c * (q[0] ** 2 - 1.0) * qd[0]) <= 1e-14 * abs(f[0])
    h = 1e-6
    fq = (O.fnl_and_tangent(m, q + h, qd)[0] - O.fnl_and_tangent(m, q - h, qd)[0]) / (2 * h)
    fv = (O.fnl_and_tangent(m, q, qd + h)[0] - O.fnl_and_tangent(m, q, qd - h)[0]) / (2 * h)
    np.testing.assert_allclose(Kt[0, 0], fq[0], rtol=1e-8)
    np.testing.assert_allclose(Ct[0, 0], fv[0], rtol=1e-8)


def test_dR_domega_of_an_unknown_frequency_matches_fd():
    """Eq. (23), i > e: the trajectories do not move with w_2 (bit-identical Z(2 pi)) and dR/dw_2
    is the rotation term, checked against central differences of R."""
    m = I.van_der_pol(omega_n=WN, eps=0.2, F=(10.0,))
    S, H, S1 = [8], [3], 48
    rho = np.array([2.7])
    U = 2 * H[0] + 1
    Z = np.random.default_rng(3).standard_normal(2 * U) * 0.3
    prob, rj, cols = UF.residual_unknown(m, S, H, S1, rho, Z, W1, [0], tol=0, maxit=8)
    h = 1e-6
    Rp = O.residual_jacobian(O.FSEProblem(m, S, H, S1, rho + h / W1), Z, W1, want_jacobian=False, tol=0, maxit=8)
    Rm = O.residual_jacobian(O.FSEProblem(m, S, H, S1, rho - h / W1), Z, W1, want_jacobian=False, tol=0, maxit=8)
    assert np.array_equal(Rp.Z2pi, rj.Z2pi) and np.array_equal(Rm.Z2pi, rj.Z2pi)
    fd = (Rp.R - Rm.R) / (2 * h)
    np.testing.assert_allclose(cols[0], fd, rtol=0, atol=1e-7 * np.abs(cols[0]).max())


def test_free_linear_oscillator_rotation_number_closed_form():
    """Undamped linear oscillator, no forcing: Newmark (average acceleration) turns the state
    by alpha = 2 atan(nu Delta / 2) per step (nu = w_n / w_1, Delta = 2 pi / S1) with
    u = -nu A sin, so the torus z(0, phi_2) = [A cos phi_2; -nu A sin phi_2] solves Eq. (16)
    exactly at rho = S1 alpha / (2 pi); any other rho leaves a residual."""
    m = I.van_der_pol(omega_n=WN, eps=0.0, F=(0.0,))
    S, H, S1 = [5], [2], 64
    nu = WN / W1
    rho_star = S1 * 2.0 * math.atan(nu * math.pi / S1) / (2.0 * math.pi)
    A = 1.7
    U = 2 * H[0] + 1
    C = np.zeros((2, U))
    C[0, 1] = A
    C[1, 2] = -nu * A
    Z = C.reshape(-1)
    R = O.residual_jacobian(O.FSEProblem(m, S, H, S1, [rho_star]), Z, W1, want_jacobian=False, tol=1e-14,
                            maxit=5).R
    assert np.linalg.norm(R) <= 1e-12 * np.linalg.norm(Z)
    R2 = O.residual_jacobian(O.FSEProblem(m, S, H, S1, [rho_star + 1e-3]), Z, W1, want_jacobian=False,
                             tol=1e-14, maxit=5).R
    assert np.linalg.norm(R2) >= 1e-3 * np.linalg.norm(Z)


def test_residual_is_equivariant_under_sample_shifts():
    """With no forcing along phi_2 (e = 1) a torus shifted by one sample spacing is the same
    set of trajectories: R(S Z) = S R(Z) with S = expm(theta grad_2) (Eq. 19), theta = 2 pi / S_2."""
    m = I.van_der_pol(omega_n=WN, eps=0.2, F=(10.0,))
    S, H, S1 = [7], [3], 40
    prob = O.FSEProblem(m, S, H, S1, [2.7])
    Z = np.random.default_rng(11).standard_normal(2 * prob.U) * 0.5
    Sh = scipy.linalg.expm((2.0 * np.pi / S[0]) * UF.nabla_phi(prob.ktab, 0))
    shift = lambda v: (v.reshape(2, prob.U) @ Sh.T).reshape(-1)
    R = O.residual_jacobian(prob, Z, W1, want_jacobian=False, tol=0, maxit=8).R
    Rs = O.residual_jacobian(prob, shift(Z), W1, want_jacobian=False, tol=0, maxit=8).R
    np.testing.assert_allclose(Rs, shift(R), rtol=0, atol=1e-11 * np.abs(R).max())


def test_vdp_torus_with_unknown_frequency_against_brute_force():
    """Forced van der Pol oscillator (d = 2, e = 1): w_2, the frequency of the self-excited
    motion, is an unknown.  Newton on Eq. (Cont1) with the phase condition of Eq. (18) from the
    first-harmonic guess (amplitude 2, w_2 = w_n) converges quadratically; at the solution J
    nearly annihilates the phase direction (the reason for the condition); and a long integration from
    two points of the solved torus lands, after 20 periods of w_1, on the torus rotated by
    20 * 2 pi rho (Eq. 16), which pins both the torus and its rotation number."""
    m = I.van_der_pol(omega_n=WN, eps=0.2, F=(10.0,))
    S, H, S1 = [24], [9], 256
    U = 2 * H[0] + 1
    rho0 = np.array([WN / W1])
    C = np.zeros((2, U))
    C[0, 0] = 10.0 / (WN ** 2 - W1 ** 2)       # forced linear response at phi_1 = 0
    C[0, 1] = 2.0                              # limit cycle, first harmonic
    C[1, 2] = -2.0 * rho0[0]
    Z, rho, hist, ok = UF.solve_torus_unknown(m, S, H, S1, rho0, C.reshape(-1), W1, [0], rel_tol=1e-11,
                                              max_newton=10)
    assert ok and len(hist) <= 8, hist
    # measured 0.99699: 1 - eps^2/16 (Lindstedt) less the Newmark period elongation at ~95 steps a cycle
    assert 0.9960 < rho[0] * W1 / WN < 0.9980, rho[0] * W1 / WN
    prob, rj, cols = UF.residual_unknown(m, S, H, S1, rho, Z, W1, [0], tol=1e-12, maxit=30)
    # a continuous phase shift is a symmetry of the truncated torus only up to its truncation
    # (sample shifts are exact, see the equivariance test): measured 3.9e-7, a random direction ~1
    g = UF.phase_gradient(prob, Z, 0)
    nJ = np.linalg.norm(rj.J, 2)
    assert np.linalg.norm(rj.J @ g) <= 1e-5 * nJ * np.linalg.norm(g)
    v = np.random.default_rng(2).standard_normal(g.size)
    assert np.linalg.norm(rj.J @ v) >= 1e-2 * nJ * np.linalg.norm(v)
    for phi0 in (0.0, 1.3):
        z0 = UF.torus_point(prob, Z, [phi0])
        k = 20
        tr = O.integrate_trajectory(m, W1, rho, np.array([phi0]), z0[:1], z0[1:], S1, tol=1e-13, maxit=30,
                                    sens=False, n_steps=k * S1)
        zk = UF.torus_point(prob, Z, [phi0 + 2.0 * np.pi * k * rho[0]])
        assert np.abs(tr.zT - zk).max() <= 3e-5 * np.abs(zk).max(), np.abs(tr.zT - zk).max()


def test_dR_domega1_with_the_unknown_frequency_held_fixed_matches_fd():
    """dR/dw_1 at fixed w_2 (unknown of its own): the integration term plus the rotation term of
    rho_2 = w_2 / w_1 (Eq. 23, 24), against central differences of R in w_1 with w_2 fixed."""
    m = I.van_der_pol(omega_n=WN, eps=0.2, F=(10.0,))
    S, H, S1 = [8], [3], 48
    rho = np.array([2.7])
    w2 = rho[0] * W1
    U = 2 * H[0] + 1
    Z = np.random.default_rng(4).standard_normal(2 * U) * 0.3
    prob, rj, cols = UF.residual_unknown(m, S, H, S1, rho, Z, W1, [0], tol=0, maxit=8)
    an = UF.dR_domega1_unknown(prob, rj, W1, [0])
    h = 1e-6 * W1
    R = {}
    for sgn in (1, -1):
        w1 = W1 + sgn * h
        R[sgn] = O.residual_jacobian(O.FSEProblem(m, S, H, S1, [w2 / w1]), Z, w1, want_jacobian=False, tol=0,
                                     maxit=8).R
    fd = (R[1] - R[-1]) / (2 * h)
    np.testing.assert_allclose(an, fd, rtol=0, atol=1e-6 * np.abs(an).max())
    # the rotation term matters: dropping it misses the derivative
    assert np.abs(rj.dR_dw - fd).max() > 1e-3 * np.abs(fd).max()
