"""Pins of the oracle's Newmark / Newton / sensitivity code (App. E) and f_nl."""
import math

import numpy as np
import pytest

from oracle import fse_oracle as O
from paper_2508_06302_gb300 import inputs as I


def _fd_tangent(model, q, h=1e-7):
    n = q.shape[0]
    Kfd = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = h * max(1.0, abs(q[j]))
        fp, _, _ = O.fnl_and_tangent(model, q + e, np.zeros(n))
        fm, _, _ = O.fnl_and_tangent(model, q - e, np.zeros(n))
        Kfd[:, j] = (fp - fm) / (2 * e[j])
    return Kfd


@pytest.mark.parametrize("maker", [lambda: I.chain(6), lambda: I.vk_beam(n_el=6),
                                   lambda: I.flat_shell(nx=4, ny=3)])
def test_tangent_matches_fd(maker):
    m = maker()
    rng = np.random.default_rng(0)
    q = 1e-2 * rng.standard_normal(m.n)
    _, Kt, Ct = O.fnl_and_tangent(m, q, np.zeros(m.n))
    np.testing.assert_allclose(Kt, _fd_tangent(m, q), rtol=1e-6, atol=1e-6 * np.abs(Kt).max())
    assert np.all(Ct == 0)


def _vk_energy(EA, L, loc, npts=24):
    """EA/2 int (u' w'^2 + w'^4/4) dx by a 24-point rule, Hermite slope written out directly."""
    x, w = np.polynomial.legendre.leggauss(npts)
    du = (loc[3] - loc[0]) / L
    E = 0.0
    for xi, wi in zip(x, w):
        s = 0.5 * (xi + 1)
        wp = ((6 * s * s - 6 * s) * loc[1] + L * (1 - 4 * s + 3 * s * s) * loc[2]
              + (6 * s - 6 * s * s) * loc[4] + L * (3 * s * s - 2 * s) * loc[5]) / L
        E += 0.5 * L * wi * 0.5 * EA * (du * wp * wp + 0.25 * wp ** 4)
    return E


def test_vk_force_is_energy_gradient():
    """The von Karman element force is the gradient of the stretching energy."""
    m = I.vk_beam(n_el=3)
    rng = np.random.default_rng(1)
    q = 1e-2 * rng.standard_normal(m.n)
    f, _, _ = O.fnl_and_tangent(m, q, np.zeros(m.n))
    g = np.zeros(m.n)
    h = 1e-7
    for e in range(m.n_nl):
        dof = m.nl_dof[e]
        EA, L = m.nl_p[e, 0], m.nl_p[e, 1]
        loc = np.array([q[d] if d >= 0 else 0.0 for d in dof])
        for a in range(6):
            if dof[a] < 0:
                continue
            lp, lm = loc.copy(), loc.copy()
            lp[a] += h
            lm[a] -= h
            g[dof[a]] += (_vk_energy(EA, L, lp) - _vk_energy(EA, L, lm)) / (2 * h)
    np.testing.assert_allclose(f, g, rtol=1e-6, atol=1e-8 * np.abs(f).max())


def _closed_form(m, w1, rho, S1, H):
    """Steady discrete response of the linear Newmark scheme to each forcing component.

    q_k = Re(Q e^{i lam k Delta}) with (K + w s D + w^2 s^2 M) Q = F and
    s = (2i/Delta) tan(lam Delta / 2) solves Eq. (E4)-(E2) exactly for every k.
    """
    n = m.n
    U = O.u_tilde(H)
    Dl = 2 * math.pi / S1

    def resp(lam, F):
        s = 2j / Dl * math.tan(lam * Dl / 2)
        Q = np.linalg.solve(m.K + w1 * s * m.D + w1 ** 2 * s * s * m.M, F)
        return Q, s * Q

    C = np.zeros((2 * n, U))
    Q1, U1 = resp(1.0, m.F[0])
    C[:n, 0], C[n:, 0] = Q1.real, U1.real
    if m.F.shape[0] > 1:
        Q2, U2 = resp(rho[0], m.F[1])
        C[:n, 1], C[n:, 1] = Q2.real, U2.real
        C[:n, 2], C[n:, 2] = -Q2.imag, -U2.imag
    return C.reshape(-1)


@pytest.mark.parametrize("maker,S,H,S1", [(lambda: I.eb_beam(), [16], [7], 128),
                                          (lambda: I.chain(8), [7], [3], 40),
                                          (lambda: I.vk_beam(n_el=8), [9], [4], 32)])
def test_linear_closed_form_is_a_root(maker, S, H, S1):
    m = maker().linear_only()
    w1 = 1.1 * m.omega_n1
    rho = [I.GOLDEN]
    prob = O.FSEProblem(m, S, H, S1, rho)
    Z = _closed_form(m, w1, rho, S1, H)
    rj = O.residual_jacobian(prob, Z, w1, want_jacobian=False, tol=0, maxit=2)
    assert np.linalg.norm(rj.R) <= 1e-11 * np.linalg.norm(Z)
    # a wrong forcing phase, sign or rotation direction is not a root
    rj2 = O.residual_jacobian(O.FSEProblem(m, S, H, S1, [-I.GOLDEN]), Z, w1, want_jacobian=False,
                              tol=0, maxit=2)
    assert np.linalg.norm(rj2.R) > 1e-3 * np.linalg.norm(Z)


def test_newmark_second_order_convergence():
    """Discrete steady amplitude -> continuous one with error ratio ~4 per doubling of S1."""
    m = I.eb_beam().linear_only()
    w1 = 1.1 * m.omega_n1
    Qc = np.linalg.solve(m.K - w1 ** 2 * m.M + 1j * w1 * m.D, m.F[0])
    errs = []
    for S1 in (32, 64, 128, 256):
        Z = _closed_form(m, w1, [I.GOLDEN], S1, [1]).reshape(2 * m.n, 3)
        errs.append(np.linalg.norm(Z[:m.n, 0] - Qc.real))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.7 < r < 4.3 for r in ratios), ratios


def test_discrete_energy_balance():
    """E_{k+1}-E_k = dq.(e_{k+1}+e_k)/2 - dq.(f_{k+1}+f_k)/2 - w Delta/4 (u_{k+1}+u_k).D(u_{k+1}+u_k)."""
    m = I.chain(6, c=0.7)
    w1 = 1.3 * m.omega_n1
    rho = [0.7]
    S1 = 64
    Dl = 2 * math.pi / S1
    rng = np.random.default_rng(2)
    q0 = 1e-3 * rng.standard_normal(m.n)
    u0 = 1e-3 * rng.standard_normal(m.n)
    tr = O.integrate_trajectory(m, w1, rho, np.array([0.3]), q0, u0, S1, tol=0, maxit=8,
                                sens=False, keep_history=True)
    worst = 0.0
    for k in range(S1):
        (q, u, a), (qn, un, an) = tr.history[k], tr.history[k + 1]
        E = lambda q_, u_: 0.5 * w1 ** 2 * u_ @ m.M @ u_ + 0.5 * q_ @ m.K @ q_
        f0, _, _ = O.fnl_and_tangent(m, q, w1 * u)
        f1, _, _ = O.fnl_and_tangent(m, qn, w1 * un)
        e0 = O.forcing(m, k * Dl, [0.3], rho)
        e1 = O.forcing(m, (k + 1) * Dl, [0.3], rho)
        dq = qn - q
        us = un + u
        rhs = 0.5 * dq @ (e1 + e0) - 0.5 * dq @ (f1 + f0) - w1 * Dl / 4 * us @ m.D @ us
        lhs = E(qn, un) - E(q, u)
        worst = max(worst, abs(lhs - rhs) / (abs(E(q, u)) + 1e-30))
    assert worst < 1e-10


def test_undamped_free_linear_conserves_energy():
    m = I.chain(5)
    m = m.linear_only()
    m.D = np.zeros_like(m.D)
    m.F = np.zeros_like(m.F)
    w1 = m.omega_n1
    rng = np.random.default_rng(4)
    tr = O.integrate_trajectory(m, w1, [0.5], np.array([0.0]), rng.standard_normal(5),
                                rng.standard_normal(5), 50, tol=0, maxit=2, sens=False,
                                keep_history=True)
    E = [0.5 * w1 ** 2 * u @ m.M @ u + 0.5 * q @ m.K @ q for q, u, _ in tr.history]
    assert np.ptp(E) <= 1e-12 * E[0]


@pytest.mark.parametrize("maker", [lambda: I.chain(5), lambda: I.vk_beam(n_el=4),
                                   lambda: I.van_der_pol(F=(10.0,))])
def test_sensitivities_match_central_differences(maker):
    m = maker()
    w1 = 1.2 * m.omega_n1
    rho = [I.GOLDEN]
    S1 = 24
    rng = np.random.default_rng(5)
    n = m.n
    # small for the von Karman beam, limit-cycle size for the self-excited damper (C_t != 0)
    scale = {3: 1e-4, 4: 1.0}.get(int(m.nl_type[0]) if m.n_nl else 0, 2e-2)
    q0 = scale * rng.standard_normal(n)
    u0 = scale * rng.standard_normal(n)
    phis = np.array([1.1])
    tr = O.integrate_trajectory(m, w1, rho, phis, q0, u0, S1, tol=0, maxit=16, sens=True)
    z0 = np.concatenate([q0, u0])
    h = 1e-6
    for j in range(2 * n):
        hp = 1e-4 * np.abs(z0).max()
        zp, zm = z0.copy(), z0.copy()
        zp[j] += hp
        zm[j] -= hp
        tp = O.integrate_trajectory(m, w1, rho, phis, zp[:n], zp[n:], S1, tol=0, maxit=16, sens=False)
        tm = O.integrate_trajectory(m, w1, rho, phis, zm[:n], zm[n:], S1, tol=0, maxit=16, sens=False)
        fd = (tp.zT - tm.zT) / (2 * hp)
        np.testing.assert_allclose(tr.Phi[:, j], fd, rtol=1e-5, atol=1e-6 * np.abs(tr.Phi).max())
    hw = 1e-6 * w1
    tp = O.integrate_trajectory(m, w1 + hw, rho, phis, q0, u0, S1, tol=0, maxit=16, sens=False)
    tm = O.integrate_trajectory(m, w1 - hw, rho, phis, q0, u0, S1, tol=0, maxit=16, sens=False)
    fd = (tp.zT - tm.zT) / (2 * hw)
    np.testing.assert_allclose(tr.dz_dw, fd, rtol=1e-5, atol=1e-6 * np.abs(tr.dz_dw).max())


def test_linear_monodromy_same_for_all_trajectories():
    """f_nl = 0: Phi_s does not depend on the start point or the forcing phase."""
    m = I.chain(4).linear_only()
    prob = O.FSEProblem(m, [5], [2], 16, [0.3])
    rng = np.random.default_rng(6)
    rj = O.residual_jacobian(prob, rng.standard_normal(2 * 4 * 5), 1.1 * m.omega_n1, tol=0,
                             maxit=2, dense=False)
    for s in range(1, 5):
        np.testing.assert_allclose(rj.Phi[s], rj.Phi[0], rtol=1e-12, atol=1e-13)


def test_newton_counts_and_nonconvergence_flag():
    m = I.eb_beam()
    w1 = 1.1 * m.omega_n1
    tr = O.integrate_trajectory(m, w1, [I.GOLDEN], np.array([0.0]), np.zeros(m.n), np.zeros(m.n),
                                128, tol=1e-10, maxit=20, sens=False)
    assert tr.converged and max(tr.newton_iters) <= 6 and min(tr.newton_iters) >= 1
    tr1 = O.integrate_trajectory(m, w1, [I.GOLDEN], np.array([0.0]), 1e-3 * np.ones(m.n),
                                 np.zeros(m.n), 128, tol=1e-14, maxit=1, sens=False)
    assert not tr1.converged
