"""FSE-Shooting with a priori unknown base frequencies (Sec. 3.2: Eq. Cont1, Eq. 18, Eq. 19,
Eq. 23, Eq. 24), plain FP64 on the CPU.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: nothing in the product path imports it,
and it shares no code with the CUDA path.

With e forcing components and d > e base frequencies, the frequencies w_i, i > e, are not set
by the model: they join Z(0) as unknowns, and each adds one phase condition, because a torus
shifted along phi_i is again a solution (Sec. 3.2.2).  Readings used here:

* Eq. (19): grad_i is block-diagonal over the harmonics, [[0, k_il], [-k_il, 0]] acting on the
  (cos, sin) coefficient pair of harmonic l, 0 on the constant; (I (x) grad_i) Z holds the
  coefficients of dz/dphi_i.
* Eq. (24), i >= 2: the rotation angles are 2 pi k~_l . rho with rho_i = w_i / w_1, so
  dR(rho)/dw_i = (2 pi / w_1) diag(0, Upsilon_il) R(rho); the printed prefactor 2 pi / w_i is
  read as 2 pi / w_1 (it is the derivative of rho_i with respect to w_i).
* Eq. (23), i > e: the trajectories do not depend on w_i (no forcing phase moves with it), so
  dR/dw_i is the rotation term alone, (I (x) dR(rho)/dw_i) Z(2 pi).
* Eq. (18) with Z* = the Newton correction: the correction dZ of every iteration is orthogonal
  to (I (x) grad_i) Z at the current iterate, i.e. the Newton system is bordered by the rows
  ((I (x) grad_i) Z)^T and the columns dR/dw_i.

Pinned by tests/test_oracle_unknown_freq.py: grad_i against finite differences of the
trigonometric interpolant, dR(rho)/dw_i against finite differences of R(rho), dR/dw_i against
finite differences of the residual (in w_i, and in w_1 with the unknown w_i held fixed), the
closed-form discrete free oscillation (whose rotation
number Newmark fixes exactly), the shift equivariance of the residual, and a brute-force
long-time integration that stays on the solved torus with the solved frequency.
"""
from __future__ import annotations

import numpy as np

from oracle import fse_oracle as O


def nabla_phi(ktab, j):
    """grad_i of Eq. (19) for angle phi_{j+2} (column j of the harmonic table), U~ x U~."""
    L = ktab.shape[0] - 1
    N = np.zeros((2 * L + 1, 2 * L + 1))
    for l in range(L):
        k = float(ktab[l, j])
        N[1 + 2 * l, 2 + 2 * l] = k
        N[2 + 2 * l, 1 + 2 * l] = -k
    return N


def phase_gradient(prob, Z, j):
    """(I_2n (x) grad_{j+2}) Z: the coefficients of dz(0, phi~)/dphi_{j+2} (Eq. 18)."""
    C = np.asarray(Z, dtype=np.float64).reshape(2 * prob.n, prob.U)
    return (C @ nabla_phi(prob.ktab, j).T).reshape(-1)


def drotation_domega(ktab, rho, omega1, j):
    """dR(rho)/dw_{j+2} of Eq. (24): (2 pi / w_1) diag(0, Upsilon_l) R(rho), Upsilon_l =
    [[0, -k_lj], [k_lj, 0]]."""
    L = ktab.shape[0] - 1
    Ups = np.zeros((2 * L + 1, 2 * L + 1))
    for l in range(L):
        k = float(ktab[l, j])
        Ups[1 + 2 * l, 2 + 2 * l] = -k
        Ups[2 + 2 * l, 1 + 2 * l] = k
    return (2.0 * np.pi / omega1) * Ups @ O.rotation(ktab, rho)


def _check_unknown(model, unknown):
    e = model.F.shape[0]
    for j in unknown:
        # forcing component j + 1 would move its phase with rho_j (Eq. E1): then w_{j+2} is set
        if j + 1 < e:
            raise ValueError("w_%d is the frequency of forcing component %d, not an unknown" % (j + 2, j + 1))


def residual_unknown(model, S, H, S1, rho, Z0, omega1, unknown, tol=1e-10, maxit=20):
    """R(Z(0), w) of Eq. (16) at rho, with the dense dR/dZ(0) (Eq. 22) and, for every unknown
    frequency w_{j+2}, j in ``unknown``, dR/dw_{j+2} (Eq. 23, rotation term only).

    Returns (prob, ResidualJacobian, list of dR/dw columns)."""
    _check_unknown(model, unknown)
    prob = O.FSEProblem(model, list(S), list(H), S1, np.asarray(rho, dtype=np.float64))
    rj = O.residual_jacobian(prob, np.asarray(Z0, dtype=np.float64), omega1, want_jacobian=True, dense=True,
                             tol=tol, maxit=maxit)
    Z2 = rj.Z2pi.reshape(2 * prob.n, prob.U)
    cols = [(Z2 @ drotation_domega(prob.ktab, prob.rho, omega1, j).T).reshape(-1) for j in unknown]
    return prob, rj, cols


def dR_domega1_unknown(prob, rj, omega1, unknown):
    """dR/dw_1 of Eq. (23) when the frequencies w_{j+2}, j in ``unknown``, are held fixed (they
    are unknowns of their own, Eq. Cont1) and the forced ratios are fixed (Eq. Cont2): the
    integration term of ``residual_jacobian`` (rho fixed) plus the rotation term, whose angles
    2 pi k~_l . rho move through rho_j = w_{j+2} / w_1, d rho_j / d w_1 = -rho_j / w_1 (the
    Upsilon_1 case of Eq. 24 restricted to the unknown frequencies)."""
    Z2 = rj.Z2pi.reshape(2 * prob.n, prob.U)
    dR = np.zeros((prob.U, prob.U))
    for j in unknown:
        # dR(rho)/drho_j = w_1 dR(rho)/dw_{j+2}, times drho_j/dw_1 = -rho_j / w_1
        dR -= prob.rho[j] * drotation_domega(prob.ktab, prob.rho, omega1, j)
    return rj.dR_dw + (Z2 @ dR.T).reshape(-1)


def newton_step_unknown(model, S, H, S1, rho, Z0, omega1, unknown, tol=1e-10, maxit=20):
    """One Newton update of (Z(0), w_u) for Eq. (Cont1) at fixed w_1 (Sec. 3.3 step 6): the
    system [J, dR/dw_u; G^T, 0] [dZ; dw_u] = -[R; 0] with G the phase gradients of Eq. (18).

    Returns (Z_new, rho_new, ||R(Z0)||_2, max |phase condition| of the correction)."""
    prob, rj, cols = residual_unknown(model, S, H, S1, rho, Z0, omega1, unknown, tol, maxit)
    m = rj.R.size
    u = len(unknown)
    A = np.zeros((m + u, m + u))
    A[:m, :m] = rj.J
    for a, j in enumerate(unknown):
        A[:m, m + a] = cols[a]
        A[m + a, :m] = phase_gradient(prob, Z0, j)
    rhs = np.concatenate([-rj.R, np.zeros(u)])
    d = np.linalg.solve(A, rhs)
    Z_new = np.asarray(Z0, dtype=np.float64) + d[:m]
    rho_new = np.array(prob.rho, dtype=np.float64)
    for a, j in enumerate(unknown):
        rho_new[j] += d[m + a] / omega1              # w_{j+2} = rho_j w_1, w_1 fixed
    pc = max((abs(float(A[m + a, :m] @ d[:m])) for a in range(u)), default=0.0)
    return Z_new, rho_new, float(np.linalg.norm(rj.R)), pc


def solve_torus_unknown(model, S, H, S1, rho0, Z0, omega1, unknown, rel_tol=1e-10, max_newton=20,
                        tol=1e-12, maxit=30):
    """Newton on Eq. (Cont1) at fixed w_1 until ||R||_2 <= rel_tol ||Z(0)||_2.

    Returns (Z, rho, history of ||R||_2, converged)."""
    Z = np.asarray(Z0, dtype=np.float64).copy()
    rho = np.asarray(rho0, dtype=np.float64).copy()
    hist = []
    for _ in range(max_newton):
        prob = O.FSEProblem(model, list(S), list(H), S1, rho)
        R = O.residual_jacobian(prob, Z, omega1, want_jacobian=False, tol=tol, maxit=maxit).R
        rn = float(np.linalg.norm(R))
        hist.append(rn)
        if rn <= rel_tol * max(np.linalg.norm(Z), 1e-30):
            return Z, rho, hist, True
        Z, rho, _, _ = newton_step_unknown(model, S, H, S1, rho, Z, omega1, unknown, tol, maxit)
    return Z, rho, hist, False


def torus_point(prob, Z, phi):
    """z(0, phi~) = (I_2n (x) H(k~, phi~)) Z(0) (Eq. 10) at one point phi~."""
    C = np.asarray(Z, dtype=np.float64).reshape(2 * prob.n, prob.U)
    return C @ O.basis_row(prob.ktab, np.atleast_1d(np.asarray(phi, dtype=np.float64)))
