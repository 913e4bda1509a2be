"""FSE-Shooting in the hyper-time domain (Sec. 3.4, Eq. FSES_T), plain FP64 on the CPU.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: nothing in the product path imports it,
and it shares no code with the CUDA path.

The unknowns are the trajectory start points zbar(0, phi~_s), s < S~ (stored (S~, 2n)), instead
of the Fourier coefficients Z(0).  The terminal points are mapped back through the band-limited
interpolant and rotated:
    R_T(zbar(0), w) = (I_2n (x) Gamma R(rho) Gamma^-1) zbar(2 pi) - zbar(0)
with Gamma (S~ x U~) and Gamma^-1 (U~ x S~) of App. D, which need not be square here.  Its
Jacobian is (I_2n (x) Gamma R Gamma^-1) blockdiag_s(Phi_s) - I.  When zbar(0) = Gamma Z(0) the
residual is Gamma applied to the residual of Eq. (16), so both forms have the same tori.
Pinned by tests/test_oracle_hypertime.py: that identity, the chain rule between the two
Jacobians, and a hyper-time Newton solve that lands on Gamma times the Eq. (16) torus.
"""
from __future__ import annotations

import numpy as np

from oracle import fse_oracle as O


def interpolate_rotate(prob):
    """P = Gamma R(rho) Gamma^-1 (S~ x S~): samples -> coefficients -> rotation -> samples."""
    return prob.G @ prob.R @ prob.Gi


def residual_jacobian_hypertime(prob, zbar0, omega1, want_jacobian=True, tol=1e-10, maxit=20):
    """R_T of Eq. (FSES_T) at start points zbar0 (S~ x 2n); returns (R_T (S~ x 2n), J_T or None)
    with J_T[(s, i), (t, j)] = P[s, t] Phi_t[i, j] - delta."""
    zbar0 = np.asarray(zbar0, dtype=np.float64)
    n = prob.n
    N = prob.N
    zbT = np.zeros((N, 2 * n))
    Phi = np.zeros((N, 2 * n, 2 * n)) if want_jacobian else None
    for s in range(N):
        tr = O.integrate_trajectory(prob.model, omega1, prob.rho, prob.T[:, s], zbar0[s, :n], zbar0[s, n:],
                                    prob.S1, tol=tol, maxit=maxit, sens=want_jacobian)
        zbT[s] = tr.zT
        if want_jacobian:
            Phi[s] = tr.Phi
    P = interpolate_rotate(prob)
    RT = P @ zbT - zbar0
    JT = None
    if want_jacobian:
        m = N * 2 * n
        JT = np.einsum('st,tij->sitj', P, Phi, optimize=True).reshape(m, m) - np.eye(m)
    return RT, JT


def solve_hypertime(prob, zbar0, omega1, rel_tol=1e-10, max_newton=20, tol=1e-12, maxit=30):
    """Newton on R_T = 0 with the dense J_T until ||R_T||_2 <= rel_tol ||zbar(0)||_2.

    Returns (zbar0, history of ||R_T||_2, converged)."""
    zb = np.asarray(zbar0, dtype=np.float64).copy()
    hist = []
    for _ in range(max_newton):
        RT, JT = residual_jacobian_hypertime(prob, zb, omega1, True, tol, maxit)
        rn = float(np.linalg.norm(RT))
        hist.append(rn)
        if rn <= rel_tol * max(np.linalg.norm(zb), 1e-30):
            return zb, hist, True
        zb = zb + np.linalg.solve(JT, -RT.reshape(-1)).reshape(zb.shape)
    return zb, hist, False
