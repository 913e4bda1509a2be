"""Continuation with an FP64 fallback context (fse_set_fallback).

On the nearly undamped 447-dof von Karman beam (d = 2, N = 64, H = 31, S1 = 512, 0.05 N per
forcing component) the FP32 tangents move a Floquet multiplier across the unit circle and
Newton with the mixed-precision Jacobian does not contract (see test_gpu_vk447_precision).
With an FP64 context attached, the continuation driver corrects the rejected points again in
FP64 from the same prediction: every point is accepted at ||R|| <= 1e-9 ||Z|| (FP64 Newton on
this beam levels off near 2e-10 with GMRES at 1e-10), and the accepted tori equal those of
plain FP64 Newton from the same starts.  Also: the attach checks
that both contexts describe one problem."""
import dataclasses

import numpy as np
import pytest

from paper_2508_06302_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _linear_start(wl):
    """Discrete closed-form response with f_nl dropped (trapezoid steps), per forcing component."""
    m, n, w1 = wl.model, wl.model.n, wl.omega1
    Dl = 2 * np.pi / wl.S1
    C = np.zeros((2 * n, wl.U_tilde))
    for lam, F, col in [(1.0, m.F[0], None), (wl.rho[0], m.F[1], 1)]:
        s = 2j / Dl * np.tan(lam * Dl / 2)
        Q = np.linalg.solve(m.K + w1 * s * m.D + w1 ** 2 * s * s * m.M, F)
        if col is None:
            C[:n, 0], C[n:, 0] = Q.real, (s * Q).real
        else:
            C[:n, 1], C[n:, 1] = Q.real, (s * Q).real
            C[:n, 2], C[n:, 2] = -Q.imag, -(s * Q).imag
    return C.reshape(-1)


def _fp64_newton(ctx, Z, w, steps=8, stop=1e-9):
    for _ in range(steps):
        Z, rn, rc = ctx.newton_step(Z, w)
        R, st, its, rc = ctx.residual_jacobian(Z, w, want_jacobian=False)
        if np.linalg.norm(R) <= stop * np.linalg.norm(Z):
            break
    return Z, np.linalg.norm(R) / np.linalg.norm(Z)


def test_fallback_accepts_the_points_the_mixed_form_rejects():
    from paper_2508_06302_gb300 import fse
    m = I.vk_beam(F1=0.05, F2=0.05)
    wl = dataclasses.replace(I.workload_vkbeam447(), model=m, omega1=1.1 * m.omega_n1, newton_tol=1e-11)
    Z0 = _linear_start(wl)
    c32 = fse.Context.from_workload(wl, precision="mixed_fp32")
    c64 = fse.Context.from_workload(wl, precision="fp64")
    for c in (c32, c64):
        c.set_linear_solver("gmres", rel_tol=1e-10, restart=80, max_iters=1600)
    c32.set_fallback(c64)
    omegas = wl.omega1 * np.array([1.0, 1.0005])
    Z, pts, rc = fse.fse_continue(c32, omegas, Z0, rel_tol=1e-9, max_newton=6)
    print("points:", [(p["status"], p["fallback"], p["newton_iters"], "%.1e" % (p["res"] / p["znorm"])) for p in pts])
    assert rc == 0 and all(p["status"] == 0 for p in pts)
    assert all(p["res"] <= 1e-9 * p["znorm"] for p in pts)
    assert any(p["fallback"] == 1 for p in pts)
    # the same tori from plain FP64 Newton: point 0 from the linear start, point 1 from point 0
    Zr0, r0 = _fp64_newton(c64, Z0.copy(), omegas[0])
    Zr1, r1 = _fp64_newton(c64, Zr0.copy(), omegas[1])
    e0 = np.linalg.norm(Z[0] - Zr0) / np.linalg.norm(Zr0)
    e1 = np.linalg.norm(Z[1] - Zr1) / np.linalg.norm(Zr1)
    print("FP64 Newton residuals %.1e %.1e; fallback tori vs FP64 Newton %.2e %.2e" % (r0, r1, e0, e1))
    assert e0 <= 1e-9 and e1 <= 1e-9
    c32.set_fallback(None)
    c32.close()
    c64.close()


def test_fallback_attach_checks_the_problem():
    from paper_2508_06302_gb300 import fse
    m = I.chain(6)
    c32 = fse.Context(m, 2, [8], [3], [I.GOLDEN], 32, precision="mixed_fp32")
    c64 = fse.Context(m, 2, [8], [3], [I.GOLDEN], 32, precision="fp64")
    other_n = fse.Context(m, 2, [6], [2], [I.GOLDEN], 32, precision="fp64")
    other_s1 = fse.Context(m, 2, [8], [3], [I.GOLDEN], 64, precision="fp64")
    c32.set_fallback(c64)
    c32.set_fallback(None)
    for bad in (other_n, other_s1, c32):
        with pytest.raises(fse.FSEError):
            c32.set_fallback(bad)
    with pytest.raises(fse.FSEError):   # the primary must be the mixed-precision one
        c64.set_fallback(c32)
    for c in (c32, c64, other_n, other_s1):
        c.close()
