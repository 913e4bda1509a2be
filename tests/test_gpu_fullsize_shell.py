"""Parity at the benchmark's full size: the 1872-dof shell, d = 2, N = 64, H = 31,
S1 = 1000, in the precision bench.py times (FP64 state, FP32 tangents) and in plain
FP64, on what the oracle can compute in seconds: the first two Newmark steps of the
period (fse_set_steps) for the residual of all 64 trajectories, and the monodromy
block and w_1 column of one sampled trajectory; and, with 8 trajectories (H = 3),
over the first 16 steps, long enough for every ring of the step loop to wrap
around several times.  Per-step Newton with a fixed iteration count on both
sides."""
import numpy as np
import pytest

from oracle import fse_oracle as O
from paper_2508_06302_gb300 import inputs as I

pytestmark = pytest.mark.gpu

STEPS, MAXIT, SAMPLE = 2, 3, 5


@pytest.fixture(scope="module")
def reference():
    wl = I.workload_shell1872()
    m = wl.model
    prob = O.FSEProblem(m, wl.S, wl.H, wl.S1, wl.rho)
    Z = I.random_coeffs(m.n, wl.U_tilde, 1e-5, seed=11)
    r = O.residual_jacobian(prob, Z, wl.omega1, want_jacobian=False, tol=0, maxit=MAXIT, n_steps=STEPS)
    zb = O.idft(prob, Z)
    tr = O.integrate_trajectory(m, wl.omega1, prob.rho, prob.T[:, SAMPLE], zb[SAMPLE, :m.n], zb[SAMPLE, m.n:],
                                wl.S1, tol=0, maxit=MAXIT, sens=True, n_steps=STEPS)
    return wl, Z, r.R, tr.Phi, tr.dz_dw


@pytest.mark.parametrize("precision,tol_phi", [("mixed_fp32", 1e-5), ("fp64", 1e-11)])
def test_shell1872_truncated_period_against_oracle(reference, precision, tol_phi):
    from paper_2508_06302_gb300 import fse
    wl, Z, R_ref, Phi_ref, dz_ref = reference
    ctx = fse.Context.from_workload(wl, precision=precision, newton_tol=0, newton_maxit=MAXIT)
    ctx.set_steps(STEPS)
    R, st, it, rc = ctx.residual_jacobian(Z, wl.omega1, want_jacobian=True)
    assert rc == 0
    scale = np.linalg.norm(Z) + np.linalg.norm(R_ref)
    err_R = np.linalg.norm(R - R_ref) / scale
    Phi, dz = ctx.monodromy_traj(SAMPLE)
    err_P = np.linalg.norm(Phi - Phi_ref) / np.linalg.norm(Phi_ref)
    err_d = np.linalg.norm(dz - dz_ref) / np.linalg.norm(dz_ref)
    print("shell1872 %s: R %.2e, Phi_%d %.2e, dz/dw %.2e" % (precision, err_R, SAMPLE, err_P, err_d))
    assert err_R <= 1e-10
    assert err_P <= tol_phi
    assert err_d <= 100 * tol_phi
    ctx.close()


LONG_STEPS, LONG_SAMPLE = 16, 3


@pytest.fixture(scope="module")
def reference_long():
    # the same 1872-dof shell with 8 trajectories (H = 3) so that the oracle follows 16 steps in
    # seconds: the factor buffers (step parity), the tangent-value ring (step mod 3), the two-stream
    # overlap and the solves' shared rings all wrap around several times
    wl = I.workload_shell1872(S=[8], H=[3])
    m = wl.model
    prob = O.FSEProblem(m, wl.S, wl.H, wl.S1, wl.rho)
    Z = I.random_coeffs(m.n, wl.U_tilde, 1e-5, seed=12)
    r = O.residual_jacobian(prob, Z, wl.omega1, want_jacobian=False, tol=0, maxit=MAXIT, n_steps=LONG_STEPS)
    zb = O.idft(prob, Z)
    s = LONG_SAMPLE
    tr = O.integrate_trajectory(m, wl.omega1, prob.rho, prob.T[:, s], zb[s, :m.n], zb[s, m.n:], wl.S1, tol=0,
                                maxit=MAXIT, sens=True, n_steps=LONG_STEPS)
    return wl, Z, r.R, tr.Phi, tr.dz_dw


@pytest.mark.parametrize("precision,tol_phi", [("mixed_fp32", 1e-4), ("fp64", 1e-11)])
def test_shell1872_sixteen_steps_against_oracle(reference_long, precision, tol_phi):
    from paper_2508_06302_gb300 import fse
    wl, Z, R_ref, Phi_ref, dz_ref = reference_long
    ctx = fse.Context.from_workload(wl, precision=precision, newton_tol=0, newton_maxit=MAXIT)
    ctx.set_steps(LONG_STEPS)
    R, st, it, rc = ctx.residual_jacobian(Z, wl.omega1, want_jacobian=True)
    assert rc == 0
    err_R = np.linalg.norm(R - R_ref) / (np.linalg.norm(Z) + np.linalg.norm(R_ref))
    Phi, dz = ctx.monodromy_traj(LONG_SAMPLE)
    err_P = np.linalg.norm(Phi - Phi_ref) / np.linalg.norm(Phi_ref)
    err_d = np.linalg.norm(dz - dz_ref) / np.linalg.norm(dz_ref)
    print("shell1872 N=8, %d steps, %s: R %.2e, Phi_%d %.2e, dz/dw %.2e"
          % (LONG_STEPS, precision, err_R, LONG_SAMPLE, err_P, err_d))
    assert err_R <= 1e-10
    assert err_P <= tol_phi
    assert err_d <= 100 * tol_phi
    ctx.close()
