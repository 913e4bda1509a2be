"""Parity on the d = 3 workload at its full size: the 243-dof ACM plate with 40 seeded cubic
springs, three forcing frequencies (w_1, sqrt 2 w_1, sqrt 3 w_1), 16 x 16 = 256 trajectories on
the 2-torus, H = 7 x 7 (U~ = 225, 109,350 unknowns, the multi-index harmonic table of App. B),
S1 = 400.  Over the first STEPS Newmark steps of the period (fse_set_steps), what the oracle
computes in seconds: the residual of all 256 trajectories and the monodromy block and w_1
column of one sampled trajectory, in the benchmarked precision and in FP64, fixed per-step
Newton count on both sides."""
import numpy as np
import pytest

from oracle import fse_oracle as O
from paper_2508_06302_gb300 import inputs as I

pytestmark = pytest.mark.gpu

STEPS, MAXIT, SAMPLE = 8, 3, 77


@pytest.fixture(scope="module")
def reference():
    wl = I.workload_plate243()
    m = wl.model
    prob = O.FSEProblem(m, wl.S, wl.H, wl.S1, wl.rho)
    assert prob.N == 256 and prob.U == 225
    Z = I.random_coeffs(m.n, wl.U_tilde, 1e-5, seed=13)
    r = O.residual_jacobian(prob, Z, wl.omega1, want_jacobian=False, tol=0, maxit=MAXIT, n_steps=STEPS)
    zb = O.idft(prob, Z)
    tr = O.integrate_trajectory(m, wl.omega1, prob.rho, prob.T[:, SAMPLE], zb[SAMPLE, :m.n], zb[SAMPLE, m.n:],
                                wl.S1, tol=0, maxit=MAXIT, sens=True, n_steps=STEPS)
    return wl, Z, r.R, tr.Phi, tr.dz_dw


@pytest.mark.parametrize("precision,tol_phi", [("mixed_fp32", 1e-4), ("fp64", 1e-11)])
def test_plate243_d3_truncated_period_against_oracle(reference, precision, tol_phi):
    from paper_2508_06302_gb300 import fse
    wl, Z, R_ref, Phi_ref, dz_ref = reference
    ctx = fse.Context.from_workload(wl, precision=precision, newton_tol=0, newton_maxit=MAXIT)
    assert ctx.N == 256 and ctx.U == 225
    ctx.set_steps(STEPS)
    R, st, it, rc = ctx.residual_jacobian(Z, wl.omega1, want_jacobian=True)
    assert rc == 0
    err_R = np.linalg.norm(R - R_ref) / (np.linalg.norm(Z) + np.linalg.norm(R_ref))
    Phi, dz = ctx.monodromy_traj(SAMPLE)
    err_P = np.linalg.norm(Phi - Phi_ref) / np.linalg.norm(Phi_ref)
    err_d = np.linalg.norm(dz - dz_ref) / np.linalg.norm(dz_ref)
    print("plate243 d=3 N=256 H=7x7, %d steps, %s: R %.2e, Phi_%d %.2e, dz/dw %.2e"
          % (STEPS, precision, err_R, SAMPLE, err_P, err_d))
    assert err_R <= 1e-10
    assert err_P <= tol_phi
    assert err_d <= 100 * tol_phi
    ctx.close()
