"""A priori unknown base frequencies on the GPU (Sec. 3.2: Eq. Cont1, 18, 19, 23, 24), through the
C ABI, against the FP64 oracle (oracle/unknown_freq.py) on the forced van der Pol oscillator: its
self-excited frequency w_2 is set by no forcing and joins Z(0) as an unknown.

Checked: the residual, monodromies and d zbar / d w_1 with the velocity-dependent element
(C_t != 0 in K_eff and in the tangent recurrence) at 1e-10 (FP64 tangents) and 1e-3 (FP32
tangents); and the bordered Newton (phase condition + rotation-derivative column, dense LU and
GMRES) from the first-harmonic guess onto the oracle's torus and w_2 within 1e-9 relative."""
import numpy as np
import pytest

from oracle import fse_oracle as O
from oracle import unknown_freq as UF
from paper_2508_06302_gb300 import inputs as I

pytestmark = pytest.mark.gpu

WN = 10.0
W1 = WN / 2.7


def _fse():
    from paper_2508_06302_gb300 import fse
    fse.load()
    return fse


@pytest.mark.parametrize("precision,tol_phi", [("fp64", 1e-10), ("mixed_fp32", 1e-3)])
def test_vdp_residual_and_monodromy_match_oracle(precision, tol_phi):
    m = I.van_der_pol(omega_n=WN, eps=0.2, F=(10.0,))
    S, H, S1, rho = [8], [3], 48, [2.7]
    prob = O.FSEProblem(m, S, H, S1, rho)
    Z = np.random.default_rng(3).standard_normal(2 * prob.U) * 0.3
    ref = O.residual_jacobian(prob, Z, W1, want_jacobian=True, dense=False, tol=0, maxit=8)
    fse = _fse()
    ctx = fse.Context(m, 2, S, H, rho, S1, newton_tol=0, newton_maxit=8, precision=precision)
    R, st, it, rc = ctx.residual_jacobian(Z, W1, want_jacobian=True)
    assert rc == 0
    Phi, dz = ctx.monodromy()
    e_R = np.linalg.norm(R - ref.R) / (np.linalg.norm(Z) + np.linalg.norm(ref.R))
    e_P = np.linalg.norm(Phi - ref.Phi) / np.linalg.norm(ref.Phi)
    e_d = np.linalg.norm(dz - ref.dz_dw) / np.linalg.norm(ref.dz_dw)
    print("van der Pol %s: R %.2e, Phi %.2e, dz/dw %.2e" % (precision, e_R, e_P, e_d))
    assert e_R <= 1e-10
    assert e_P <= tol_phi
    assert e_d <= max(tol_phi, 1e-10) * 10
    ctx.close()


def _guess(U, rho0):
    C = np.zeros((2, U))
    C[0, 0] = 10.0 / (WN ** 2 - W1 ** 2)       # forced linear response at phi_1 = 0
    C[0, 1] = 2.0                              # limit cycle, first harmonic
    C[1, 2] = -2.0 * rho0
    return C.reshape(-1)


def _shift(Z, theta, H):
    """The torus shifted by theta along phi_2: harmonic k's (cos, sin) pair rotated by k theta
    (d = 2, harmonic order [1, cos k, sin k, ...] of Eq. 11)."""
    C = np.asarray(Z).reshape(2, 2 * H[0] + 1).copy()
    out = C.copy()
    for k in range(1, H[0] + 1):
        a, b = C[:, 2 * k - 1], C[:, 2 * k]
        c, s = np.cos(k * theta), np.sin(k * theta)
        out[:, 2 * k - 1] = c * a + s * b
        out[:, 2 * k] = -s * a + c * b
    return out.reshape(-1)


def _align_phase(Zr, Z, H):
    """theta minimising ||shift(Zr, theta) - Z|| (Newton from the first harmonic's phase)."""
    C, Cr = np.asarray(Z).reshape(2, -1), np.asarray(Zr).reshape(2, -1)
    theta = np.arctan2(Cr[0, 2], Cr[0, 1]) - np.arctan2(C[0, 2], C[0, 1])
    for _ in range(20):
        h = 1e-7
        f = lambda t: np.sum((_shift(Zr, t, H) - Z) ** 2)
        g = (f(theta + h) - f(theta - h)) / (2 * h)
        gg = (f(theta + h) - 2 * f(theta) + f(theta - h)) / (h * h)
        if gg <= 0:
            break
        theta -= g / gg
    return theta


@pytest.fixture(scope="module")
def vdp_torus():
    m = I.van_der_pol(omega_n=WN, eps=0.2, F=(10.0,))
    S, H, S1 = [24], [9], 256
    rho0 = np.array([WN / W1])
    Zr, rho_r, hist, ok = UF.solve_torus_unknown(m, S, H, S1, rho0, _guess(2 * H[0] + 1, rho0[0]), W1, [0],
                                                 rel_tol=1e-13, max_newton=12, tol=0, maxit=8)
    assert ok, hist
    return m, S, H, S1, rho0, Zr, rho_r


@pytest.mark.parametrize("precision,solver", [("fp64", "dense"), ("fp64", "gmres"), ("mixed_fp32", "dense")])
def test_unknown_frequency_newton_matches_oracle(vdp_torus, precision, solver):
    m, S, H, S1, rho0, Zr, rho_r = vdp_torus
    U = 2 * H[0] + 1
    fse = _fse()
    ctx = fse.Context(m, 2, S, H, list(rho0), S1, newton_tol=0, newton_maxit=8, precision=precision)
    if solver == "gmres":
        ctx.set_linear_solver("gmres", rel_tol=1e-12, restart=80, max_iters=800)
    Z, rho = _guess(U, rho0[0]), rho0.copy()
    norms = []
    for _ in range(14):
        Z, rho, rn, rc = ctx.newton_step_unknown(Z, W1, rho, [0])
        norms.append(rn)
    ctx.set_rho(rho)
    R, _, _, _ = ctx.residual_jacobian(Z, W1, want_jacobian=False)
    # the torus is unique only up to a shift along phi_2 (the symmetry the phase condition of Eq. 18
    # removes from each Newton correction, not from the end point): compare after aligning the phase
    theta = _align_phase(Zr, Z, H)
    e_Z = np.linalg.norm(Z - _shift(Zr, theta, H)) / np.linalg.norm(Zr)
    e_w = abs(rho[0] - rho_r[0]) / abs(rho_r[0])
    print("unknown w_2 %s/%s: ||R|| %s; phase offset %.2e rad, Z error %.2e, w_2 error %.2e, w_2 / w_n = %.6f"
          % (precision, solver, ["%.1e" % x for x in norms], theta, e_Z, e_w, rho[0] * W1 / WN))
    assert np.linalg.norm(R) <= 1e-12 * np.linalg.norm(Z)
    assert e_Z <= 1e-9 and e_w <= 1e-9
    ctx.close()


def test_forced_frequency_cannot_be_unknown():
    fse = _fse()
    m = I.van_der_pol(omega_n=WN, eps=0.2, F=(10.0, 3.0))      # e = 2: w_2 is forced
    ctx = fse.Context(m, 2, [8], [3], [2.7], 48, newton_tol=0, newton_maxit=8)
    with pytest.raises(fse.FSEError) as ei:
        ctx.newton_step_unknown(np.zeros(ctx.n_unknowns), W1, [2.7], [0])
    assert ei.value.code == fse.FSE_EINVAL
    ctx.close()
