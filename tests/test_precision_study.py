"""Why the mixed-precision tangents are FP32 and not TF32 / BF16 tensor-core operands.

The sensitivities of App. E (Eq. E5-E9, differentiated Newmark step) are propagated here with
every product's operands rounded to p significand bits (FP32 p = 24, TF32 p = 11, BF16 p = 8)
and the results stored in FP32, as a tensor-core GEMM with FP32 accumulation would; the step
solve is a product with the explicit inverse of K_eff, as in the blocked solves.  The reference
is the FP64 oracle's monodromy of the same trajectory.  Linear beam, so that Phi_s is the same
for every trajectory and the outer Newton contraction has a closed form per harmonic: with
J = (I (x) R Gamma^-1) blockdiag(Phi) (I (x) Gamma) - I (Eq. 22), harmonic l sees
e^{i theta_l} Phi - I, and an error dPhi in the monodromy gives the inexact-Newton factor
max_l rho((e^{i theta_l} Phi - I)^-1 e^{i theta_l} dPhi) (Sec. 3.3 with an approximate J).
"""
import numpy as np

from oracle import fse_oracle as O
from paper_2508_06302_gb300 import inputs as I

S1 = 128
H = 7


def _round(x, p):
    """Round to p significand bits, nearest-even (exponent range unchanged)."""
    if p >= 53:
        return x
    m, e = np.frexp(x)
    return np.ldexp(np.round(m * 2.0 ** p) / 2.0 ** p, e)


def _tangent_monodromy(model, w, p_op):
    """Phi = [X; V][:, :2n] after S1 steps of the Eq. E8 recurrence (f_nl = 0), operands of
    every product rounded to p_op bits, or split into two TF32 parts ("3xtf32"), results to
    FP32 (FP64 throughout when p_op = 53)."""
    n = model.n
    Dl = 2.0 * np.pi / S1
    a0c, a1c, a2c = 4.0 / Dl ** 2, 4.0 / Dl, 2.0 / Dl
    M, D, K = model.M, model.D, model.K
    wM = w * w * M
    Keff_inv = np.linalg.inv(wM * a0c + w * a2c * D + K)
    st = (lambda x: x) if p_op == 53 else (lambda x: _round(x, 24))

    def mm(A, B):
        if p_op == "3xtf32":   # split operands a = hi + lo, both TF32; the lo*lo term dropped
            Ah, Bh = _round(A, 11), _round(B, 11)
            Al, Bl = _round(A - Ah, 11), _round(B - Bh, 11)
            return st(Ah @ Bh + (Ah @ Bl + Al @ Bh))
        return st(_round(A, p_op) @ _round(B, p_op))

    X = np.zeros((n, 2 * n))
    V = np.zeros((n, 2 * n))
    X[:, :n] = np.eye(n)
    V[:, n:] = np.eye(n)
    W = np.linalg.solve(wM, -K @ X - w * D @ V)   # consistent start (equation of motion at phi_1 = 0)
    for _ in range(S1):
        rhs = st(mm(wM, st(a0c * X + a1c * V + W)) + mm(w * D, st(a2c * X + V)))
        Xn = mm(Keff_inv, rhs)
        Vn = st(a2c * (Xn - X) - V)
        Wn = st(a0c * (Xn - X) - a1c * V - W)
        X, V, W = Xn, Vn, Wn
    return np.concatenate([X, V])


def _contraction(Phi, dPhi, rho):
    r = 0.0
    for l in range(H + 1):
        lam = np.exp(2j * np.pi * l * rho)
        A = lam * Phi - np.eye(Phi.shape[0])
        r = max(r, float(np.max(np.abs(np.linalg.eigvals(np.linalg.solve(A, lam * dPhi))))))
    return r


def test_fp32_tangents_keep_newton_contracting_tf32_and_bf16_do_not():
    m = I.eb_beam().linear_only()
    w = 1.1 * m.omega_n1
    z = np.zeros(m.n)
    ref = O.integrate_trajectory(m, w, [I.GOLDEN], np.zeros(1), z, z, S1, tol=0, maxit=1).Phi
    nref = np.linalg.norm(ref)
    # the harness in FP64 is the oracle's recurrence
    assert np.linalg.norm(_tangent_monodromy(m, w, 53) - ref) <= 1e-11 * nref
    err, con = {}, {}
    for name, p in (("fp32", 24), ("tf32", 11), ("bf16", 8), ("3xtf32", "3xtf32")):
        P = _tangent_monodromy(m, w, p)
        err[name] = np.linalg.norm(P - ref) / nref
        con[name] = _contraction(ref, P - ref, I.GOLDEN)
    # measured: fp32 2.0e-5 / 0.008, tf32 0.28 / 128, bf16 1.7 / 127, 3xtf32 6.4e-5 / 0.019
    assert err["fp32"] < 1e-4 and con["fp32"] < 0.05, (err, con)
    assert err["tf32"] > 0.05 and con["tf32"] > 1.0, (err, con)
    assert err["bf16"] > 0.5 and con["bf16"] > 1.0, (err, con)
    # a split (3 x TF32) product recovers FP32-level tangents
    assert err["3xtf32"] < 1e-4 and con["3xtf32"] < 0.05, (err, con)
