"""Plain FP64 CPU oracle of FSE-Shooting (arXiv 2508.06302).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or
links this module; only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` use it.  It shares no code with the CUDA
path: every function here is a direct, slow, step-by-step restatement of the
paper's definitions in NumPy float64, written so that a reader can check it
against the paper by eye.

Conventions (readings of the paper where it is silent or ambiguous):

* The state is z = [q; u] with u = q' = dq/dphi_1 (App. E, Eq. E8), not the
  physical velocity of Eq. (2); Eq. (F3) converts for the Lyapunov part.
* Coefficients Z are state-major: Z[i * U~ + c] is coefficient c of state i
  (Eq. 10, App. D), and coefficient c follows the trigonometric basis of
  Eq. (11): [1, cos(k_1.phi), sin(k_1.phi), ..., cos(k_L.phi), sin(k_L.phi)].
* The forcing is e(phi_1, phi~) = F_1 cos(phi_1) + sum_{j>=2} F_j cos(phi_j + rho_j phi_1)
  (Eq. E1 with Eq. 25).  The frequency ratios rho_j are held fixed, so the
  rotation R(rho) and the forcing phases do not depend on w_1.
* The initial acceleration a_0 comes from the equation of motion at phi_1 = 0.
* Per-step Newton (App. E): full Newton started from the previous
  displacement q_k (the paper does not name a predictor; the constant one
  is the robust choice for the stiff axial and membrane modes of FE models),
  stopping when ||dq||_inf <= tol * ||q_{k+1}||_inf (at least one
  iteration); tol <= 0 means "exactly maxit iterations".

Parity status of each function is stated in its docstring.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

NL_CUBIC_GROUND = 1
NL_CUBIC_DIFF = 2
NL_VK_BEAM = 3
NL_VDP = 4


# -----------------------------------------------------------------------------
# App. B: harmonic index selection  K~^d
# -----------------------------------------------------------------------------

def harmonic_table(H):
    """Rows of K~^d for K_j = [0, 1, ..., H_j], j = 2..d (App. B, Eq. B1-B2).

    Returns an int array of shape ((U~+1)/2, d-1).  Rows 0..L~-1 are k~_1..k~_L
    (in the order of Eq. B1-B2) and the last row is the zero row k~_0, which
    carries the constant term of Eq. (11).

    d = 2: K~^2 = [k_2; 0].
    d > 2: K~^d = [K^{d,g}; K~^{d,b}] with
       K^{d,g}  = [1_{L_d} (x) K~^{d-1,r},       -k_d (x) 1_{L~^{d-1}}]
       K~^{d,b} = [1_{L_d+1} (x) K~^{d-1},  [k_d; 0] (x) 1_{L~^{d-1}+1}]
    where K~^{d-1,r} is K~^{d-1} without its zero row.
    Pinned by the row count (U~+1)/2 and by the discrete orthogonality of the
    basis it generates (tests/test_oracle_aft.py).
    """
    H = list(H)
    if len(H) == 0:
        return np.zeros((1, 0), dtype=np.int64)
    k2 = np.arange(1, H[0] + 1)
    table = np.concatenate([k2[:, None], np.zeros((1, 1), np.int64)], axis=0)
    for Hd in H[1:]:
        kd = np.arange(1, Hd + 1)
        prev_r = table[:-1]                     # K~^{d-1,r}
        Lprev = prev_r.shape[0]
        g_left = np.kron(np.ones((len(kd), 1), np.int64), prev_r)
        g_right = np.kron(-kd[:, None], np.ones((Lprev, 1), np.int64))
        g = np.concatenate([g_left, g_right], axis=1)
        kd0 = np.concatenate([kd, [0]])
        b_left = np.kron(np.ones((len(kd0), 1), np.int64), table)
        b_right = np.kron(kd0[:, None], np.ones((table.shape[0], 1), np.int64))
        b = np.concatenate([b_left, b_right], axis=1)
        table = np.concatenate([g, b], axis=0)
    return table


def u_tilde(H) -> int:
    """U~ = prod_j (2 H_j + 1) (Sec. 3.1)."""
    return int(np.prod([2 * h + 1 for h in H])) if len(H) else 1


# -----------------------------------------------------------------------------
# App. D: sample grid, Gamma and Gamma^{-1};  Eq. (14): rotation R(rho)
# -----------------------------------------------------------------------------

def sample_grid(S):
    """T = [T_2; ...; T_d] of Eq. (D1): column s holds phi~_s.

    T_j = 1^T_{S_{j+1}..S_d} (x) phibar_j (x) 1^T_{S_2..S_{j-1}}, so phi_2
    varies fastest; phibar_j = 2 pi [0..S_j-1] / S_j.
    """
    S = list(S)
    Stot = int(np.prod(S)) if S else 1
    T = np.zeros((len(S), Stot))
    for j, Sj in enumerate(S):
        phibar = 2.0 * np.pi * np.arange(Sj) / Sj
        before = int(np.prod(S[:j])) if j > 0 else 1
        after = int(np.prod(S[j + 1:])) if j + 1 < len(S) else 1
        T[j] = np.kron(np.ones(after), np.kron(phibar, np.ones(before)))
    return T


def basis_row(ktab, phi):
    """H(k~, phi~) of Eq. (11) at one point phi~ (vector of length d-1)."""
    L = ktab.shape[0] - 1
    out = np.zeros(2 * L + 1)
    out[0] = 1.0
    for l in range(L):
        arg = float(np.dot(ktab[l], phi))
        out[1 + 2 * l] = math.cos(arg)
        out[2 + 2 * l] = math.sin(arg)
    return out


def gamma(ktab, T):
    """Gamma (S~ x U~) of Eq. (D2): row s is H(k~, phi~_s)."""
    return np.stack([basis_row(ktab, T[:, s]) for s in range(T.shape[1])])


def gamma_inv(ktab, T):
    """Gamma^{-1} (U~ x S~) of Eq. (D3): (1/S~)[1; 2cos; 2sin; ...]."""
    Stot = T.shape[1]
    G = gamma(ktab, T)
    Gi = 2.0 * G.T / Stot
    Gi[0] = 1.0 / Stot
    return Gi


def rotation(ktab, rho):
    """R(rho) of Eq. (14): diag(1, [[c, -s], [s, c]]_l) with angle 2 pi k~_l . rho."""
    L = ktab.shape[0] - 1
    R = np.zeros((2 * L + 1, 2 * L + 1))
    R[0, 0] = 1.0
    for l in range(L):
        th = 2.0 * np.pi * float(np.dot(ktab[l], rho))
        c, s = math.cos(th), math.sin(th)
        R[1 + 2 * l, 1 + 2 * l] = c
        R[1 + 2 * l, 2 + 2 * l] = -s
        R[2 + 2 * l, 1 + 2 * l] = s
        R[2 + 2 * l, 2 + 2 * l] = c
    return R


# -----------------------------------------------------------------------------
# nonlinear forces f_nl(q, qdot) and tangents (the model of Eq. 1 / Eq. 25)
# -----------------------------------------------------------------------------

_GL5 = np.polynomial.legendre.leggauss(5)


def _vk_hermite_slope(xi, L):
    """dN/dx of the Hermite cubic (w1, th1, w2, th2) at xi in [-1, 1]."""
    # N1 = 1 - 3s^2 + 2s^3, N2 = L(s - 2s^2 + s^3), N3 = 3s^2 - 2s^3, N4 = L(-s^2 + s^3), s = x/L
    s = 0.5 * (xi + 1.0)
    dN_ds = np.array([-6 * s + 6 * s * s, L * (1 - 4 * s + 3 * s * s), 6 * s - 6 * s * s,
                      L * (-2 * s + 3 * s * s)])
    return dN_ds / L


def fnl_and_tangent(model, q, qdot):
    """f_nl(q, qdot) and its Jacobians K_t = df/dq, C_t = df/dqdot.

    Element types (see the input module): cubic grounded spring, cubic
    difference spring, and the 2-node von Karman beam whose nonlinear
    internal force is the gradient of the axial-stretching energy
    EA/2 int (u' w'^2 + w'^4/4) dx with u linear and w Hermite cubic,
    integrated exactly by 5-point Gauss-Legendre.  The self-excited damper
    f = p0 (q^2 - 1) qdot (van der Pol) is the only element that depends on qdot
    (C_t != 0); it is a test model for base frequencies that no forcing defines.
    Pinned by finite differences of f_nl (tests/test_oracle_newmark.py,
    tests/test_oracle_unknown_freq.py).
    """
    n = q.shape[0]
    f = np.zeros(n)
    Kt = np.zeros((n, n))
    Ct = np.zeros((n, n))
    for e in range(model.nl_type.shape[0]):
        t = int(model.nl_type[e])
        dof = model.nl_dof[e]
        p = model.nl_p[e]
        if t == NL_CUBIC_GROUND:
            i = int(dof[0])
            k3 = p[0]
            f[i] += k3 * q[i] ** 3
            Kt[i, i] += 3.0 * k3 * q[i] ** 2
        elif t == NL_CUBIC_DIFF:
            i, j = int(dof[0]), int(dof[1])
            k3 = p[0]
            dlt = q[i] - q[j]
            fe = k3 * dlt ** 3
            ke = 3.0 * k3 * dlt ** 2
            f[i] += fe
            f[j] -= fe
            Kt[i, i] += ke
            Kt[j, j] += ke
            Kt[i, j] -= ke
            Kt[j, i] -= ke
        elif t == NL_VDP:
            i = int(dof[0])
            c = p[0]
            f[i] += c * (q[i] * q[i] - 1.0) * qdot[i]
            Kt[i, i] += 2.0 * c * q[i] * qdot[i]
            Ct[i, i] += c * (q[i] * q[i] - 1.0)
        elif t == NL_VK_BEAM:
            EA, L = p[0], p[1]
            loc = np.array([q[int(g)] if g >= 0 else 0.0 for g in dof[:6]])
            ua = loc[[0, 3]]
            wb = loc[[1, 2, 4, 5]]
            du = (ua[1] - ua[0]) / L
            fe = np.zeros(6)
            ke = np.zeros((6, 6))
            bu = np.array([-1.0 / L, 1.0 / L])
            for xi, wq in zip(*_GL5):
                jac = 0.5 * L * wq
                Nd = _vk_hermite_slope(xi, L)
                wp = float(Nd @ wb)
                # axial-stretching energy density EA/2 (u' w'^2 + w'^4 / 4)
                fe[[0, 3]] += jac * 0.5 * EA * wp * wp * bu
                fe[[1, 2, 4, 5]] += jac * EA * (du * wp + 0.5 * wp ** 3) * Nd
                kub = jac * EA * wp * np.outer(bu, Nd)
                ke[np.ix_([0, 3], [1, 2, 4, 5])] += kub
                ke[np.ix_([1, 2, 4, 5], [0, 3])] += kub.T
                ke[np.ix_([1, 2, 4, 5], [1, 2, 4, 5])] += jac * EA * (du + 1.5 * wp * wp) * np.outer(Nd, Nd)
            for a in range(6):
                ga = int(dof[a])
                if ga < 0:
                    continue
                f[ga] += fe[a]
                for b in range(6):
                    gb = int(dof[b])
                    if gb >= 0:
                        Kt[ga, gb] += ke[a, b]
        else:
            raise ValueError("unknown nonlinear element type %d" % t)
    return f, Kt, Ct


# -----------------------------------------------------------------------------
# App. E: Newmark average acceleration with per-step Newton and sensitivities
# -----------------------------------------------------------------------------

def forcing(model, phi1, phis, rho):
    """e(phi_1, phi~_s + rho phi_1) of Eq. (E1): F_1 cos(phi_1) + sum F_j cos(phi_j + rho_j phi_1)."""
    e = model.F[0] * math.cos(phi1)
    for j in range(1, model.F.shape[0]):
        e = e + model.F[j] * math.cos(phis[j - 1] + rho[j - 1] * phi1)
    return e


@dataclass
class TrajectoryResult:
    zT: np.ndarray                      # z(2 pi) = [q; u]  (2n)
    Phi: Optional[np.ndarray] = None    # d z(2 pi) / d z(0)  (2n x 2n), Eq. (E8)
    dz_dw: Optional[np.ndarray] = None  # d z(2 pi) / d w_1   (2n)
    newton_iters: list = field(default_factory=list)
    converged: bool = True
    history: Optional[list] = None      # optional per-step (q, u, a)


def integrate_trajectory(model, omega1, rho, phis, q0, u0, S1, tol=1e-10, maxit=20,
                         sens=True, keep_history=False, n_steps=None):
    """Integrate one trajectory phi_1: 0 -> 2 pi with Newmark (App. E).

    Scaled equation of motion (Eq. E2):
        w^2 M a + w D u + K q + f_nl(q, w u) - e = 0.
    Steps (Eq. E3-E7), Delta = 2 pi / S1:
        u_{k+1} = 2/Delta (q_{k+1} - q_k) - u_k
        a_{k+1} = 4/Delta^2 (q_{k+1} - q_k) - 4/Delta u_k - a_k
        S q_{k+1} + f_nl(q_{k+1}, w u_{k+1}(q_{k+1})) = b
        S = w^2 4/Delta^2 M + w 2/Delta D + K
        b = e_{k+1} + w^2 M (4/Delta^2 q_k + 4/Delta u_k + a_k) + w D (2/Delta q_k + u_k)
    solved by full Newton with K_eff = S + K_t + w 2/Delta C_t, started at q_k.

    Sensitivities (Eq. E8, E9) by differentiating the same step: with
    X = dq/dp, V = du/dp, W = da/dp for p in (q_0, u_0, w_1):
        K_eff X_{k+1} = w^2 M (4/D^2 X_k + 4/D V_k + W_k) + w (D + C_t)(2/D X_k + V_k)
                        [ - 2 w M a_{k+1} - (D + C_t) u_{k+1} in the w_1 column ]
        V_{k+1} = 2/D (X_{k+1} - X_k) - V_k,  W_{k+1} = 4/D^2 (X_{k+1} - X_k) - 4/D V_k - W_k
    with X_0 = [I 0 0], V_0 = [0 I 0] and W_0 from the equation of motion at
    phi_1 = 0.  ``n_steps`` (default S1) truncates the run (for sampled tests).
    Pinned by the discrete closed form of the linear case, by the discrete
    energy balance and by central finite differences.
    """
    n = q0.shape[0]
    w = float(omega1)
    Dl = 2.0 * np.pi / S1
    a0c, a1c, a2c = 4.0 / Dl ** 2, 4.0 / Dl, 2.0 / Dl
    M, D, K = model.M, model.D, model.K
    S = w * w * a0c * M + w * a2c * D + K
    q = q0.astype(np.float64).copy()
    u = u0.astype(np.float64).copy()
    # consistent initial acceleration from Eq. (E2) at phi_1 = 0
    f0, Kt0, Ct0 = fnl_and_tangent(model, q, w * u)
    e0 = forcing(model, 0.0, phis, rho)
    wM = w * w * M
    a = np.linalg.solve(wM, e0 - w * D @ u - K @ q - f0)
    if sens:
        X = np.zeros((n, 2 * n + 1))
        V = np.zeros((n, 2 * n + 1))
        X[:, :n] = np.eye(n)
        V[:, n:2 * n] = np.eye(n)
        rhs0 = -(K + Kt0) @ X - w * (D + Ct0) @ V
        rhs0[:, 2 * n] += -2.0 * w * M @ a - (D + Ct0) @ u
        W = np.linalg.solve(wM, rhs0)
    iters = []
    converged = True
    hist = [(q.copy(), u.copy(), a.copy())] if keep_history else None
    steps = S1 if n_steps is None else n_steps
    for k in range(steps):
        phi_next = (k + 1) * Dl
        b = forcing(model, phi_next, phis, rho) + wM @ (a0c * q + a1c * u + a) + w * D @ (a2c * q + u)
        qn = q.copy()                                  # predictor: previous displacement
        it = 0
        ok = False
        while it < maxit:
            un = a2c * (qn - q) - u
            fn, Kt, Ct = fnl_and_tangent(model, qn, w * un)
            r = S @ qn + fn - b
            Keff = S + Kt + w * a2c * Ct
            dq = -np.linalg.solve(Keff, r)
            qn = qn + dq
            it += 1
            if tol > 0 and np.max(np.abs(dq)) <= tol * np.max(np.abs(qn)):
                ok = True
                break
        if tol <= 0:
            ok = True
        converged = converged and ok
        iters.append(it)
        un = a2c * (qn - q) - u
        an = a0c * (qn - q) - a1c * u - a
        if sens:
            _, Kt, Ct = fnl_and_tangent(model, qn, w * un)
            Keff = S + Kt + w * a2c * Ct
            rhs = wM @ (a0c * X + a1c * V + W) + w * (D + Ct) @ (a2c * X + V)
            rhs[:, 2 * n] += -2.0 * w * M @ an - (D + Ct) @ un
            Xn = np.linalg.solve(Keff, rhs)
            Vn = a2c * (Xn - X) - V
            Wn = a0c * (Xn - X) - a1c * V - W
            X, V, W = Xn, Vn, Wn
        q, u, a = qn, un, an
        if keep_history:
            hist.append((q.copy(), u.copy(), a.copy()))
    res = TrajectoryResult(zT=np.concatenate([q, u]), newton_iters=iters, converged=converged,
                           history=hist)
    if sens:
        res.Phi = np.concatenate([X[:, :2 * n], V[:, :2 * n]], axis=0)
        res.dz_dw = np.concatenate([X[:, 2 * n], V[:, 2 * n]])
    return res


# -----------------------------------------------------------------------------
# Sec. 3.1 / 3.3: the FSE-Shooting residual and its Jacobian
# -----------------------------------------------------------------------------

@dataclass
class FSEProblem:
    """Precomputed tables for one (model, torus discretisation, rho)."""

    model: object
    S: list
    H: list
    S1: int
    rho: np.ndarray
    ktab: np.ndarray = None
    T: np.ndarray = None
    G: np.ndarray = None
    Gi: np.ndarray = None
    R: np.ndarray = None

    def __post_init__(self):
        for Sj, Hj in zip(self.S, self.H):
            if Sj < 2 * Hj + 1:
                raise ValueError("sampling rule S_j >= 2 H_j + 1 violated (Sec. 3.1)")
        self.rho = np.asarray(self.rho, dtype=np.float64)
        self.ktab = harmonic_table(self.H)
        self.T = sample_grid(self.S)
        self.G = gamma(self.ktab, self.T)
        self.Gi = gamma_inv(self.ktab, self.T)
        self.R = rotation(self.ktab, self.rho)

    @property
    def n(self):
        return self.model.n

    @property
    def U(self):
        return self.G.shape[1]

    @property
    def N(self):
        return self.G.shape[0]


@dataclass
class ResidualJacobian:
    R: np.ndarray                        # residual, Eq. (16), state-major (2n U~)
    Z2pi: np.ndarray                     # Z(2 pi), Eq. (21)
    zbar0: np.ndarray                    # (N, 2n) trajectory start points, Eq. (20)
    zbarT: np.ndarray                    # (N, 2n) trajectory end points
    Phi: Optional[np.ndarray] = None     # (N, 2n, 2n) monodromy blocks, Eq. (E8)
    dz_dw: Optional[np.ndarray] = None   # (N, 2n)
    J: Optional[np.ndarray] = None       # dense dR/dZ(0), Eq. (22)
    dR_dw: Optional[np.ndarray] = None   # dR/dw_1, Eq. (23) with rho fixed
    newton_iters: Optional[np.ndarray] = None
    converged: bool = True


def idft(prob, Z0):
    """Eq. (20): zbar(0, phi~) = (I_2n (x) Gamma) Z(0); returned as (N, 2n)."""
    C = Z0.reshape(2 * prob.n, prob.U)
    return (C @ prob.G.T).T


def dft_rotate(prob, zbarT):
    """Eq. (21) and Eq. (15): Z(2 pi) = (I (x) Gamma^-1) zbar(2 pi), Zhat = (I (x) R) Z(2 pi)."""
    Z2 = zbarT.T @ prob.Gi.T             # (2n, U~)
    Zhat = Z2 @ prob.R.T
    return Z2.reshape(-1), Zhat.reshape(-1)


def residual_jacobian(prob, Z0, omega1, want_jacobian=True, dense=True, tol=1e-10, maxit=20,
                      n_steps=None):
    """R(Z(0), w) = (I_2n (x) R(rho)) Z(2 pi) - Z(0)  (Eq. 16) by the pipeline of Eq. (17).

    With ``want_jacobian`` also returns the monodromy blocks and, if ``dense``,
    dR/dZ(0) of Eq. (22) and dR/dw_1 of Eq. (23) (rho fixed, so the rotation
    term of Eq. 23 vanishes: only the integration term remains).
    """
    n = prob.n
    zb0 = idft(prob, Z0)
    N = prob.N
    zbT = np.zeros((N, 2 * n))
    Phi = np.zeros((N, 2 * n, 2 * n)) if want_jacobian else None
    dzw = np.zeros((N, 2 * n)) if want_jacobian else None
    iters = []
    conv = True
    for s in range(N):
        tr = integrate_trajectory(prob.model, omega1, prob.rho, prob.T[:, s], zb0[s, :n],
                                  zb0[s, n:], prob.S1, tol=tol, maxit=maxit, sens=want_jacobian,
                                  n_steps=n_steps)
        zbT[s] = tr.zT
        iters.append(tr.newton_iters)
        conv = conv and tr.converged
        if want_jacobian:
            Phi[s] = tr.Phi
            dzw[s] = tr.dz_dw
    Z2, Zhat = dft_rotate(prob, zbT)
    out = ResidualJacobian(R=Zhat - Z0, Z2pi=Z2, zbar0=zb0, zbarT=zbT, Phi=Phi, dz_dw=dzw,
                           newton_iters=np.array(iters), converged=conv)
    if want_jacobian and dense:
        out.J = jacobian_dense(prob, Phi)
        out.dR_dw = jacobian_domega(prob, dzw)
    return out


def jacobian_dense(prob, Phi):
    """Eq. (22): dR/dZ(0) = (I (x) R Gamma^-1) blockdiag_s(Phi_s) (I (x) Gamma) - I.

    Entry [(i, u), (j, v)] = sum_s (R Gamma^-1)[u, s] Phi_s[i, j] Gamma[s, v] - delta.
    """
    RG = prob.R @ prob.Gi                # (U, N)
    J = np.einsum('us,sij,sv->iujv', RG, Phi, prob.G, optimize=True)
    m = 2 * prob.n * prob.U
    J = J.reshape(m, m)
    return J - np.eye(m)


def jacobian_apply(prob, Phi, v):
    """Eq. (22) applied to a vector without forming J: i-DFT, Phi_s, DFT, rotate, minus v."""
    zb = idft(prob, v)                   # (N, 2n)
    y = np.einsum('sij,sj->si', Phi, zb)
    _, Zhat = dft_rotate(prob, y)
    return Zhat - v


def jacobian_domega(prob, dz_dw):
    """Eq. (23), i = 1, rho fixed: dR/dw_1 = (I (x) R Gamma^-1) dzbar(2 pi)/dw_1."""
    _, out = dft_rotate(prob, dz_dw)
    return out


def newton_step(prob, Z0, omega1, tol=1e-10, maxit=20):
    """Sec. 3.3 step 6: one Newton-Raphson update Z(0) <- Z(0) - J^{-1} R (w_1 fixed)."""
    rj = residual_jacobian(prob, Z0, omega1, want_jacobian=True, dense=True, tol=tol, maxit=maxit)
    dZ = -np.linalg.solve(rj.J, rj.R)
    return Z0 + dZ, rj


def solve_torus(prob, Z0, omega1, rel_tol=1e-10, max_newton=20, tol=1e-10, maxit=20):
    """Newton-Raphson on Eq. (16) at fixed w_1 until ||R||_2 <= rel_tol * ||Z(0)||_2."""
    Z = Z0.copy()
    hist = []
    for _ in range(max_newton):
        rj = residual_jacobian(prob, Z, omega1, want_jacobian=True, dense=True, tol=tol, maxit=maxit)
        rn = float(np.linalg.norm(rj.R))
        hist.append(rn)
        if rn <= rel_tol * max(np.linalg.norm(Z), 1e-300):
            return Z, hist, True
        Z = Z - np.linalg.solve(rj.J, rj.R)
    rj = residual_jacobian(prob, Z, omega1, want_jacobian=False, tol=tol, maxit=maxit)
    rn = float(np.linalg.norm(rj.R))
    hist.append(rn)
    return Z, hist, rn <= rel_tol * max(np.linalg.norm(Z), 1e-300)


# -----------------------------------------------------------------------------
# App. F: Lyapunov exponents from the monodromy by-product
# -----------------------------------------------------------------------------

def lyapunov(prob, Phi, omega1, N_Ly, h):
    """First-order Lyapunov exponents sigma_1..sigma_h (1/s), App. F.

    Psi_s = D_w Phi_s D_w^{-1}, D_w = diag(I_n, w I_n) converts [q; u] to the
    physical [q; qdot] (Eq. F3).  Psi(phi~) is the trigonometric interpolant of
    the samples Psi_s with the same harmonics (coefficients Gamma^{-1} Psi),
    evaluated at phi~^{i-1} = 2 (i-1) pi rho.  Discrete Gram-Schmidt by QR:
    Q_i R_i = Psi(phi~^{i-1}) Q_{i-1}, Q_0 = I[:, :h];
    sigma_j = (1 / (N_Ly T_1)) sum_i ln |R_i[j, j]| (Eq. F2 at t = N_Ly T_1).
    """
    n2 = Phi.shape[1]
    n = n2 // 2
    w = float(omega1)
    dvec = np.concatenate([np.ones(n), w * np.ones(n)])
    Psi = Phi * dvec[None, :, None] / dvec[None, None, :]
    coef = np.einsum('us,sij->uij', prob.Gi, Psi)      # trigonometric coefficients
    T1 = 2.0 * np.pi / w
    Q = np.eye(n2)[:, :h]
    acc = np.zeros(h)
    for i in range(1, N_Ly + 1):
        phi = 2.0 * (i - 1) * np.pi * prob.rho
        Hrow = basis_row(prob.ktab, phi)
        Psi_i = np.einsum('u,uij->ij', Hrow, coef)
        A = Psi_i @ Q
        Q, Rr = np.linalg.qr(A)
        acc += np.log(np.abs(np.diag(Rr)))
    return acc / (N_Ly * T1)
