"""Seeded synthetic finite-element inputs for FSE-Shooting workloads.

This module builds the structural models (M, D, K, nonlinear element
records, forcing vectors) and the run parameters that both the CUDA path and
the CPU oracle consume.  It holds none of the shooting method's arithmetic:
no Newmark step, no AFT, no residual.  Everything here is textbook
finite-element assembly (Euler-Bernoulli / von Karman beams, Q4 membrane,
ACM rectangular plate bending) plus seeded random draws, so that the same
seed always yields bit-identical inputs on every machine.

The equation of motion the models feed is Eq. (1) with Theta = I and the
forcing of Eq. (25):  M q'' + D q' + K q + f_nl(q) = sum_i F_i cos(w_i t).

Nonlinear element records (``nl_type``, ``nl_dof``, ``nl_p``) follow the
C-ABI ``fse_nl_elem`` layout:

* type 1, cubic grounded spring:   f[dof0] += p0 * q[dof0]^3
* type 2, cubic difference spring: d = q[dof0]-q[dof1]; f[dof0] += p0 d^3, f[dof1] -= p0 d^3
* type 3, 2-node von Karman beam element, dofs (u1, w1, th1, u2, w2, th2),
  p0 = EA, p1 = element length; a dof of -1 is clamped (zero).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

NL_CUBIC_GROUND = 1
NL_CUBIC_DIFF = 2
NL_VK_BEAM = 3
NL_VDP = 4             # self-excited (van der Pol) damper: f[d0] += p0 (q[d0]^2 - 1) qdot[d0]

GOLDEN = (1.0 + math.sqrt(5.0)) / 2.0


@dataclasses.dataclass
class FEModel:
    """Dense second-order structural model, Eq. (1) of the paper."""

    name: str
    M: np.ndarray          # (n, n) float64, symmetric positive definite
    D: np.ndarray          # (n, n) float64 viscous damping
    K: np.ndarray          # (n, n) float64 linear stiffness
    nl_type: np.ndarray    # (m,) int32
    nl_dof: np.ndarray     # (m, 6) int32, -1 = unused / clamped
    nl_p: np.ndarray       # (m, 6) float64
    F: np.ndarray          # (e, n) forcing amplitude vectors, Eq. (25)
    omega_n1: float        # first undamped natural frequency [rad/s]

    @property
    def n(self) -> int:
        return self.M.shape[0]

    @property
    def n_nl(self) -> int:
        return int(self.nl_type.shape[0])

    def linear_only(self) -> "FEModel":
        """Same model with every nonlinear element removed (f_nl = 0)."""
        return dataclasses.replace(
            self, nl_type=self.nl_type[:0].copy(), nl_dof=self.nl_dof[:0].copy(),
            nl_p=self.nl_p[:0].copy())


@dataclasses.dataclass
class Workload:
    """One FSE-Shooting problem: model + torus discretisation + frequencies."""

    name: str
    model: FEModel
    d: int                 # number of base frequencies
    S: list                # S_j, j = 2..d (trajectory grid), N = prod(S)
    H: list                # highest harmonic H_j, K_j = [0..H_j]
    S1: int                # Newmark steps per period T1
    rho: list              # rho_j = w_j / w_1, j = 2..d (fixed)
    omega1: float          # w_1 [rad/s]
    newton_tol: float = 1e-10
    newton_maxit: int = 20

    @property
    def N(self) -> int:
        return int(np.prod(self.S)) if self.S else 1

    @property
    def U_tilde(self) -> int:
        return int(np.prod([2 * h + 1 for h in self.H])) if self.H else 1

    @property
    def n_unknowns(self) -> int:
        return 2 * self.model.n * self.U_tilde

    @property
    def omega(self) -> np.ndarray:
        return np.array([self.omega1] + [r * self.omega1 for r in self.rho])


# ----------------------------------------------------------------------------
# element matrices (textbook FE)
# ----------------------------------------------------------------------------

def _gauss(npts: int):
    x, w = np.polynomial.legendre.leggauss(npts)
    return x, w


def beam_bending_element(EI: float, rhoA: float, L: float):
    """Hermite cubic Euler-Bernoulli element, dofs (w1, th1, w2, th2)."""
    k = EI / L**3 * np.array([[12, 6 * L, -12, 6 * L],
                              [6 * L, 4 * L * L, -6 * L, 2 * L * L],
                              [-12, -6 * L, 12, -6 * L],
                              [6 * L, 2 * L * L, -6 * L, 4 * L * L]], dtype=np.float64)
    m = rhoA * L / 420.0 * np.array([[156, 22 * L, 54, -13 * L],
                                     [22 * L, 4 * L * L, 13 * L, -3 * L * L],
                                     [54, 13 * L, 156, -22 * L],
                                     [-13 * L, -3 * L * L, -22 * L, 4 * L * L]], dtype=np.float64)
    return k, m


def bar_element(EA: float, rhoA: float, L: float):
    k = EA / L * np.array([[1.0, -1.0], [-1.0, 1.0]])
    m = rhoA * L / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])
    return k, m


def _first_mode(M: np.ndarray, K: np.ndarray) -> float:
    import scipy.linalg
    w2 = scipy.linalg.eigh(K, M, eigvals_only=True, subset_by_index=[0, 0])[0]
    return float(math.sqrt(w2))


def _empty_nl():
    return (np.zeros((0,), np.int32), np.full((0, 6), -1, np.int32), np.zeros((0, 6)))


# ----------------------------------------------------------------------------
# Config: clamped-clamped Euler-Bernoulli beam with a grounded cubic spring
# ----------------------------------------------------------------------------

def eb_beam(n_el: int = 10, E: float = 210e9, rho: float = 7800.0, L: float = 1.0,
            b: float = 0.02, h: float = 0.01, alpha: float = 1e-2, beta: float = 1e-5,
            k3: float = 1e9, F1: float = 5.0, F2: float = 5.0) -> FEModel:
    """Clamped-clamped beam, n_el Hermite elements, dofs (w, th) per interior node.

    Bending about the thin axis: I = b h^3 / 12.  D = alpha M + beta K.
    A cubic spring to ground acts on the midspan deflection, where both
    forcing components are applied.
    """
    A = b * h
    I = b * h**3 / 12.0
    Le = L / n_el
    nn = n_el + 1
    Kg = np.zeros((2 * nn, 2 * nn))
    Mg = np.zeros((2 * nn, 2 * nn))
    ke, me = beam_bending_element(E * I, rho * A, Le)
    for e in range(n_el):
        idx = [2 * e, 2 * e + 1, 2 * e + 2, 2 * e + 3]
        Kg[np.ix_(idx, idx)] += ke
        Mg[np.ix_(idx, idx)] += me
    free = list(range(2, 2 * nn - 2))
    K = Kg[np.ix_(free, free)].copy()
    M = Mg[np.ix_(free, free)].copy()
    D = alpha * M + beta * K
    n = K.shape[0]
    mid_node = n_el // 2                 # global node index
    w_mid = 2 * (mid_node - 1)           # interior node numbering starts at node 1
    nl_type = np.array([NL_CUBIC_GROUND], np.int32)
    nl_dof = np.full((1, 6), -1, np.int32)
    nl_dof[0, 0] = w_mid
    nl_p = np.zeros((1, 6))
    nl_p[0, 0] = k3
    F = np.zeros((2, n))
    F[0, w_mid] = F1
    F[1, w_mid] = F2
    return FEModel("eb_beam_%d" % n, M, D, K, nl_type, nl_dof, nl_p, F, _first_mode(M, K))


# ----------------------------------------------------------------------------
# Config: clamped-clamped von Karman beam (axial + bending, 3 dofs per node)
# ----------------------------------------------------------------------------

def vk_beam(n_el: int = 150, E: float = 4.5e10, rho: float = 1780.0, L: float = 2.7,
            b: float = 0.01, h: float = 0.01, alpha: float = 0.0, beta: float = 2.0 / 9.0 * 1e-4,
            F1: float = 20.0, F2: float = 20.0) -> FEModel:
    """Clamped-clamped von Karman beam, dofs [x_i, v_i, th_i] per interior node.

    3 n_el - 3 free dofs (Sec. 4.1).  Forcing on dof 3 n_el / 2 - 1 (1-based),
    the midspan transverse displacement (Eq. 25).  The geometric (axial
    stretching) nonlinearity is carried by one type-3 record per element.
    """
    A = b * h
    I = b * h**3 / 12.0
    Le = L / n_el
    nn = n_el + 1
    ndof = 3 * nn
    Kg = np.zeros((ndof, ndof))
    Mg = np.zeros((ndof, ndof))
    kb, mb = beam_bending_element(E * I, rho * A, Le)
    ka, ma = bar_element(E * A, rho * A, Le)
    for e in range(n_el):
        ia = [3 * e, 3 * e + 3]
        ib = [3 * e + 1, 3 * e + 2, 3 * e + 4, 3 * e + 5]
        Kg[np.ix_(ia, ia)] += ka
        Mg[np.ix_(ia, ia)] += ma
        Kg[np.ix_(ib, ib)] += kb
        Mg[np.ix_(ib, ib)] += mb
    free = list(range(3, ndof - 3))
    gmap = -np.ones(ndof, np.int64)
    gmap[free] = np.arange(len(free))
    K = Kg[np.ix_(free, free)].copy()
    M = Mg[np.ix_(free, free)].copy()
    D = alpha * M + beta * K
    n = K.shape[0]
    nl_type = np.full((n_el,), NL_VK_BEAM, np.int32)
    nl_dof = np.full((n_el, 6), -1, np.int32)
    nl_p = np.zeros((n_el, 6))
    for e in range(n_el):
        g = [3 * e, 3 * e + 1, 3 * e + 2, 3 * e + 3, 3 * e + 4, 3 * e + 5]
        nl_dof[e] = [gmap[x] for x in g]
        nl_p[e, 0] = E * A
        nl_p[e, 1] = Le
    F = np.zeros((2, n))
    fdof = 3 * n_el // 2 - 1 - 1         # 1-based index 3N/2-1 -> 0-based
    F[0, fdof] = F1
    F[1, fdof] = F2
    return FEModel("vk_beam_%d" % n, M, D, K, nl_type, nl_dof, nl_p, F, _first_mode(M, K))


# ----------------------------------------------------------------------------
# plate / shell elements on a regular rectangular grid
# ----------------------------------------------------------------------------

def _acm_matrices(a: float, bb: float, Dflex: float, nu: float, rho_t: float):
    """ACM (Adini-Clough-Melosh) 12-dof rectangle a x bb.

    Node order (0,0), (a,0), (a,bb), (0,bb); dofs per node (w, th_x, th_y)
    with th_x = dw/dy and th_y = -dw/dx.  Stiffness from the exact
    integral of B^T D B; consistent translational mass rho t int N^T N.
    """
    def P(x, y):
        return np.array([1, x, y, x * x, x * y, y * y, x**3, x * x * y, x * y * y, y**3,
                         x**3 * y, x * y**3], dtype=np.float64)

    def Px(x, y):
        return np.array([0, 1, 0, 2 * x, y, 0, 3 * x * x, 2 * x * y, y * y, 0, 3 * x * x * y, y**3])

    def Py(x, y):
        return np.array([0, 0, 1, 0, x, 2 * y, 0, x * x, 2 * x * y, 3 * y * y, x**3, 3 * x * y * y])

    def Pxx(x, y):
        return np.array([0, 0, 0, 2, 0, 0, 6 * x, 2 * y, 0, 0, 6 * x * y, 0])

    def Pyy(x, y):
        return np.array([0, 0, 0, 0, 0, 2, 0, 0, 2 * x, 6 * y, 0, 6 * x * y])

    def Pxy(x, y):
        return np.array([0, 0, 0, 0, 1, 0, 0, 2 * x, 2 * y, 0, 3 * x * x, 3 * y * y])

    nodes = [(0.0, 0.0), (a, 0.0), (a, bb), (0.0, bb)]
    C = np.zeros((12, 12))
    for i, (x, y) in enumerate(nodes):
        C[3 * i] = P(x, y)
        C[3 * i + 1] = Py(x, y)
        C[3 * i + 2] = -Px(x, y)
    Ci = np.linalg.inv(C)
    Db = Dflex * np.array([[1, nu, 0], [nu, 1, 0], [0, 0, (1 - nu) / 2]])
    xg, wg = _gauss(5)
    k = np.zeros((12, 12))
    m = np.zeros((12, 12))
    for xi, wi in zip(xg, wg):
        for yj, wj in zip(xg, wg):
            x = 0.5 * a * (xi + 1)
            y = 0.5 * bb * (yj + 1)
            w = wi * wj * 0.25 * a * bb
            B = -np.vstack([Pxx(x, y), Pyy(x, y), 2 * Pxy(x, y)]) @ Ci
            k += w * B.T @ Db @ B
            N = P(x, y) @ Ci
            m += w * rho_t * np.outer(N, N)
    return 0.5 * (k + k.T), 0.5 * (m + m.T)


def _q4_membrane(a: float, bb: float, E: float, nu: float, t: float, rho: float):
    """Bilinear plane-stress rectangle, dofs (u, v) per node, same node order."""
    Dm = E * t / (1 - nu * nu) * np.array([[1, nu, 0], [nu, 1, 0], [0, 0, (1 - nu) / 2]])
    xg, wg = _gauss(2)
    xg3, wg3 = _gauss(3)
    k = np.zeros((8, 8))
    m = np.zeros((8, 8))
    sx = np.array([-1, 1, 1, -1.0])
    sy = np.array([-1, -1, 1, 1.0])

    def shape(xi, eta):
        N = 0.25 * (1 + sx * xi) * (1 + sy * eta)
        dNx = 0.25 * sx * (1 + sy * eta) * (2.0 / a)
        dNy = 0.25 * sy * (1 + sx * xi) * (2.0 / bb)
        return N, dNx, dNy

    for xi, wi in zip(xg, wg):
        for eta, wj in zip(xg, wg):
            _, dNx, dNy = shape(xi, eta)
            B = np.zeros((3, 8))
            B[0, 0::2] = dNx
            B[1, 1::2] = dNy
            B[2, 0::2] = dNy
            B[2, 1::2] = dNx
            k += wi * wj * 0.25 * a * bb * B.T @ Dm @ B
    for xi, wi in zip(xg3, wg3):
        for eta, wj in zip(xg3, wg3):
            N, _, _ = shape(xi, eta)
            Nm = np.zeros((2, 8))
            Nm[0, 0::2] = N
            Nm[1, 1::2] = N
            m += wi * wj * 0.25 * a * bb * rho * t * Nm.T @ Nm
    return k, m


def _grid_plate(nx: int, ny: int, Lx: float, Ly: float, E: float, nu: float, rho: float,
                t: float, dofs_per_node: int):
    """Clamped rectangular plate (3 dofs/node) or flat shell (6 dofs/node).

    Nodes (i, j), i = 0..nx along x, j = 0..ny along y.  All edge nodes are
    clamped.  Free nodes are numbered with j (the short side) fastest, which
    keeps the half-bandwidth near (ny + 1) * dofs_per_node.
    Returns M, K, free-node lookup and coordinates.
    """
    a = Lx / nx
    bb = Ly / ny
    Dflex = E * t**3 / (12 * (1 - nu * nu))
    kb, mb = _acm_matrices(a, bb, Dflex, nu, rho * t)
    if dofs_per_node == 6:
        km, mm = _q4_membrane(a, bb, E, nu, t, rho)
    free_id = -np.ones((nx + 1, ny + 1), np.int64)
    cnt = 0
    for i in range(1, nx):
        for j in range(1, ny):
            free_id[i, j] = cnt
            cnt += 1
    n = cnt * dofs_per_node
    K = np.zeros((n, n))
    M = np.zeros((n, n))
    if dofs_per_node == 3:
        off_w = 0
    else:
        off_w = 2
    # drilling stiffness / inertia for the 6-dof shell (decoupled, textbook penalty choice)
    k_drill = 1e-3 * Dflex
    m_drill_per_area = rho * t**3 / 12.0
    for i in range(nx):
        for j in range(ny):
            corner = [(i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)]
            ids = [free_id[c] for c in corner]
            # bending: local dofs 3c + {0,1,2} -> node offset off_w + {0,1,2}
            gb = []
            for c, nid in enumerate(ids):
                for r in range(3):
                    gb.append(-1 if nid < 0 else nid * dofs_per_node + off_w + r)
            for p_ in range(12):
                if gb[p_] < 0:
                    continue
                for q_ in range(12):
                    if gb[q_] < 0:
                        continue
                    K[gb[p_], gb[q_]] += kb[p_, q_]
                    M[gb[p_], gb[q_]] += mb[p_, q_]
            if dofs_per_node == 6:
                gm = []
                for c, nid in enumerate(ids):
                    for r in range(2):
                        gm.append(-1 if nid < 0 else nid * 6 + r)
                for p_ in range(8):
                    if gm[p_] < 0:
                        continue
                    for q_ in range(8):
                        if gm[q_] < 0:
                            continue
                        K[gm[p_], gm[q_]] += km[p_, q_]
                        M[gm[p_], gm[q_]] += mm[p_, q_]
                for nid in ids:
                    if nid >= 0:
                        K[nid * 6 + 5, nid * 6 + 5] += 0.25 * k_drill
                        M[nid * 6 + 5, nid * 6 + 5] += 0.25 * m_drill_per_area * a * bb
    K = 0.5 * (K + K.T)
    M = 0.5 * (M + M.T)
    return M, K, free_id, a, bb


def kirchhoff_plate(nx: int = 10, ny: int = 10, Lx: float = 1.0, Ly: float = 1.0,
                    E: float = 210e9, nu: float = 0.3, rho: float = 7800.0, t: float = 0.01,
                    alpha: float = 1e-2, beta: float = 1e-5, n_springs: int = 40,
                    F: float = 5.0, e_count: int = 3, seed: int = 0) -> FEModel:
    """Clamped square ACM plate, 3 dofs (w, th_x, th_y) per interior node.

    ``n_springs`` grounded cubic springs on w at seeded distinct nodes with
    k3 ~ U[1e8, 1e9]; all ``e_count`` forcing components act on w at one
    seeded node.  Draw order: spring nodes, spring k3, forcing node.
    """
    M, K, free_id, _, _ = _grid_plate(nx, ny, Lx, Ly, E, nu, rho, t, 3)
    D = alpha * M + beta * K
    n = K.shape[0]
    n_nodes = n // 3
    rng = np.random.default_rng(seed)
    nodes = rng.choice(n_nodes, n_springs, replace=False)
    k3 = rng.uniform(1e8, 1e9, n_springs)
    fnode = int(rng.integers(n_nodes))
    nl_type = np.full((n_springs,), NL_CUBIC_GROUND, np.int32)
    nl_dof = np.full((n_springs, 6), -1, np.int32)
    nl_p = np.zeros((n_springs, 6))
    nl_dof[:, 0] = 3 * nodes
    nl_p[:, 0] = k3
    Fv = np.zeros((e_count, n))
    Fv[:, 3 * fnode] = F
    return FEModel("acm_plate_%d" % n, M, D, K, nl_type, nl_dof, nl_p, Fv, _first_mode(M, K))


def flat_shell(nx: int = 25, ny: int = 14, Lx: float = 2.0, Ly: float = 1.0, E: float = 70e9,
               nu: float = 0.33, rho: float = 2700.0, t: float = 0.01, visc: float = 1e5,
               zeta1: float = 0.01, F1: float = 40.0, F2: float = 20.0, seed: int = 0) -> FEModel:
    """Flat rectangular clamped shell: Q4 membrane + ACM bending + drilling, 6 dofs/node.

    dofs per node (u, v, w, th_x, th_y, th_z).  Rayleigh damping with
    beta = visc / E (material damping rate over modulus) and alpha set so
    that the first mode has damping ratio ``zeta1``.  Cubic springs
    k3 ~ U[1e8, 1e9] (seeded) on w_i - w_j for every grid-adjacent pair of
    free nodes, enumerated row-major (free node order), horizontal (x)
    neighbours first, then vertical (y).  Forcing on w at the free node
    nearest (Lx/4, Ly/2).
    """
    M, K, free_id, a, bb = _grid_plate(nx, ny, Lx, Ly, E, nu, rho, t, 6)
    n = K.shape[0]
    w1 = _first_mode(M, K)
    beta = visc / E
    alpha = 2 * w1 * (zeta1 - beta * w1 / 2)
    D = alpha * M + beta * K
    pairs = []
    for j in range(1, ny):                 # horizontal neighbours (i, j) - (i+1, j)
        for i in range(1, nx - 1):
            pairs.append((free_id[i, j], free_id[i + 1, j]))
    for j in range(1, ny - 1):             # vertical neighbours (i, j) - (i, j+1)
        for i in range(1, nx):
            pairs.append((free_id[i, j], free_id[i, j + 1]))
    rng = np.random.default_rng(seed)
    k3 = rng.uniform(1e8, 1e9, len(pairs))
    m = len(pairs)
    nl_type = np.full((m,), NL_CUBIC_DIFF, np.int32)
    nl_dof = np.full((m, 6), -1, np.int32)
    nl_p = np.zeros((m, 6))
    for s, (p0, p1) in enumerate(pairs):
        nl_dof[s, 0] = p0 * 6 + 2
        nl_dof[s, 1] = p1 * 6 + 2
        nl_p[s, 0] = k3[s]
    ix = int(round((Lx / 4) / a))
    jy = int(round((Ly / 2) / bb))
    fnode = free_id[min(max(ix, 1), nx - 1), min(max(jy, 1), ny - 1)]
    Fv = np.zeros((2, n))
    Fv[0, fnode * 6 + 2] = F1
    Fv[1, fnode * 6 + 2] = F2
    return FEModel("flat_shell_%d" % n, M, D, K, nl_type, nl_dof, nl_p, Fv, w1)


def chain(n: int = 8, m: float = 1.0, k: float = 1e4, c: float = 1.0, k3: float = 1e8,
          F: tuple = (1.0, 0.5)) -> FEModel:
    """Fixed-fixed spring-mass chain: a tiny model for quick tests.

    Unit masses, linear springs k between neighbours and to the walls,
    damping D = c/2 M + c/(2k) K, cubic difference springs (k3/2) between
    neighbours and a grounded cubic spring k3 at the first mass.  Forcing
    component i acts on the middle mass with amplitude F[i].
    """
    K = np.zeros((n, n))
    for i in range(n):
        K[i, i] = 2 * k
        if i + 1 < n:
            K[i, i + 1] = K[i + 1, i] = -k
    M = m * np.eye(n)
    D = 0.5 * c * M / m + 0.5 * (c / k) * K
    nl_type = [NL_CUBIC_GROUND] + [NL_CUBIC_DIFF] * (n - 1)
    nl_dof = np.full((n, 6), -1, np.int32)
    nl_p = np.zeros((n, 6))
    nl_dof[0, 0] = 0
    nl_p[0, 0] = k3
    for i in range(n - 1):
        nl_dof[i + 1, 0] = i
        nl_dof[i + 1, 1] = i + 1
        nl_p[i + 1, 0] = 0.5 * k3
    Fv = np.zeros((len(F), n))
    for i, f in enumerate(F):
        Fv[i, n // 2] = f
    return FEModel("chain_%d" % n, M, D, K, np.array(nl_type, np.int32), nl_dof, nl_p, Fv,
                   _first_mode(M, K))


def van_der_pol(omega_n: float = 10.0, eps: float = 0.2, F: tuple = (1.0,)) -> FEModel:
    """One self-excited oscillator q'' - eps omega_n (1 - q^2) q' + omega_n^2 q = sum F_i cos(w_i t).

    Unit mass, no viscous damping, the textbook van der Pol damper as element type NL_VDP
    (p0 = eps omega_n).  Its limit cycle (amplitude near 2, frequency near omega_n for small
    eps) supplies a base frequency that no forcing defines: with e forcing components and
    d > e base frequencies the remaining ones are unknowns of the torus (Sec. 3.2).
    """
    M = np.eye(1)
    D = np.zeros((1, 1))
    K = np.array([[omega_n * omega_n]])
    nl_type = np.array([NL_VDP], np.int32)
    nl_dof = np.full((1, 6), -1, np.int32)
    nl_dof[0, 0] = 0
    nl_p = np.zeros((1, 6))
    nl_p[0, 0] = eps * omega_n
    Fv = np.array(F, dtype=np.float64).reshape(-1, 1)
    return FEModel("van_der_pol", M, D, K, nl_type, nl_dof, nl_p, Fv, omega_n)


# ----------------------------------------------------------------------------
# the named workloads
# ----------------------------------------------------------------------------

def workload_beam18(**kw) -> Workload:
    """18-dof clamped-clamped beam, d=2, N=16 (H=7), S1=128, tol 1e-10."""
    m = eb_beam()
    w1 = 1.1 * m.omega_n1
    wl = Workload("beam18_d2_N16_H7_S128", m, 2, [16], [7], 128, [GOLDEN], w1, 1e-10, 20)
    return dataclasses.replace(wl, **kw) if kw else wl


def workload_vkbeam447(**kw) -> Workload:
    """447-dof von Karman beam, d=2, N=64 (H=31), S1=512."""
    m = vk_beam()
    w1 = 1.1 * m.omega_n1
    wl = Workload("vkbeam447_d2_N64_H31_S512", m, 2, [64], [31], 512, [GOLDEN], w1, 1e-10, 20)
    return dataclasses.replace(wl, **kw) if kw else wl


def workload_plate243(**kw) -> Workload:
    """243-dof ACM plate with 40 springs, d=3, 16x16 trajectories (H2=H3=7), S1=400."""
    m = kirchhoff_plate()
    w1 = 1.1 * m.omega_n1
    wl = Workload("plate243_d3_N256_H7x7_S400", m, 3, [16, 16], [7, 7], 400,
                  [math.sqrt(2.0), math.sqrt(3.0)], w1, 1e-10, 20)
    return dataclasses.replace(wl, **kw) if kw else wl


def workload_shell1872(**kw) -> Workload:
    """1872-dof flat clamped shell, d=2, N=64 (H=31), S1=1000."""
    m = flat_shell()
    w1 = 1.0 * m.omega_n1
    wl = Workload("shell1872_d2_N64_H31_S1000", m, 2, [64], [31], 1000, [GOLDEN], w1, 1e-10, 20)
    return dataclasses.replace(wl, **kw) if kw else wl


def shell_batch_points(model: Optional[FEModel] = None):
    """The 8 batched continuation points of uneven trajectory count.

    N_i = {32, 36, ..., 64} with H_i = floor((N_i - 1) / 2) so that the
    sampling rule S >= 2H + 1 holds, at w1 = w_n1 * {0.95, 1.0, ..., 1.3}.
    """
    m = model if model is not None else flat_shell()
    Ns = [32, 36, 40, 44, 48, 52, 56, 64]
    facs = [0.95, 1.0, 1.05, 1.1, 1.15, 1.2, 1.25, 1.3]
    out = []
    for Ni, f in zip(Ns, facs):
        out.append(Workload("shell%d_d2_N%d_H%d_S1000" % (m.n, Ni, (Ni - 1) // 2), m, 2, [Ni],
                            [(Ni - 1) // 2], 1000, [GOLDEN], f * m.omega_n1, 1e-10, 20))
    return out


def random_coeffs(n: int, U_tilde: int, scale: float, seed: int) -> np.ndarray:
    """Seeded random Fourier coefficient vector Z(0) (state-major, 2n*U~)."""
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal(2 * n * U_tilde)


def mlp_init(n_in: int = 3, n_hidden: int = 256, n_out: int = 64, seed: int = 0) -> dict:
    """Seeded Glorot-uniform weights and zero biases of the 3-layer predictor MLP.

    Draw order: W1, W2, W3 (each row-major, out x in).
    """
    rng = np.random.default_rng(seed)

    def glorot(fo, fi):
        lim = math.sqrt(6.0 / (fi + fo))
        return rng.uniform(-lim, lim, (fo, fi))

    W1 = glorot(n_hidden, n_in)
    W2 = glorot(n_hidden, n_hidden)
    W3 = glorot(n_out, n_hidden)
    return {"W1": W1, "b1": np.zeros(n_hidden), "W2": W2, "b2": np.zeros(n_hidden),
            "W3": W3, "b3": np.zeros(n_out)}
