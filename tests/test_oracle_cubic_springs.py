"""Pins of the cubic spring forces of f_nl (Eq. 1) against their definitions.

The grounded spring adds k3 q_i^3 to row i; the difference spring with
s = q_i - q_j adds k3 s^3 to row i and its reaction -k3 s^3 to row j (Eq. 1 with
the springs of the benchmark shell and the beams).  These tests fix the scale
and the reaction sign of the force itself, independently of its tangent:
literal values worked by hand, two static equilibria with closed-form roots,
and the energy of a free undamped run measured with the spring potential
k3 s^4 / 4.  A mistake planted in the oracle's force (a factor 2 on k3, a
flipped reaction) is shown to fail each kind of check.
"""
import math

import numpy as np
import pytest
from scipy import optimize

from oracle import fse_oracle as O
from paper_2508_06302_gb300 import inputs as I


def _model(n, K, springs, M=None, D=None, F=None):
    """Dense model with the given springs [(type, dof_i, dof_j, k3)]."""
    m = len(springs)
    nl_type = np.array([s[0] for s in springs], np.int32)
    nl_dof = np.full((m, 6), -1, np.int32)
    nl_p = np.zeros((m, 6))
    for e, (t, i, j, k3) in enumerate(springs):
        nl_dof[e, 0] = i
        if t == I.NL_CUBIC_DIFF:
            nl_dof[e, 1] = j
        nl_p[e, 0] = k3
    return I.FEModel(name="springs", M=np.eye(n) if M is None else M,
                     D=np.zeros((n, n)) if D is None else D, K=np.asarray(K, float),
                     nl_type=nl_type, nl_dof=nl_dof, nl_p=nl_p,
                     F=np.zeros((1, n)) if F is None else F, omega_n1=1.0)


def test_grounded_spring_literal_values():
    # k3 = 2.5 on dof 1, q_1 = -0.7: f_1 = 2.5 * (-0.343) = -0.8575, K_t[1, 1] = 3 * 2.5 * 0.49 = 3.675
    m = _model(3, np.zeros((3, 3)), [(I.NL_CUBIC_GROUND, 1, -1, 2.5)])
    f, Kt, _ = O.fnl_and_tangent(m, np.array([0.3, -0.7, 1.1]), np.zeros(3))
    np.testing.assert_allclose(f, [0.0, -0.8575, 0.0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(Kt, np.diag([0.0, 3.675, 0.0]), rtol=0, atol=1e-14)


def test_difference_spring_literal_values_and_reaction():
    # k3 = 4 between dofs 0 and 2, s = 0.3 - 1.1 = -0.8: k3 s^3 = -2.048 on dof 0, +2.048 on dof 2;
    # tangent 3 k3 s^2 = 7.68 on the diagonal, -7.68 off it
    m = _model(3, np.zeros((3, 3)), [(I.NL_CUBIC_DIFF, 0, 2, 4.0)])
    f, Kt, _ = O.fnl_and_tangent(m, np.array([0.3, -0.7, 1.1]), np.zeros(3))
    np.testing.assert_allclose(f, [-2.048, 0.0, 2.048], rtol=0, atol=1e-14)
    assert f[0] + f[2] == 0.0          # action and reaction cancel
    assert f[0] < 0.0                  # q_0 < q_2: the spring pulls dof 0 up (restoring, like K q)
    np.testing.assert_allclose(Kt, [[7.68, 0, -7.68], [0, 0, 0], [-7.68, 0, 7.68]], rtol=0, atol=1e-13)


def _cardano(k, k3, F):
    """Real root of k q + k3 q^3 = F (k, k3 > 0: one real root)."""
    p, r = k / k3, -F / k3
    disc = math.sqrt((r / 2) ** 2 + (p / 3) ** 3)
    return np.cbrt(-r / 2 + disc) + np.cbrt(-r / 2 - disc)


def _static_root(model, F, x0):
    """K q + f_nl(q) = F solved with the oracle's force only (numerical Jacobian, no K_t)."""
    def g(q):
        f, _, _ = O.fnl_and_tangent(model, q, np.zeros_like(q))
        return model.K @ q + f - F
    sol, info, ier, msg = optimize.fsolve(g, x0, xtol=1e-14, full_output=True)
    # ier 3 ("no further improvement") at this xtol still means a root if the residual is tiny
    assert np.abs(g(sol)).max() <= 1e-10 * np.abs(F).max(), msg
    return sol


def _grounded_equilibrium_error():
    k, k3, F = 1e4, 1e8, 50.0
    m = _model(1, [[k]], [(I.NL_CUBIC_GROUND, 0, -1, k3)])
    q = _static_root(m, np.array([F]), np.array([F / k]))
    return abs(q[0] - _cardano(k, k3, F)) / abs(_cardano(k, k3, F))


def _series_equilibrium_error():
    # ground --k-- dof 0 --cubic k3-- dof 1 <- F: the chain carries F, so k q_0 = F and
    # k3 (q_1 - q_0)^3 = F, i.e. q_0 = F / k and q_1 = F / k + (F / k3)^(1/3)
    k, k3, F = 2e3, 5e7, 30.0
    m = _model(2, [[k, 0.0], [0.0, 0.0]], [(I.NL_CUBIC_DIFF, 0, 1, k3)])
    q = _static_root(m, np.array([0.0, F]), np.array([F / k, F / k + 0.5 * np.cbrt(F / k3)]))
    exact = np.array([F / k, F / k + np.cbrt(F / k3)])
    return np.abs(q - exact).max() / np.abs(exact).max()


def test_grounded_spring_static_equilibrium_is_the_cardano_root():
    assert _grounded_equilibrium_error() < 1e-12


def test_series_spring_static_equilibrium_closed_form():
    assert _series_equilibrium_error() < 1e-12


def _free_run_energy_drift(S1=4000):
    """Relative spread of E = w^2/2 u.M u + q.K q/2 + sum k3 s^4/4 over a free undamped run."""
    m = I.chain(4, c=0.0, k3=1e8, F=(0.0, 0.0))
    m.D = np.zeros_like(m.D)
    m.F = np.zeros_like(m.F)
    w1 = m.omega_n1
    rng = np.random.default_rng(11)
    q0 = 2e-2 * rng.standard_normal(m.n)   # the cubic energy is of the order of the linear one here
    tr = O.integrate_trajectory(m, w1, [0.5], np.array([0.0]), q0, np.zeros(m.n), S1, tol=0,
                                maxit=12, sens=False, keep_history=True)

    def potential(q):
        V = 0.0
        for e in range(m.n_nl):
            i, j = int(m.nl_dof[e, 0]), int(m.nl_dof[e, 1])
            s = q[i] - (q[j] if int(m.nl_type[e]) == I.NL_CUBIC_DIFF else 0.0)
            V += 0.25 * m.nl_p[e, 0] * s ** 4
        return V

    E = np.array([0.5 * w1 ** 2 * u @ m.M @ u + 0.5 * q @ m.K @ q + potential(q) for q, u, _ in tr.history])
    lin = 0.5 * q0 @ m.K @ q0
    assert potential(q0) > 0.2 * lin          # the nonlinearity carries real energy
    return np.ptp(E) / E[0]


def test_free_undamped_run_conserves_spring_energy():
    # the trapezoidal work of the cubic force differs from the potential change by O(Delta^2)
    assert _free_run_energy_drift() < 1e-4


@pytest.mark.parametrize("mistake", ["k3_twice", "reaction_flipped"])
def test_planted_force_mistakes_fail_the_pins(monkeypatch, mistake):
    """A consistent error in f and K_t (which the finite-difference pin cannot see) fails here."""
    real = O.fnl_and_tangent

    def wrong(model, q, qdot):
        f, Kt, Ct = real(model, q, qdot)
        if mistake == "k3_twice":
            return 2.0 * f, 2.0 * Kt, Ct
        f = f.copy()
        for e in range(model.n_nl):
            if int(model.nl_type[e]) == I.NL_CUBIC_DIFF:
                i, j = int(model.nl_dof[e, 0]), int(model.nl_dof[e, 1])
                s = q[i] - q[j]
                f[j] += 2.0 * model.nl_p[e, 0] * s ** 3   # -k3 s^3 becomes +k3 s^3
        return f, Kt, Ct

    monkeypatch.setattr(O, "fnl_and_tangent", wrong)
    if mistake == "k3_twice":
        assert _grounded_equilibrium_error() > 1e-3
        assert _free_run_energy_drift(S1=400) > 1e-2
    else:
        with pytest.raises(AssertionError):
            test_difference_spring_literal_values_and_reaction()
        try:
            err = _series_equilibrium_error()
        except AssertionError:      # no root at all is a failure too
            err = np.inf
        assert err > 1e-3
