"""Outer Newton step with the matrix-free GMRES solve of J dZ = -R (Sec. 3.3
step 6 with the structured products of Eq. 22), through the C ABI: it must give
the dense-LU update, and a torus converged with it must equal the oracle's."""
import numpy as np
import pytest

from oracle import fse_oracle as O
from paper_2508_06302_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _fse():
    from paper_2508_06302_gb300 import fse
    return fse


def _ctx(fse, name):
    if name == "vk87":
        m = I.vk_beam(n_el=30, F1=1.0, F2=1.0)
        return m, fse.Context(m, 2, [5], [2], [I.GOLDEN], 48, newton_tol=0, newton_maxit=16), 1.1
    m = I.flat_shell(nx=6, ny=4)
    return m, fse.Context(m, 2, [5], [2], [I.GOLDEN], 20, newton_tol=0, newton_maxit=16), 1.0


@pytest.mark.parametrize("name", ["vk87", "shell90"])
def test_gmres_update_equals_dense_update(name):
    fse = _fse()
    m, ctx, f = _ctx(fse, name)
    w1 = f * m.omega_n1
    Z = I.random_coeffs(m.n, ctx.U, 1e-6 if name == "vk87" else 1e-4, seed=5)
    ctx.set_linear_solver("dense")
    Zd, rn_d, rc_d = ctx.newton_step(Z.copy(), w1)
    assert ctx.linear_stats() == (0, 0.0)
    ctx.set_linear_solver("gmres", rel_tol=1e-12, restart=60, max_iters=600)
    Zg, rn_g, rc_g = ctx.newton_step(Z.copy(), w1)
    it, rel = ctx.linear_stats()
    assert rc_g == 0 and 0 < it <= 600 and rel <= 1e-12
    assert rn_d == rn_g
    dZd, dZg = Zd - Z, Zg - Z
    assert np.linalg.norm(dZg - dZd) <= 1e-8 * np.linalg.norm(dZd)
    ctx.close()


def test_gmres_newton_converges_to_oracle_torus():
    fse = _fse()
    m = I.eb_beam()
    w1 = 1.1 * m.omega_n1
    ctx = fse.Context(m, 2, [16], [7], [I.GOLDEN], 64, newton_tol=0, newton_maxit=6)
    ctx.set_linear_solver("gmres", rel_tol=1e-11, restart=30, max_iters=300)
    Z = np.zeros(ctx.n_unknowns)
    for _ in range(8):
        Z, rn, rc = ctx.newton_step(Z, w1)
    prob = O.FSEProblem(m, [16], [7], 64, [I.GOLDEN])
    Zr, hist, ok = O.solve_torus(prob, np.zeros(ctx.n_unknowns), w1, rel_tol=1e-12, tol=0, maxit=6)
    assert ok
    assert np.linalg.norm(Z - Zr) <= 1e-9 * np.linalg.norm(Zr)
    ctx.close()


def test_gmres_continuation_with_chord_corrector():
    """Continuation with GMRES and the chord corrector lands on the same tori as full Newton + LU."""
    fse = _fse()
    m = I.eb_beam()
    ctx = fse.Context(m, 2, [16], [7], [I.GOLDEN], 64, newton_tol=0, newton_maxit=6)
    omegas = m.omega_n1 * np.linspace(1.05, 1.12, 4)
    Zd, pd, rc1 = fse.fse_continue(ctx, omegas, np.zeros(ctx.n_unknowns), rel_tol=1e-11, max_newton=10)
    ctx.set_linear_solver("gmres", rel_tol=1e-10, restart=30, max_iters=300)
    Zg, pg, rc2 = fse.fse_continue(ctx, omegas, np.zeros(ctx.n_unknowns), rel_tol=1e-11, max_newton=20, chord=True)
    assert rc1 == 0 and rc2 == 0
    assert np.abs(Zg - Zd).max() <= 1e-8 * np.abs(Zd).max()
    # the chord corrector evaluates the Jacobian once per point
    assert all(p["evals"] == p["newton_iters"] + 1 for p in pg)
    ctx.close()


def test_linear_solver_rejects_bad_settings():
    fse = _fse()
    m = I.chain(4)
    ctx = fse.Context(m, 2, [7], [3], [0.5], 16)
    for args in [("gmres", 0.0, 10, 10), ("gmres", 1e-8, 0, 10), ("gmres", 1e-8, 300, 10)]:
        with pytest.raises(fse.FSEError) as ei:
            ctx.set_linear_solver(*args)
        assert ei.value.code == fse.FSE_EINVAL
    ctx.close()
