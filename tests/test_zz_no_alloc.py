"""fse_lyapunov_noalloc (static device scratch, no allocation) against
fse_lyapunov, through the C ABI.

Collected last on purpose: it must give the same exponents whether it is the
first call of the process to touch the static scratch or whether other
contexts ran before it.  Two calls in a row with different h and N_Ly check
that what the previous call left in the shared scratch does not leak into the
next result.
"""
import numpy as np
import pytest

from paper_2508_06302_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ATOL = 1e-6   # the exponent tolerance of the Lyapunov parity test (1/s)


def _converged_beam_torus(fse):
    m = I.eb_beam()
    w1 = 1.1 * m.omega_n1
    ctx = fse.Context(m, 2, [16], [7], [I.GOLDEN], 64, newton_tol=0, newton_maxit=6)
    Z = np.zeros(ctx.n_unknowns)
    for _ in range(8):
        Z, rn, rc = ctx.newton_step(Z, w1)
    return ctx, Z, w1


def test_noalloc_matches_lyapunov_two_calls():
    from paper_2508_06302_gb300 import fse
    ctx, Z, w1 = _converged_beam_torus(fse)
    ref1 = ctx.lyapunov(Z, w1, N_Ly=60, h=6)
    ref2 = ctx.lyapunov(Z, w1, N_Ly=40, h=3)
    na1 = ctx.lyapunov_noalloc(Z, w1, N_Ly=60, h=6)
    na2 = ctx.lyapunov_noalloc(Z, w1, N_Ly=40, h=3)
    assert np.all(np.isfinite(na1)) and np.all(np.isfinite(na2))
    np.testing.assert_allclose(na1, ref1, rtol=0, atol=ATOL)
    np.testing.assert_allclose(na2, ref2, rtol=0, atol=ATOL)
    # a second context of another size reuses the same scratch
    m = I.chain(6)
    ctx2 = fse.Context(m, 2, [7], [3], [I.GOLDEN], 24, newton_tol=0, newton_maxit=16)
    Z2 = I.random_coeffs(m.n, ctx2.U, 5e-3, seed=3)
    w2 = 1.15 * m.omega_n1
    ref3 = ctx2.lyapunov(Z2, w2, N_Ly=30, h=2 * m.n)
    na3 = ctx2.lyapunov_noalloc(Z2, w2, N_Ly=30, h=2 * m.n)
    np.testing.assert_allclose(na3, ref3, rtol=0, atol=ATOL)
    ctx2.close()
    ctx.close()


def test_noalloc_rejects_sizes_beyond_the_scratch():
    from paper_2508_06302_gb300 import fse
    m = I.chain(2100)                      # 2 n h = 268800 > FSE_NOALLOC_MAX_QH at h = 64
    ctx = fse.Context(m, 2, [3], [1], [I.GOLDEN], 8, newton_tol=0, newton_maxit=2)
    Z = np.zeros(ctx.n_unknowns)
    with pytest.raises(fse.FSEError) as ei:
        ctx.lyapunov_noalloc(Z, 1.1 * m.omega_n1, N_Ly=2, h=64)
    assert ei.value.code == fse.FSE_EINVAL
    assert "FSE_NOALLOC_MAX_QH" in str(ei.value)
    ctx.close()
