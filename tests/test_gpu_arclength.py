"""Pseudo-arclength continuation (App. C, Eq. C1-C3) through a fold: a 2-dof chain
with a hardening cubic spring (k3 = 1e9, F1 = 2 N, light damping), whose branch in
w_1 climbs to a turning point near 1.36 w_n1 and comes back; stepping w_1 cannot
pass it.  Every point must be a torus: converged on the GPU and confirmed by the
oracle's own residual."""
import numpy as np
import pytest

from oracle import fse_oracle as O
from paper_2508_06302_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_arclength_passes_the_fold():
    from paper_2508_06302_gb300 import fse
    m = I.chain(2, k=1e4, c=1.0, k3=1e9, F=(2.0, 0.0))
    wn = m.omega_n1
    ctx = fse.Context(m, 2, [5], [2], [I.GOLDEN], 64, newton_tol=1e-13, newton_maxit=30)
    Zn, pts, rc = fse.fse_continue(ctx, [0.9 * wn], np.zeros(ctx.n_unknowns), rel_tol=1e-11, max_newton=20)
    assert rc == 0
    nz = np.linalg.norm(Zn[0])
    Z, om, info, rc = fse.fse_continue_arclength(ctx, Zn[0], 0.9 * wn, 0.1 * nz, 120, direction=1,
                                                 rel_tol=1e-11, max_newton=12, omega_min=0.5 * wn,
                                                 omega_max=2.5 * wn, ds_max=3 * nz)
    f = om / wn
    k = int(np.argmax(f))
    print("arclength: %d points, w_1/w_n1 from %.3f to the turning point %.4f (point %d) and back to %.3f; "
          "Newton updates per point max %d" % (len(f), f[0], f[k], k, f[-1], max(p["newton_iters"] for p in info)))
    assert rc == 0 and len(f) == 120
    assert all(p["status"] == 0 and p["res"] <= 1e-11 * p["znorm"] for p in info)
    # w_1 rises to a turning point and then decreases: the path went round the fold
    assert 10 < k < len(f) - 10
    assert 1.30 < f[k] < 1.42 and f[-1] < f[k] - 0.05
    assert np.all(np.diff(f[:k]) > 0) and np.all(np.diff(f[k + 1:]) < 0)
    # independent check: the oracle's residual at points before, at and after the fold
    prob = O.FSEProblem(m, [5], [2], 64, [I.GOLDEN])
    for j in (k // 2, k, (k + len(f)) // 2, len(f) - 1):
        r = O.residual_jacobian(prob, Z[j], om[j], want_jacobian=False, tol=1e-13, maxit=30)
        assert np.linalg.norm(r.R) <= 1e-9 * np.linalg.norm(Z[j]), j
    ctx.close()
