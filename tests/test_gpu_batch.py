"""fse_batch_*: several contexts of different trajectory counts evaluated together,
on their own streams or replayed as one captured CUDA graph, give exactly the
results of evaluating each context alone (the kernels are deterministic)."""
import numpy as np
import pytest

from paper_2508_06302_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _contexts(fse):
    m = I.eb_beam()
    out = []
    for S, H in ([8], [3]), ([12], [5]), ([16], [7]):
        out.append(fse.Context(m, 2, S, H, [I.GOLDEN], 64, newton_tol=0, newton_maxit=6))
    return m, out


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_equals_individual_evaluations(use_graph):
    from paper_2508_06302_gb300 import fse
    m, ctxs = _contexts(fse)
    omegas = m.omega_n1 * np.array([1.05, 1.1, 1.15])
    batch = fse.Batch(ctxs, use_graph=use_graph)
    for call, seed in enumerate((1, 2)):      # two calls in a row: the second replays the graph
        Zs = [I.random_coeffs(m.n, c.U, 1e-3, seed=seed + 10 * k) for k, c in enumerate(ctxs)]
        Rb, st, rc = batch.residual_jacobian(Zs, omegas, want_jacobian=True)
        assert rc == 0 and np.all(st == 0)
        mono_b = [c.monodromy() for c in ctxs]
        for k, c in enumerate(ctxs):
            R, st1, it, rc1 = c.residual_jacobian(Zs[k], omegas[k], want_jacobian=True)
            assert rc1 == 0
            assert np.array_equal(R, Rb[k]), (call, k, np.abs(R - Rb[k]).max())
            Phi, dz = c.monodromy()
            assert np.array_equal(Phi, mono_b[k][0]) and np.array_equal(dz, mono_b[k][1])
    # a change of w_1 re-captures the graph
    omegas2 = omegas * 1.01
    Rb, st, rc = batch.residual_jacobian(Zs, omegas2, want_jacobian=False)
    for k, c in enumerate(ctxs):
        R, st1, it, rc1 = c.residual_jacobian(Zs[k], omegas2[k], want_jacobian=False)
        assert np.array_equal(R, Rb[k])
    batch.close()
    for c in ctxs:
        c.close()
