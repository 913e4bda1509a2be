"""The Python binding rejects wrongly sized arrays with ValueError before any call into the C
library (which reads and writes whole vectors of the sizes the context fixes).  No GPU: the
objects are built without a device context and never reach the library."""
import numpy as np
import pytest

from paper_2508_06302_gb300 import fse


def _fake_context(n_unknowns=30, n=3, U=5, N=5):
    c = object.__new__(fse.Context)
    c.h = None                      # close() / __del__ do nothing
    c.n_unknowns, c.U, c.N, c.n, c.band, c.d = n_unknowns, U, N, n, 1, 2
    return c


def test_context_methods_check_sizes():
    c = _fake_context()
    bad = np.zeros(c.n_unknowns - 1)
    with pytest.raises(ValueError):
        c.residual_jacobian(bad, 1.0)
    with pytest.raises(ValueError):
        c.newton_step(bad, 1.0)
    with pytest.raises(ValueError):
        c.lyapunov(bad, 1.0, 10, 2)
    with pytest.raises(ValueError):
        c.lyapunov_noalloc(bad, 1.0, 10, 2)
    with pytest.raises(ValueError):
        c.lyapunov(np.zeros(c.n_unknowns), 1.0, 10, 0)
    with pytest.raises(ValueError):
        c.jacobian_apply(np.zeros((2, c.n_unknowns + 1)))


def test_continuation_entry_points_check_sizes():
    fse.load()                       # the library loads without a GPU; nothing is called
    c = _fake_context()
    with pytest.raises(ValueError):
        fse.fse_continue(c, [1.0, 1.1], np.zeros(c.n_unknowns + 2))
    with pytest.raises(ValueError):
        fse.fse_continue(c, [], np.zeros(c.n_unknowns))
    with pytest.raises(ValueError):
        fse.fse_continue_arclength(c, np.zeros(3), 1.0, 0.1, 5)
    with pytest.raises(ValueError):
        fse.fse_continue_arclength(c, np.zeros(c.n_unknowns), 1.0, 0.1, 0)


def test_batch_and_mlp_check_sizes():
    b = object.__new__(fse.Batch)
    b.h = None
    b.ctx = [_fake_context(30), _fake_context(40)]
    with pytest.raises(ValueError):
        b.residual_jacobian([np.zeros(30)], [1.0, 1.0])                  # one vector for two points
    with pytest.raises(ValueError):
        b.residual_jacobian([np.zeros(30), np.zeros(30)], [1.0, 1.0])    # second point has 40
    with pytest.raises(ValueError):
        b.residual_jacobian([np.zeros(30), np.zeros(40)], [1.0])          # one frequency
    m = object.__new__(fse.Mlp)
    m.h = None
    m.dims, m.np = (3, 256, 64), 3 * 256 + 256 + 256 * 256 + 256 + 256 * 64 + 64
    with pytest.raises(ValueError):
        m.forward(np.zeros((4, 2)))
    with pytest.raises(ValueError):
        m.grad(np.zeros((4, 3)), np.zeros((4, 63)))
    with pytest.raises(ValueError):
        m.train(np.zeros((4, 3)), np.zeros((5, 64)), 1, 1e-3)
    with pytest.raises(ValueError):
        m.set_params({k: np.zeros(1) for k in fse.Mlp.ORDER})
