"""Tensor-core banded tangent solves (FSE_SOLVE_TC, tcgen05 kind::tf32 with split operands)
against the FP64 oracle and against the FP32 SIMT solves, through the C ABI.

App. E propagates the 2n+1 sensitivity columns of every trajectory through the factor of the
effective stiffness; these cases cover half-bandwidths 0 (one dof), 1-32, 38 and 74 (one,
two and three coupled 32-row blocks), one and several trajectories, d = 2 and d = 3,
and a partial last block.  Tolerances: residual 1e-10 relative (FP64 state path in every
mode), monodromy 1e-3 relative against the oracle over the period (as for the SIMT FP32
solves), and the tensor-core monodromy within 1e-4 relative of the SIMT one.
"""
import numpy as np
import pytest

from oracle import fse_oracle as O
from paper_2508_06302_gb300 import inputs as I

pytestmark = pytest.mark.gpu

import math

CASES = {
    "chain1_n1": (lambda: I.chain(1), 2, [5], [2], 24, [I.GOLDEN], 1.1, 1e-3),
    "chain6_d2": (lambda: I.chain(6), 2, [7], [3], 24, [I.GOLDEN], 1.15, 1e-3),
    "beam18_d2": (lambda: I.eb_beam(), 2, [16], [7], 64, [I.GOLDEN], 1.1, 1e-3),
    "vk87_d2": (lambda: I.vk_beam(n_el=30, F1=1.0, F2=1.0), 2, [5], [2], 48, [I.GOLDEN], 1.1, 1e-6),
    "shell90_d2": (lambda: I.flat_shell(nx=6, ny=4), 2, [5], [2], 20, [I.GOLDEN], 1.0, 1e-4),
    "shell150_d2": (lambda: I.flat_shell(nx=6, ny=6), 2, [3], [1], 16, [I.GOLDEN], 1.0, 1e-4),
    "shell198_d2": (lambda: I.flat_shell(nx=4, ny=12), 2, [3], [1], 16, [I.GOLDEN], 1.0, 1e-4),
    "shell252_b92_d2": (lambda: I.flat_shell(nx=4, ny=15), 2, [3], [1], 16, [I.GOLDEN], 1.0, 1e-4),
    "chain4_N1_H0": (lambda: I.chain(4, F=(2.0, 0.0), c=3.0), 2, [1], [0], 24, [I.GOLDEN], 1.2, 1e-3),
    "plate27_d3": (lambda: I.kirchhoff_plate(nx=4, ny=4, n_springs=3), 3, [3, 3], [1, 1], 16,
                   [math.sqrt(2), math.sqrt(3)], 1.1, 1e-4),
}


def _fse():
    from paper_2508_06302_gb300 import fse
    fse.load()
    return fse


@pytest.mark.parametrize("name", list(CASES))
def test_tc_solves_match_oracle_and_simt(name):
    mk, d, S, H, S1, rho, wf, sc = CASES[name]
    m = mk()
    w1 = wf * m.omega_n1
    prob = O.FSEProblem(m, S, H, S1, rho)
    U = O.u_tilde(H)
    Z = I.random_coeffs(m.n, U, sc, seed=7)
    ref = O.residual_jacobian(prob, Z, w1, want_jacobian=True, dense=False, tol=0, maxit=16)
    fse = _fse()
    ctx = fse.Context(m, d, S, H, rho, S1, newton_tol=0.0, newton_maxit=16, precision="mixed_fp32")
    out = {}
    for kind in ("tc", "simt"):
        ctx.set_tangent_solve(kind)
        R, st, it, rc = ctx.residual_jacobian(Z, w1, want_jacobian=True)
        assert rc == 0
        Phi, dz = ctx.monodromy()
        out[kind] = (R, Phi, dz)
    R, Phi, dz = out["tc"]
    assert np.array_equal(R, out["simt"][0])      # the FP64 state path does not see the solve kernel
    nR = np.linalg.norm(Z) + np.linalg.norm(ref.R)
    e_R = np.linalg.norm(R - ref.R) / nR
    e_P = np.linalg.norm(Phi - ref.Phi) / np.linalg.norm(ref.Phi)
    e_d = np.linalg.norm(dz - ref.dz_dw) / max(np.linalg.norm(ref.dz_dw), 1e-300)
    e_TS = np.linalg.norm(Phi - out["simt"][1]) / np.linalg.norm(out["simt"][1])
    e_S = np.linalg.norm(out["simt"][1] - ref.Phi) / np.linalg.norm(ref.Phi)
    print("%s (b=%d): TC vs oracle R %.1e Phi %.1e dz/dw %.1e; SIMT vs oracle Phi %.1e; TC vs SIMT %.1e"
          % (name, ctx.band, e_R, e_P, e_d, e_S, e_TS))
    assert e_R <= 1e-10
    assert e_P <= 1e-3
    assert e_d <= 1e-2
    assert e_TS <= 1e-4
    ctx.close()


def test_tc_solve_rejected_where_it_does_not_apply():
    fse = _fse()
    m = I.chain(4)
    ctx = fse.Context(m, 2, [7], [3], [0.5], 16, precision="fp64")
    with pytest.raises(fse.FSEError) as ei:
        ctx.set_tangent_solve("tc")
    assert ei.value.code == fse.FSE_EINVAL
    ctx.set_tangent_solve("simt")
    ctx.close()
    wide = I.flat_shell(nx=3, ny=18)          # half-bandwidth 110 > 96
    ctx = fse.Context(wide, 2, [5], [2], [I.GOLDEN], 20, precision="mixed_fp32")
    assert ctx.band > 96
    with pytest.raises(fse.FSEError) as ei:
        ctx.set_tangent_solve("tc")
    assert ei.value.code == fse.FSE_EINVAL
    ctx.close()
