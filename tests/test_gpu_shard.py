"""Trajectory shards on the GPU (fse_setup_shard, fse_set_reduce) through the C ABI.

(1) One process, two shard contexts without a reduction: their partial sums of Eq. 21 / 22 / 23
add up to the unsharded context's residual, J v and dR/dw_1 (1e-13).  (2) Two processes (gloo,
world size 2) sharing this GPU, each with its shard context and the package's reduction: the
residual, J v and a GMRES Newton solve equal the unsharded context's (1e-12) and are
bit-identical on both ranks.  The ranks only exchange host copies between launches; no kernel
waits on another process."""
import os
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2508_06302_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CASE = dict(d=2, S=[16], H=[7], rho=[I.GOLDEN], S1=64)


def _model():
    return I.eb_beam()


@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32"])
def test_shard_partial_sums_add_up(precision):
    from paper_2508_06302_gb300 import fse
    from paper_2508_06302_gb300.shard import shard_range
    m = _model()
    w1 = 1.1 * m.omega_n1
    kw = dict(newton_tol=0, newton_maxit=6, precision=precision)
    full = fse.Context(m, CASE["d"], CASE["S"], CASE["H"], CASE["rho"], CASE["S1"], **kw)
    Z = I.random_coeffs(m.n, full.U, 1e-3, seed=3)
    V = I.random_coeffs(m.n, full.U, 1.0, seed=4)
    R, _, _, rc = full.residual_jacobian(Z, w1, True)
    JV = full.jacobian_apply(V)
    dW = full.jacobian_domega()
    parts = []
    for r in range(3):
        sh = fse.Context(m, CASE["d"], CASE["S"], CASE["H"], CASE["rho"], CASE["S1"],
                         shard=shard_range(16, r, 3), **kw)
        assert sh.N == shard_range(16, r, 3)[1] - shard_range(16, r, 3)[0]
        Pr, _, _, rc = sh.residual_jacobian(Z, w1, True)
        parts.append((Pr, sh.jacobian_apply(V), sh.jacobian_domega()))
        with pytest.raises(fse.FSEError):
            sh.lyapunov(Z, w1, 10, 2)
        sh.close()
    Rs = sum(p[0] for p in parts) - Z
    Js = sum(p[1] for p in parts) - V
    Ws = sum(p[2] for p in parts)
    for a, b in ((Rs, R), (Js, JV), (Ws, dW)):
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()
    full.close()


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2508_06302_gb300 import fse, shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    m = _model()
    w1 = 1.1 * m.omega_n1
    ctx = shard.shard_context(m, CASE["d"], CASE["S"], CASE["H"], CASE["rho"], CASE["S1"], newton_tol=0,
                              newton_maxit=6, precision="fp64")
    ctx.set_linear_solver("gmres", rel_tol=1e-12, restart=60, max_iters=600)
    Z = I.random_coeffs(m.n, ctx.U, 1e-3, seed=3)
    V = I.random_coeffs(m.n, ctx.U, 1.0, seed=4)
    R, _, _, _ = ctx.residual_jacobian(Z, w1, True)
    JV = ctx.jacobian_apply(V)
    Zn = np.zeros(ctx.n_unknowns)
    for _ in range(6):
        Zn, rn, rc = ctx.newton_step(Zn, w1)
    out[rank] = (R, JV, Zn)
    ctx.close()
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_process_shards_on_one_gpu_match_the_unsharded_context():
    from paper_2508_06302_gb300 import fse
    world, port = 2, 29751
    spawn = mp.get_context("spawn")
    with spawn.Manager() as mgr:
        out = mgr.dict()
        procs = [spawn.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(280)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    (R0, J0, Z0), (R1, J1, Z1) = res[0], res[1]
    assert np.array_equal(R0, R1) and np.array_equal(J0, J1) and np.array_equal(Z0, Z1)
    m = _model()
    w1 = 1.1 * m.omega_n1
    full = fse.Context(m, CASE["d"], CASE["S"], CASE["H"], CASE["rho"], CASE["S1"], newton_tol=0, newton_maxit=6)
    full.set_linear_solver("gmres", rel_tol=1e-12, restart=60, max_iters=600)   # the shards' outer solver
    Z = I.random_coeffs(m.n, full.U, 1e-3, seed=3)
    V = I.random_coeffs(m.n, full.U, 1.0, seed=4)
    R, _, _, _ = full.residual_jacobian(Z, w1, True)
    JV = full.jacobian_apply(V)
    Zn = np.zeros(full.n_unknowns)
    for _ in range(6):
        Zn, rn, rc = full.newton_step(Zn, w1)
    assert np.abs(R0 - R).max() <= 1e-13 * np.abs(R).max()
    assert np.abs(J0 - JV).max() <= 1e-13 * np.abs(JV).max()
    assert np.linalg.norm(Z0 - Zn) <= 1e-11 * np.linalg.norm(Zn)
    full.close()
