"""Trajectory sharding of one torus over two CPU ranks (gloo, world size 2).

Each rank integrates its contiguous share of the N samples (the oracle stands in for the rank's
GPU shard here) and forms its partial DFT sums of Eq. 21 and Eq. 22; the package's
``ordered_allsum`` completes them.  Required: both ranks hold bit-identical R and J v, equal bit
for bit to the two shards' partial sums added in rank order in one process, and equal to the
unsharded oracle evaluation within rounding (1e-13)."""
import os
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _problem():
    from oracle import fse_oracle as O
    from paper_2508_06302_gb300 import inputs as I
    m = I.chain(4)
    prob = O.FSEProblem(m, [7], [3], 24, [I.GOLDEN])
    Z = I.random_coeffs(m.n, prob.U, 1e-2, seed=5)
    V = I.random_coeffs(m.n, prob.U, 1.0, seed=6)
    return prob, 1.15 * m.omega_n1, Z, V


def _partials(prob, w1, Z, V, s0, s1):
    """This shard's partial sums of (I (x) R Gamma^-1) zbar(2 pi) and of (I (x) R Gamma^-1)
    blockdiag(Phi_s) (I (x) Gamma) v over samples s0 .. s1 - 1 (state-major 2n x U~)."""
    from oracle import fse_oracle as O
    n2, U = 2 * prob.n, prob.U
    RG = prob.R @ prob.Gi                     # U x N
    zb0 = O.idft(prob, Z)
    zv = (V.reshape(n2, U) @ prob.G.T).T      # samples of v, N x 2n
    P = np.zeros((n2, U))
    Q = np.zeros((n2, U))
    for s in range(s0, s1):
        tr = O.integrate_trajectory(prob.model, w1, prob.rho, prob.T[:, s], zb0[s, :prob.n], zb0[s, prob.n:],
                                    prob.S1, tol=0, maxit=6, sens=True)
        P += np.outer(tr.zT, RG[:, s])
        Q += np.outer(tr.Phi @ zv[s], RG[:, s])
    return P.reshape(-1), Q.reshape(-1)


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2508_06302_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob, w1, Z, V = _problem()
    s0, s1 = shard.shard_range(prob.N, rank, world)
    P, Q = _partials(prob, w1, Z, V, s0, s1)
    tP, tQ = torch.from_numpy(P.copy()), torch.from_numpy(Q.copy())
    shard.ordered_allsum(tP)
    shard.ordered_allsum(tQ)
    out[rank] = (tP.numpy() - Z, tQ.numpy() - V, P, Q)
    dist.barrier()
    dist.destroy_process_group()


def test_shard_ranges_partition_the_grid():
    sys.path.insert(0, ROOT)
    from paper_2508_06302_gb300.shard import shard_range
    for N in (1, 2, 7, 16, 63, 64, 256):
        for W in range(1, min(N, 9) + 1):
            rs = [shard_range(N, r, W) for r in range(W)]
            assert rs[0][0] == 0 and rs[-1][1] == N
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            sizes = [b - a for a, b in rs]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        shard_range(3, 0, 4)


@pytest.mark.timeout(180)
def test_two_gloo_shards_reproduce_the_torus_residual_and_jv():
    sys.path.insert(0, ROOT)
    from oracle import fse_oracle as O
    world, port = 2, 29741
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(150)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    (R0, J0, P0, Q0), (R1, J1, P1, Q1) = res[0], res[1]
    assert np.array_equal(R0, R1) and np.array_equal(J0, J1)         # every rank holds the same result
    prob, w1, Z, V = _problem()
    assert np.array_equal(R0, (P0 + P1) - Z) and np.array_equal(J0, (Q0 + Q1) - V)
    ref = O.residual_jacobian(prob, Z, w1, want_jacobian=True, dense=True, tol=0, maxit=6)
    np.testing.assert_allclose(R0, ref.R, rtol=0, atol=1e-13 * np.abs(Z).max())
    np.testing.assert_allclose(J0, ref.J @ V, rtol=0, atol=1e-13 * np.abs(ref.J @ V).max())
