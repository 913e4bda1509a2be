"""Trajectory sharding of one torus over several processes (one GPU each).

Within one evaluation of Eq. (16) the N trajectories are independent (App. E); only the DFT
sums over the samples (Eq. 21 for Z(2 pi), Eq. 22 for J v, Eq. 23 for dR/dw_1) couple them.
Rank r of a world of W integrates the contiguous samples ``shard_range(N, r, W)`` in a shard
context (``fse_setup_shard``) that keeps its own monodromies; each DFT sum is formed per rank
over its samples and completed by ``ordered_allsum``: an all-gather of the per-rank partial
sums (2 n U~ doubles) followed by their sum in rank order, so every rank holds bit-identical
coefficients whatever the collective's internal order.  Every vector of the outer Newton and
GMRES iterations is replicated (2 n U~ doubles per rank); only the trajectory work is split.
"""
from __future__ import annotations


def shard_range(N: int, rank: int, world: int):
    """Contiguous sample range [s_begin, s_end) of rank ``rank``: the first N mod W ranks take one
    extra sample."""
    if not (0 <= rank < world) or N < world:
        raise ValueError("need 0 <= rank < world <= N")
    base, extra = divmod(N, world)
    s0 = rank * base + min(rank, extra)
    return s0, s0 + base + (1 if rank < extra else 0)


def ordered_allsum(t, group=None):
    """In place: t <- sum over ranks of t, summed in rank order on every rank (deterministic and
    identical on all ranks).  t is a 1-D torch tensor (CPU with gloo, CUDA with NCCL)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    if world == 1:
        return t
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t.contiguous(), group=group)
    acc = parts[0].clone()
    for p in parts[1:]:
        acc += p
    t.copy_(acc)
    return t


class _DevView:
    """A float64 CUDA buffer given by address and length, for torch.as_tensor (zero copy)."""

    def __init__(self, ptr: int, count: int):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": "<f8", "data": (ptr, False),
                                         "version": 2, "strides": None}


def shard_context(model, d, S, H, rho, S1, rank=None, world=None, group=None, **kw):
    """A shard context of this rank (fse.Context with shard=...) whose partial DFT sums are completed
    by ``ordered_allsum`` over ``group``: on the ranks' GPUs with NCCL, through host copies with
    gloo."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from . import fse
    rank = dist.get_rank(group) if rank is None else rank
    world = dist.get_world_size(group) if world is None else world
    N = int(np.prod(S)) if len(S) else 1
    ctx = fse.Context(model, d, S, H, rho, S1, shard=shard_range(N, rank, world), **kw)

    host = dist.get_backend(group) == "gloo"     # gloo ranks exchange host copies

    def reduce(ptr, count, stream):
        t = torch.as_tensor(_DevView(ptr, count), device="cuda")
        if host:
            h = t.cpu()
            ordered_allsum(h, group)
            t.copy_(h)
        else:
            ordered_allsum(t, group)
        torch.cuda.synchronize()

    ctx.set_reduce(reduce)
    return ctx
