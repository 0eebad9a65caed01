"""Sharding M2 of one state across ranks by shift range.

Shifts x are independent (the paper's parallel axis over the shift k), so a
state's work splits into contiguous shift ranges.  Each rank evaluates the
partial sum S_r = sum over its shifts of sum_z |A_x(z)|^4 (sre_sum4_range on
its GPU) and the partial sums are added with one all-reduce of a single FP64
value -- the only exchange step of the path; M2 = -log2(S / (d n2^4)).
"""
from __future__ import annotations

import math


def shard_range(d: int, rank: int, world: int) -> tuple[int, int]:
    """[begin, end) of the shifts of `rank` out of `world`: contiguous,
    sizes differing by at most one, covering [0, d) exactly."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    q, r = divmod(d, world)
    begin = rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


def m2_from_sum(S: float, n2: float, N: int) -> float:
    """M2 = -log2(S / (d n2^4)), written in logs."""
    return -(math.log2(S) - N - 4.0 * math.log2(n2))


def m2_sharded(psi, N: int, plan=None, group=None, partial_fn=None):
    """M2 of `psi` with this rank's share of the shifts.

    partial_fn(begin, end) -> (S_partial, n2) computes the rank's partial sum;
    by default the GPU plan's sre_sum4_range.  The partial sums are combined
    with torch.distributed.all_reduce (SUM) on `group`."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    b, e = shard_range(1 << N, rank, world)
    if partial_fn is None:
        out = plan.sum4_range(psi, b, e)
        S_part, n2 = out[0].item(), out[1].item()
        dev = psi.device
    else:
        S_part, n2 = partial_fn(b, e)
        dev = torch.device("cpu")
    t = torch.tensor([S_part], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return m2_from_sum(t.item(), n2, N)
