"""Sharding M2 of one state across ranks by shift range.

Shifts x are independent (the paper's parallel axis over the shift k), so a
state's work splits into contiguous shift ranges.  Each rank evaluates the
partial sum S_r = sum over its shifts of sum_z |A_x(z)|^4 (sre_sum4_range on
its GPU) and the partial sums are added with one all-reduce of a single FP64
value -- the only exchange step of the path.  The last step of Algorithm 1,
Eq. (final1) M2 = -log2(S / (d n2^4)), runs on the device through
sre_m_alpha_from_sums.
"""
from __future__ import annotations


def shard_range(d: int, rank: int, world: int) -> tuple[int, int]:
    """[begin, end) of the shifts of `rank` out of `world`: contiguous,
    sizes differing by at most one, covering [0, d) exactly."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    q, r = divmod(d, world)
    begin = rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


def _rank_world(group):
    import torch.distributed as dist
    if not dist.is_initialized():
        return 0, 1
    return dist.get_rank(group), dist.get_world_size(group)


def _all_reduce_sum(t, group, world):
    import torch.distributed as dist
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def sum_sharded(N: int, partial_fn, group=None) -> tuple[float, float]:
    """(S, n2) of a state from this rank's share of the shifts.

    partial_fn(begin, end) -> (S_partial, n2) computes the rank's partial
    sum on the host; the partials are added with one all-reduce (SUM) on
    `group`.  The sharding and the exchange are the same as m2_sharded's."""
    import torch
    rank, world = _rank_world(group)
    b, e = shard_range(1 << N, rank, world)
    S_part, n2 = partial_fn(b, e)
    t = _all_reduce_sum(torch.tensor([S_part], dtype=torch.float64), group, world)
    return t.item(), n2


def m2_sharded(psi, N: int, plan, group=None) -> float:
    """M2 of `psi` (a CUDA tensor) with this rank's share of the shifts.

    The rank's partial sum comes from plan.sum4_range, the partials are
    added on the device with one all-reduce (SUM) on `group`, and M2 follows
    from sre_m_alpha_from_sums on the device; everything runs in order on
    torch's current stream, the one the all-reduce uses."""
    from . import binding
    rank, world = _rank_world(group)
    b, e = shard_range(1 << N, rank, world)
    out = plan.sum4_range(psi, b, e)  # [S_partial, n2] on the device
    S = _all_reduce_sum(out[0:1].clone(), group, world)
    return binding.m_alpha_from_sums(S, out[1:2], N, 2).item()
