"""Point sharding across ranks (one process per GPU).

Every point is independent (the evaluation is pointwise), so thermo, rates, transport and
the JVP shard with no exchange at all.  The one quantity that crosses shards is the VJP's
ln A gradient, a sum over all points of an R-vector; it is reduced here in rank order so
the result does not depend on the communicator's reduction tree.
"""
from __future__ import annotations

GLL_POINTS_PER_ELEMENT = 512   # (p + 1)^3 at polynomial order 7


def shard_range(n_points: int, world: int, rank: int, unit: int = GLL_POINTS_PER_ELEMENT):
    """[start, stop) of this rank's points: contiguous, whole units (elements), balanced to
    within one unit; a trailing partial unit goes to the last rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    n_units = n_points // unit
    base, extra = divmod(n_units, world)
    start_u = rank * base + min(rank, extra)
    stop_u = start_u + base + (1 if rank < extra else 0)
    start = start_u * unit
    stop = stop_u * unit if rank < world - 1 else n_points
    return start, stop


def reduce_in_rank_order(vec, group=None):
    """Sum a tensor over the ranks of `group` in rank order (deterministic): gather every
    rank's contribution, then add them 0, 1, 2, ... on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [torch.empty_like(vec) for _ in range(world)]
    dist.all_gather(parts, vec.contiguous(), group=group)
    out = parts[0].clone()
    for t in parts[1:]:
        out += t
    return out


def rates_vjp_lnA_sharded(mech, T, p, Y, bar_omega, bar_hrr=None, dlnA=None, group=None):
    """This rank's VJP on its own points and the ln A gradient summed over all ranks.
    T, p, Y, bar_omega, bar_hrr are the local shard (CUDA tensors)."""
    from . import rates_vjp
    gT, gY, g = rates_vjp(mech, T, p, Y, bar_omega, bar_hrr, dlnA, want_lnA=True)
    return gT, gY, reduce_in_rank_order(g, group)
