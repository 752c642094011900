"""Term-sharded collide over several ranks, one GPU each: the multi-GPU form of eq. realQ.

The sum over p in eq. realQ (Sec. 4) is a sum of independent terms.  Rank r evaluates the
contiguous term range [p0, p1) that bz_partition_terms gives it, with bz_collide_terms, into its
own N^3 result; one all-reduce (sum) then adds the ranks' results, so that every rank holds
Qhat.  That all-reduce of N^3 complex values per collide (4 MB at N = 64 in complex128) is the
path's only exchange step; each rank reads only its slice of the alpha (or pair) table.
Batched and served work needs no exchange: it runs as independent replicas.
"""
from __future__ import annotations

from . import BZ_DATA_COMPLEX, bz_collide_terms, bz_partition_terms


def sharded_sum(P: int, data: int, world: int, rank: int, partial, all_reduce):
    """Rank `rank` of `world`: out = partial(p0, p1) over its term range, then all_reduce(out)
    (an in-place sum over the ranks).  Returns out."""
    p0, p1 = bz_partition_terms(P, data, world, rank)
    out = partial(p0, p1)
    all_reduce(out)
    return out


def collide_sharded(plan, fhat, Qhat, group=None, stream=None):
    """Qhat = Q(fhat, fhat) with the terms sharded over the ranks of `group` (torch.distributed,
    NCCL for device tensors): each rank runs its range through bz_collide_terms on `stream`, the
    all-reduce runs on torch's current stream after it.  fhat and Qhat are this rank's device
    tensors; Qhat (complex128 keeps the FP64 sum over terms) holds the full result on every rank."""
    import torch
    import torch.distributed as dist

    world, rank = dist.get_world_size(group), dist.get_rank(group)

    def partial(p0, p1):
        bz_collide_terms(plan, p0, p1, fhat, Qhat, stream)
        if stream is not None:
            torch.cuda.current_stream().wait_stream(stream)
        return Qhat

    def reduce(t):
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)

    return sharded_sum(plan.P, getattr(plan, "data", BZ_DATA_COMPLEX), world, rank, partial, reduce)
