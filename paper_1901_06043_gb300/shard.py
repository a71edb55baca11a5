"""Host-side pieces of a sharded ST-HOSVD: one tensor spread over P ranks.

The tensor is split along its last mode into P contiguous ranges.  In the
natural-descending layout (Eq. idxtolin) a range of the last index is a
contiguous range of the flat array, and for every mode n < N-1 it is a
contiguous range of the slabs r of the mode-n view (Rt, I, L).  The Gram of
Algorithm 2 is a sum over slabs, so each rank's Gram of its own shard is a
partial sum and the full Gram is the sum of the P partials; Section 5.1's
distributed Gram reduces the same partial sums across processors.  The
TTM of Algorithm 3 acts slab by slab and needs no exchange (Section 5.3).

`allreduce_fixed_order` sums the partials in rank order on every rank, so
all ranks hold bitwise-identical Grams and take identical rank decisions
(an all-reduce may combine in any order).  It works with any
torch.distributed backend (gloo on the host, NCCL on GPUs).
"""

import numpy as np


def shard_bounds(dims, world, rank):
    """[lo, hi) of the last mode owned by `rank` (balanced, contiguous)."""
    J = int(dims[-1])
    if not (0 <= rank < world) or world < 1:
        raise ValueError("rank out of range")
    return J * rank // world, J * (rank + 1) // world


def shard_dims(dims, world, rank):
    lo, hi = shard_bounds(dims, world, rank)
    return tuple(int(d) for d in dims[:-1]) + (hi - lo,)


def shard_slice(dims, world, rank):
    """Flat element range [start, stop) of the shard in the natural-descending
    array of the whole tensor."""
    lo, hi = shard_bounds(dims, world, rank)
    inner = int(np.prod(dims[:-1])) if len(dims) > 1 else 1
    return lo * inner, hi * inner


def allreduce_fixed_order(S, group=None):
    """Sum of every rank's S (a torch tensor, same shape on every rank), in
    rank order, returned on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [torch.empty_like(S) for _ in range(world)]
    dist.all_gather(parts, S.contiguous(), group=group)
    out = parts[0].clone()
    for p in parts[1:]:
        out += p
    return out
