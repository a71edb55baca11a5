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

`sharded_sthosvd` is the whole method over P ranks (Algorithm 1 in the
natural mode order): for every mode n < N-1 the local Gram of the rank's
shard, the fixed-order sum of the partials, the eigensolve and the cut on
every rank (redundantly, on identical Grams: identical ranks and factors),
then the local TTM, which needs no exchange; before the last mode, whose
index is the one the shards split, an all-gather of the shrunken partial
core (R_0 x ... x R_{N-2} x J_{N-1}), after which every rank finishes the
last mode on the whole small tensor.  The per-rank arithmetic is passed in
as `ops` (LibraryOps: the CUDA library through its C ABI, one GPU per
rank), so the exchange pattern is the same whatever computes the steps.
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


def allgather_last_mode(y, dims, world, rank, group=None):
    """The whole tensor from every rank's shard of its last mode: the
    shards are contiguous flat ranges in rank order (natural-descending
    layout), so the result is their concatenation.  Shards of unequal size
    are padded to the largest for the collective and trimmed after."""
    import torch
    import torch.distributed as dist
    inner = int(np.prod(dims[:-1])) if len(dims) > 1 else 1
    sizes = [inner * (shard_bounds(dims, world, r)[1] - shard_bounds(dims, world, r)[0])
             for r in range(world)]
    if y.numel() != sizes[rank]:
        raise ValueError("local shard size does not match its bounds")
    m = max(sizes)
    buf = torch.zeros(m, dtype=y.dtype, device=y.device)
    buf[:sizes[rank]] = y.reshape(-1)
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return torch.cat([p[:n] for p, n in zip(parts, sizes)])


class LibraryOps:
    """The per-rank steps of sharded_sthosvd on this rank's GPU, through the
    library's C ABI (tucker.Context); tensors live on the device."""

    def __init__(self, ctx, prec="fp64"):
        self.ctx, self.prec = ctx, prec

    def norm_sq(self, y):
        return self.ctx.norm_sq(y)

    def gram(self, y, dims, n):
        return self.ctx.gram(y, dims, n, self.prec)

    def eig_trunc(self, S, thr, R):
        w, U, k, d = self.ctx.eig_trunc(S, thr, R)
        return w, U.contiguous(), k, d

    def ttm(self, y, dims, n, U):
        # Y x_n U^T: A = U^T (R x I)
        return self.ctx.ttm(y, dims, n, U.t(), self.prec)

    def to_comm(self, t):
        """Tensors cross the collectives on the device for NCCL, on the host
        for gloo."""
        import torch.distributed as dist
        return t.cuda() if dist.get_backend() == "nccl" else t.cpu()

    def from_comm(self, t):
        return t.cuda()


def sharded_sthosvd(x_local, dims, world, rank, ops, eps=None, ranks=None, group=None):
    """ST-HOSVD (Algorithm 1, modes 0..N-1) of the tensor of `dims` whose
    last-mode shard [shard_bounds(dims, world, rank)) this rank holds as the
    flat natural-descending `x_local`.  Exactly one of eps / ranks.  Returns
    a dict (identical on every rank): core (flat), core_dims, factors (U_n,
    I_n x R_n), eigvals, ranks, discarded, norm_sq, threshold."""
    dims = tuple(int(d) for d in dims)
    N = len(dims)
    if (eps is None) == (ranks is None):
        raise ValueError("give exactly one of eps or ranks")
    if N < 2:
        raise ValueError("a sharded ST-HOSVD needs at least two modes")
    import torch
    local = ops.to_comm(torch.tensor([float(ops.norm_sq(x_local))], dtype=torch.float64))
    nrm2 = float(allreduce_fixed_order(local, group=group)[0])
    thr = float(eps) ** 2 * nrm2 / N if eps is not None else 0.0
    cur = list(shard_dims(dims, world, rank))
    y = x_local
    factors, eigvals, out_ranks, disc = [None] * N, [None] * N, [0] * N, [0.0] * N

    def truncate(S, n):
        R_fix = 0 if ranks is None else int(ranks[n])
        w, U, R, d = ops.eig_trunc(S, thr, R_fix)
        factors[n], eigvals[n], out_ranks[n], disc[n] = U, w, int(R), float(d)
        return U

    for n in range(N - 1):
        S_local = ops.gram(y, cur, n)
        S = ops.from_comm(allreduce_fixed_order(ops.to_comm(S_local), group=group))
        U = truncate(S, n)
        y = ops.ttm(y, cur, n, U)
        cur[n] = out_ranks[n]
    # last mode: gather the small partial core, finish it everywhere
    full = list(cur[:-1]) + [dims[-1]]
    y = ops.from_comm(allgather_last_mode(ops.to_comm(y), full, world, rank, group=group))
    S = ops.gram(y, full, N - 1)
    U = truncate(S, N - 1)
    y = ops.ttm(y, full, N - 1, U)
    full[-1] = out_ranks[N - 1]
    return {"core": y, "core_dims": tuple(full), "factors": factors, "eigvals": eigvals,
            "ranks": tuple(out_ranks), "discarded": disc, "norm_sq": nrm2, "threshold": thr}
