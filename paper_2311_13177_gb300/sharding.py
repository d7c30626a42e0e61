"""Spectral-bin sharding of one reconstruction.

The forward operator is a sum over spectral bins, y = sum_f A_f V_f (every
bin's layer is displaced and transformed on its own, Sec. 3 Eq. 2, and the
layers are summed, Sec. 4.2), so rank g can hold the bins F_g, compute the
partial blade data sum_{f in F_g} A_f V_f with its own plan (built from
delta[F_g]) and take part in ONE all-reduce (sum) of y per iteration.
Everything after that -- residual, adjoint A_f^H r, x-y TV, temporal TV (all
frames of a bin are local) and Adam -- is bin-local.  The shards are
contiguous, near-equal runs of bins in a fixed order.

The per-rank compute is libprop's prop_shard_forward / prop_shard_update;
this module holds the host-side protocol: the bin partition, the order of
the calls and the all-reduce between them, and the assembly of the loss.
"""
from __future__ import annotations


def bin_shards(nf: int, world: int):
    """[(f_begin, f_end)] for ranks 0..world-1: contiguous, sizes differ by at most 1."""
    if nf < 1 or world < 1:
        raise ValueError("nf and world must be >= 1")
    base, extra = divmod(nf, world)
    out, f = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((f, f + n))
        f += n
    return out


def allreduce_sum_(t, group=None):
    """In-place sum of a tensor over the ranks of `group` (torch.distributed).

    Complex tensors are reduced through their real view, which every backend supports."""
    import torch
    import torch.distributed as dist
    view = torch.view_as_real(t) if t.is_complex() else t
    dist.all_reduce(view, op=dist.ReduceOp.SUM, group=group)
    return t


def host_allreduce_sum_(t, group=None):
    """allreduce_sum_ through host memory, for process groups whose backend
    (gloo) reduces CPU tensors only: copy to the host, reduce, copy back."""
    h = t.detach().cpu()
    allreduce_sum_(h, group)
    t.copy_(h)
    return t


class BinShardedReconstruction:
    """This rank's part of one reconstruction sharded by spectral bin.

    shard: the rank's plan over its bins (an object with shard_forward,
    shard_update and vol_shape, normally paper_2311_13177_gb300.Plan);
    y: the measured blade data (the same on every rank); params: Adam and TV
    settings; all_reduce: sums a tensor in place over the ranks, in the same
    order on every rank (allreduce_sum_ for NCCL, host_allreduce_sum_ for
    gloo).  Iteration k: y_part = A_g V_g; all_reduce(y_part) = A V;
    shard_update on the rank's bins.  The loss of iteration k is the data
    term (the same on every rank) plus the TV parts summed over ranks, reduced
    once at the end."""

    def __init__(self, shard, y, params, all_reduce):
        self.shard, self.y, self.params, self.all_reduce = shard, y, params, all_reduce

    def run(self, iters: int, V=None):
        """iters iterations from V (zeros if None); returns (V_iters, loss trace [iters] as a tensor)."""
        import torch
        dev = self.y.device
        cur = torch.zeros(self.shard.vol_shape, dtype=self.y.dtype, device=dev) if V is None else V.clone()
        nxt = torch.empty_like(cur)
        y_sum = torch.empty_like(self.y)
        parts = torch.zeros((max(iters, 1), 2), dtype=torch.float64, device=dev)
        for k in range(1, iters + 1):
            self.shard.shard_forward(cur, y_sum, reuse_rows=k > 1)
            self.all_reduce(y_sum)
            self.shard.shard_update(self.y, y_sum, self.params, k, cur, nxt, parts[k - 1])
            cur, nxt = nxt, cur
        tv = parts[:iters, 1].clone()
        self.all_reduce(tv)
        return cur, parts[:iters, 0] + tv


def reconstruct_local_shards(plans, y, params, iters: int):
    """A bin-sharded reconstruction over several plans on ONE device (no
    collective): the plans' partial forwards are summed in place by the
    library's accumulate mode, in plan order.  Returns ([V_g], loss trace)."""
    import torch
    dev = y.device
    cur = [torch.zeros(p.vol_shape, dtype=torch.complex64, device=dev) for p in plans]
    nxt = [torch.empty_like(c) for c in cur]
    y_sum = torch.empty_like(y)
    parts = torch.zeros((len(plans), max(iters, 1), 2), dtype=torch.float64, device=dev)
    for k in range(1, iters + 1):
        for g, p in enumerate(plans):
            p.shard_forward(cur[g], y_sum, reuse_rows=k > 1, accumulate=g > 0)
        for g, p in enumerate(plans):
            p.shard_update(y, y_sum, params, k, cur[g], nxt[g], parts[g, k - 1])
        cur, nxt = nxt, cur
    trace = parts[0, :iters, 0] + parts[:, :iters, 1].sum(dim=0)
    return cur, trace
