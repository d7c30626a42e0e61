"""Spectral-bin sharding of one reconstruction across ranks (design of the
multi-GPU path).

The forward operator is a sum over spectral bins, y = sum_f A_f V_f, so rank
g can hold the bins F_g, compute the partial blade data sum_{f in F_g} A_f V_f
with its own plan (built from delta[F_g]) and take part in ONE all-reduce
(sum) of y per iteration.  Everything after that -- residual, adjoint
A_f^H r, x-y TV, temporal TV (all frames of a bin are local) and Adam -- is
bin-local.  The shards are contiguous, near-equal runs of bins in a fixed
order, so the reduction order is fixed.
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
