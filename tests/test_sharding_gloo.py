"""Bin-sharded forward/adjoint over two CPU ranks (gloo) equals the unsharded operator.

Each rank evaluates the oracle on its contiguous run of spectral bins (the
per-rank compute the GPU path would do with its own plan); the partial blade
data are summed with one all-reduce, and the bin-local adjoints concatenate.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2311_13177_gb300.sharding import bin_shards


def test_bin_shards_partition():
    for nf in (1, 3, 8, 33):
        for world in (1, 2, 3, 8):
            sh = bin_shards(nf, world)
            assert sh[0][0] == 0 and sh[-1][1] == nf
            assert all(a[1] == b[0] for a, b in zip(sh, sh[1:]))
            sizes = [b - a for a, b in sh]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle
    from paper_2311_13177_gb300.sharding import bin_shards, allreduce_sum_
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(0)
    N, L, R, Nf, T = 16, 4, 16, 5, 2
    theta = rng.uniform(0, np.pi, 3)
    delta = np.linspace(-2, 2, Nf)
    frames = [0, 1, 1]
    V = rng.standard_normal((T, N, N, Nf)) + 1j * rng.standard_normal((T, N, N, Nf))
    y = rng.standard_normal((3, L, R)) + 1j * rng.standard_normal((3, L, R))
    f0, f1 = bin_shards(Nf, world)[rank]
    g = oracle.make_geometry(N, L, R, theta, delta[f0:f1], frames, T)
    part = torch.from_numpy(oracle.forward(V[..., f0:f1], g))
    allreduce_sum_(part)
    adj = oracle.adjoint(y, g)
    pieces = [None] * world
    dist.all_gather_object(pieces, (f0, f1, adj))
    if rank == 0:
        gfull = oracle.make_geometry(N, L, R, theta, delta, frames, T)
        yf = oracle.forward(V, gfull)
        af = oracle.adjoint(y, gfull)
        cat = np.concatenate([p[2] for p in sorted(pieces, key=lambda z: z[0])], axis=-1)
        q.put((float(np.max(np.abs(part.numpy() - yf))), float(np.max(np.abs(cat - af)))))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_bin_sharding_matches_unsharded():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    ef, ea = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert ef < 1e-10 and ea < 1e-10
