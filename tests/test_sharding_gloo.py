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


class _OracleShard:
    """A rank's shard computed by the FP64 oracle (test stand-in for a GPU plan
    over the rank's bins), with the same two calls as the library's plan."""

    def __init__(self, g, params):
        import oracle
        self.o, self.g, self.p = oracle, g, params
        self.vol_shape = (g.T, g.N, g.N, g.Nf)
        self.m = self.v = None

    def shard_forward(self, V, y_part, reuse_rows=False, accumulate=False):
        y_part.copy_(torch.from_numpy(self.o.forward(V.numpy(), self.g)))

    def shard_update(self, y, y_sum, params, k, V_in, V_out, parts):
        V = V_in.numpy()
        r = y_sum.numpy() - y.numpy()
        grad = 2.0 * self.o.adjoint(r, self.g)
        tv = 0.0
        if self.p.tv_xy:
            v, gr = self.o.tv_xy(V, self.p.tv_eps)
            tv += self.p.tv_xy * v
            grad += self.p.tv_xy * gr
        if self.p.tv_t:
            v, gr = self.o.tv_t(V, self.p.tv_eps)
            tv += self.p.tv_t * v
            grad += self.p.tv_t * gr
        if k == 1:
            self.m = np.zeros(V.shape + (2,))
            self.v = np.zeros(V.shape + (2,))
        Vn, self.m, self.v = self.o.adam_step(V, grad, self.m, self.v, k, self.p)
        V_out.copy_(torch.from_numpy(Vn))
        parts[0] = float(np.sum(np.abs(r) ** 2))
        parts[1] = tv


def _driver_worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle
    from paper_2311_13177_gb300.sharding import bin_shards, allreduce_sum_, BinShardedReconstruction
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(1)
    N, L, R, Nf, T = 16, 4, 16, 5, 2
    theta = rng.uniform(0, np.pi, 3)
    delta = np.linspace(-2, 2, Nf)
    frames = [0, 1, 1]
    y = rng.standard_normal((3, L, R)) + 1j * rng.standard_normal((3, L, R))
    prm = oracle.ReconParams(iters=6, lr=2e-2, tv_xy=1e-2, tv_t=2e-2, tv_eps=1e-2)
    f0, f1 = bin_shards(Nf, world)[rank]
    g = oracle.make_geometry(N, L, R, theta, delta[f0:f1], frames, T)
    drv = BinShardedReconstruction(_OracleShard(g, prm), torch.from_numpy(y), prm, allreduce_sum_)
    V, trace = drv.run(prm.iters)
    pieces = [None] * world
    dist.all_gather_object(pieces, (f0, V.numpy()))
    if rank == 0:
        gfull = oracle.make_geometry(N, L, R, theta, delta, frames, T)
        Vo, tro = oracle.reconstruct(y, gfull, prm)
        cat = np.concatenate([p[1] for p in sorted(pieces, key=lambda z: z[0])], axis=-1)
        q.put((float(np.linalg.norm(cat - Vo) / np.linalg.norm(Vo)),
               float(np.max(np.abs(trace.numpy() - tro) / np.abs(tro)))))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharded_driver_matches_unsharded_reconstruction():
    """The host protocol of a bin-sharded reconstruction (partial forward,
    all-reduce of y, per-shard residual / adjoint / TV / Adam, loss assembled
    from the data term and the summed TV parts) over two gloo ranks gives the
    unsharded oracle reconstruction, iterate and loss trace."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_driver_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    ev, et = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert ev < 1e-12 and et < 1e-12, (ev, et)
