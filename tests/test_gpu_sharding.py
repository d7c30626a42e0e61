"""Bin-sharded reconstruction on the GPU (prop_shard_forward / prop_shard_update).

The operator is a sum over spectral bins (Sec. 3 Eq. 2, Sec. 4.2), so plans
over disjoint runs of bins, with their partial blade data summed between the
two calls, reproduce the unsharded reconstruction up to the rounding of the
bin sum.  Two forms: several plans in one process (the partial forwards
summed in place by the library's accumulate mode), and two processes on one
GPU whose partial forwards are summed by a gloo all-reduce through host
memory (the host-side stand-in for an NCCL all-reduce across GPUs).
"""
import os
import socket

import numpy as np
import pytest
import torch

import oracle
from helpers import rel, geometry, workload_case

pytestmark = pytest.mark.gpu


def _params(w, iters):
    from paper_2311_13177_gb300 import ReconParams
    return (ReconParams(iters=iters, lr=w.lr, tv_xy=w.tv_xy, tv_t=w.tv_t, tv_eps=w.tv_eps),
            oracle.ReconParams(iters=iters, lr=w.lr, tv_xy=w.tv_xy, tv_t=w.tv_t, tv_eps=w.tv_eps))


@pytest.mark.parametrize("name,parts", [("tiny", 2), ("tiny", 3), ("dyn_small", 2)])
def test_local_shards_match_unsharded_and_oracle(name, parts):
    from paper_2311_13177_gb300 import Plan
    from paper_2311_13177_gb300.sharding import bin_shards, reconstruct_local_shards
    w, p = workload_case(name)
    iters = 20
    pg, po = _params(w, iters)
    y = torch.from_numpy(p["y"]).cuda()
    full = Plan(w.N, w.L, w.R, p["theta"], p["delta"], p["blade_frame"], w.T, kb_width=8)
    V_ref, tr_ref = full.reconstruct(y, pg)
    full.destroy()
    shards = bin_shards(len(p["delta"]), parts)
    plans = [Plan(w.N, w.L, w.R, p["theta"], p["delta"][a:b], p["blade_frame"], w.T, kb_width=8) for a, b in shards]
    Vs, tr = reconstruct_local_shards(plans, y, pg, iters)
    for pl in plans:
        pl.destroy()
    V = torch.cat(Vs, dim=-1).cpu().numpy()
    tr = tr.cpu().numpy()
    e_un = rel(V, V_ref.cpu().numpy())
    assert e_un < 1e-5, e_un
    assert np.max(np.abs(tr - tr_ref) / np.abs(tr_ref)) < 1e-5
    g = geometry(w.N, w.L, w.R, p["theta"], p["delta"], p["blade_frame"], w.T)
    Vo, tro = oracle.reconstruct(p["y"].astype(np.complex128), g, po)
    assert rel(V, Vo) < 1e-3
    assert np.max(np.abs(tr - tro) / np.abs(tro)) < 1e-4


def test_shard_forward_sums_to_forward():
    """A_1 V_1 + A_2 V_2 (the second accumulated in place) equals A V; the
    row transform left by a shard update is reused only for its own V_out."""
    from paper_2311_13177_gb300 import Plan, ReconParams
    w, p = workload_case("tiny")
    rng = np.random.default_rng(3)
    V = (rng.standard_normal((1, w.N, w.N, 8)) + 1j * rng.standard_normal((1, w.N, w.N, 8))).astype(np.complex64)
    Vt = torch.from_numpy(V).cuda()
    full = Plan(w.N, w.L, w.R, p["theta"], p["delta"], p["blade_frame"], w.T, kb_width=8)
    y_ref = full.forward(Vt)
    full.destroy()
    a = Plan(w.N, w.L, w.R, p["theta"], p["delta"][:3], p["blade_frame"], w.T, kb_width=8)
    b = Plan(w.N, w.L, w.R, p["theta"], p["delta"][3:], p["blade_frame"], w.T, kb_width=8)
    y = a.shard_forward(Vt[..., :3].contiguous())
    b.shard_forward(Vt[..., 3:].contiguous(), y, accumulate=True)
    assert rel(y.cpu().numpy(), y_ref.cpu().numpy()) < 1e-6
    # a reuse request for a volume the plan did not produce recomputes the rows
    y2 = a.shard_forward(Vt[..., :3].contiguous(), reuse_rows=True)
    y3 = a.shard_forward(Vt[..., :3].contiguous())
    assert torch.equal(y2, y3)
    a.destroy()
    b.destroy()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    import torch.distributed as dist
    from helpers import workload_case as wc
    from paper_2311_13177_gb300 import Plan, ReconParams
    from paper_2311_13177_gb300.sharding import bin_shards, host_allreduce_sum_, BinShardedReconstruction
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    w, p = wc("dyn_small")
    f0, f1 = bin_shards(len(p["delta"]), world)[rank]
    plan = Plan(w.N, w.L, w.R, p["theta"], p["delta"][f0:f1], p["blade_frame"], w.T, kb_width=8)
    prm = ReconParams(iters=12, lr=w.lr, tv_xy=w.tv_xy, tv_t=w.tv_t, tv_eps=w.tv_eps)
    drv = BinShardedReconstruction(plan, torch.from_numpy(p["y"]).cuda(), prm, host_allreduce_sum_)
    V, trace = drv.run(prm.iters)
    torch.cuda.synchronize()
    q.put((rank, f0, V.cpu().numpy(), trace.cpu().numpy()))
    plan.destroy()
    dist.barrier()
    dist.destroy_process_group()


def test_two_processes_one_gpu_gloo_match_unsharded():
    """Two ranks (processes) on the one GPU, each with a plan over half the
    bins; y is all-reduced by gloo through host copies between the calls.
    No kernel of one rank waits on the other's: every exchange is on the host."""
    import torch.multiprocessing as mp
    from paper_2311_13177_gb300 import Plan
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    outs = [q.get(timeout=300) for _ in range(2)]
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    outs.sort(key=lambda o: o[1])
    V = np.concatenate([o[2] for o in outs], axis=-1)
    assert np.array_equal(outs[0][3], outs[1][3])  # every rank assembles the same loss
    w, p = workload_case("dyn_small")
    pg, _ = _params(w, 12)
    full = Plan(w.N, w.L, w.R, p["theta"], p["delta"], p["blade_frame"], w.T, kb_width=8)
    V_ref, tr_ref = full.reconstruct(torch.from_numpy(p["y"]).cuda(), pg)
    full.destroy()
    assert rel(V, V_ref.cpu().numpy()) < 1e-5
    assert np.max(np.abs(outs[0][3] - tr_ref) / np.abs(tr_ref)) < 1e-5
