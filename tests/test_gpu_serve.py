"""Request server (continuous batching) on the GPU.

Each request's result in a mix must equal the same reconstruction run alone
through prop_reconstruct (the kernels are deterministic and every request
has its own buffers, so the target is bitwise; the bar is 1e-6 relative L2).
"""
import time

import numpy as np
import pytest

import synth
from helpers import rel

pytestmark = pytest.mark.gpu


def _requests(n=8, seed=3):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        N = int(rng.choice([32, 48, 64]))
        Nf = int(rng.choice([4, 6, 8]))
        B = int(rng.choice([4, 6, 8]))
        dyn = i % 3 == 2
        w = synth.Workload(f"s{i}", N=N, Nf=Nf, delta_lo=-2.0, delta_hi=2.0, B=B, L=N // 4, R=N,
                           T=3 if dyn else 1, angles="golden" if dyn else "uniform", n_ellipses=5,
                           iters=int(rng.integers(8, 20)), tv_t=1e-2 if dyn else 0.0,
                           motion=(0, 2.0, 3.0) if dyn else None, seed=500 + i)
        out.append((w, synth.make_problem(w)))
    return out


def _params(w):
    from paper_2311_13177_gb300 import ReconParams
    return ReconParams(iters=w.iters, lr=w.lr, tv_xy=w.tv_xy, tv_t=w.tv_t, tv_eps=w.tv_eps)


def test_mixed_requests_equal_lone_runs():
    import torch
    from paper_2311_13177_gb300 import Plan
    from paper_2311_13177_gb300.serve import Server
    reqs = _requests()
    srv = Server(hbm_budget_bytes=2 << 30, max_slots=3)
    tickets = []
    for k, (w, p) in enumerate(reqs):
        tickets.append(srv.submit(w.N, w.L, w.R, p["theta"], p["delta"], p["y"], _params(w),
                                  blade_frame=p["blade_frame"], T=w.T))
        if k % 2:
            time.sleep(0.01)   # arrivals while others run
    results = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["arena_peak_bytes"] <= st["budget_bytes"] + (64 << 20)
    for (w, p), (vol, lat, loss) in zip(reqs, results):
        plan = Plan(w.N, w.L, w.R, p["theta"], p["delta"], p["blade_frame"], w.T)
        V, tr = plan.reconstruct(torch.from_numpy(p["y"]).cuda(), _params(w))
        alone = V.cpu().numpy()
        plan.destroy()
        assert rel(vol, alone) <= 1e-6, w.name
        assert lat > 0 and np.isfinite(loss)
        assert abs(loss - tr[-1]) <= 1e-9 * abs(tr[-1])


def test_admission_respects_budget_and_rejects_oversized():
    from paper_2311_13177_gb300.serve import Server, prop_plan_estimate_bytes
    from paper_2311_13177_gb300._lib import PropError
    reqs = _requests(4, seed=9)
    need = max(prop_plan_estimate_bytes(w.N, w.L, w.R, p["theta"], p["delta"], p["blade_frame"], w.T, w.iters)
               + 8 * (w.T * w.N * w.N * w.Nf + w.B * w.L * w.R) + 4096 for w, p in reqs)
    srv = Server(hbm_budget_bytes=need, max_slots=4)   # room for one request at a time
    ts = [srv.submit(w.N, w.L, w.R, p["theta"], p["delta"], p["y"], _params(w), blade_frame=p["blade_frame"],
                     T=w.T) for w, p in reqs]
    for t in ts:
        srv.wait(t)
    st = srv.stats()
    assert st["completed"] == 4 and st["arena_peak_bytes"] <= need
    # a request larger than the whole budget fails with PROP_ERR_OOM
    big = synth.Workload("big", N=256, Nf=32, delta_lo=-4, delta_hi=4, B=16, L=24, R=256, iters=2)
    pb = synth.make_problem(big)
    t = srv.submit(big.N, big.L, big.R, pb["theta"], pb["delta"], pb["y"], _params(big))
    with pytest.raises(PropError) as ei:
        srv.wait(t)
    assert ei.value.status == 2
    srv.close()


def test_cancel_and_poll():
    from paper_2311_13177_gb300.serve import Server
    from paper_2311_13177_gb300._lib import PropError
    w, p = _requests(1, seed=11)[0]
    srv = Server(hbm_budget_bytes=1 << 30, max_slots=1)
    from paper_2311_13177_gb300 import ReconParams
    long_params = ReconParams(iters=100000, lr=w.lr, tv_xy=w.tv_xy)
    t1 = srv.submit(w.N, w.L, w.R, p["theta"], p["delta"], p["y"], long_params, blade_frame=p["blade_frame"], T=w.T)
    t2 = srv.submit(w.N, w.L, w.R, p["theta"], p["delta"], p["y"], _params(w), blade_frame=p["blade_frame"], T=w.T)
    time.sleep(0.2)
    assert srv.poll(t1) == "running" and srv.poll(t2) == "pending"
    srv.cancel(t1)
    with pytest.raises(PropError) as ei:
        srv.wait(t1, timeout_ms=20000)
    assert ei.value.status == 7
    vol, lat, loss = srv.wait(t2, timeout_ms=60000)
    assert np.isfinite(vol).all()
    srv.close()


def test_same_class_requests_are_batched_and_equal_lone_runs():
    """Six requests of one kernel class (2N = 96, 8 bins) with four slots:
    the server advances them in batched iterations (one launch per stage for
    all running requests); each result is its lone reconstruction bit for bit."""
    import torch
    from paper_2311_13177_gb300 import Plan
    from paper_2311_13177_gb300.serve import Server
    reqs = []
    for i in range(6):
        dyn = i % 2 == 1
        w = synth.Workload(f"c{i}", N=48, Nf=8, delta_lo=-2.0, delta_hi=2.0, B=4 + i, L=8 + 2 * (i % 3), R=48,
                           T=2 if dyn else 1, angles="golden" if dyn else "uniform", n_ellipses=4,
                           iters=6 + 3 * i, tv_t=1e-2 if dyn else 0.0, motion=(0, 2.0, 3.0) if dyn else None,
                           seed=700 + i)
        reqs.append((w, synth.make_problem(w)))
    srv = Server(hbm_budget_bytes=2 << 30, max_slots=4)
    tickets = [srv.submit(w.N, w.L, w.R, p["theta"], p["delta"], p["y"], _params(w), blade_frame=p["blade_frame"],
                          T=w.T) for w, p in reqs]
    results = [srv.wait(t) for t in tickets]
    srv.close()
    for (w, p), (vol, lat, loss) in zip(reqs, results):
        plan = Plan(w.N, w.L, w.R, p["theta"], p["delta"], p["blade_frame"], w.T)
        V, tr = plan.reconstruct(torch.from_numpy(p["y"]).cuda(), _params(w))
        alone = V.cpu().numpy()
        plan.destroy()
        assert np.array_equal(vol, alone), w.name
        assert abs(loss - tr[-1]) <= 1e-12 * abs(tr[-1])
