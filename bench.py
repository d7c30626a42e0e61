#!/usr/bin/env python
"""Throughput of the volumetric PROPELLER reconstruction step on GB300.

A step is one full Adam iteration of the reconstruction (forward NUFFT with
the displacement phase and bin sum, residual, adjoint NUFFT, fused TV
gradient + Adam) over the static workload: a 256 x 256 image with 32
spectral bins over [-4, 4] px, 16 uniformly rotated blades x 24 lines x 256
readout samples, complex64 data from a seeded 20-ellipse water/fat phantom.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --diff-study     (differentiation workload, grid store vs recompute)

Prints one JSON line (rank 0).  Under torchrun every rank reconstructs its
own independent problem (weak scaling, no data-path collective); the
barrier and the max over ranks use torch.distributed.

Timing: W untimed iterations, then one prop_reconstruct call of K iterations
bracketed by CUDA events on the launching stream (each iteration streams a
working set larger than the 129 MB L2).  A second, profiled call gives the
per-stage times and the dominant kernel's duration for the roofline object;
`l2_flushed_iters_per_s` repeats single steps with a 256 MiB write between
them.  `e2e` times the host-buffer API (prop_reconstruct_host) with its
copies.  The reference arm times the FP64 CPU oracle on a bounded sample of
the same step (see `cpu_baseline.sample`).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "recon iters/s at 256²×32 bins×16 blades vs roofline; p50/p99 latency, mixed load"
UNIT = "iters/s"
WORKLOAD = "static"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-projection", action="store_true",
                    help="skip the projection-model (the paper's own forward model) measurement")
    ap.add_argument("--bin-chunk", type=int, default=0, help="bins per grid pass (0: the plan's default)")
    ap.add_argument("--row-kernel", type=int, default=0, choices=[0, 1, 2],
                    help="row kernel: 0 the plan's choice, 1 per-row CTAs, 2 warp-specialised")
    ap.add_argument("--diff-study", action="store_true",
                    help="differentiation workload: grid store vs recompute (memory and time), one JSON line")
    ap.add_argument("--workload", choices=["static", "dynamic", "diff"], default=WORKLOAD,
                    help="the headline line is the static workload; the others are for comparison")
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--serve-iters", type=int, default=30)
    return ap.parse_args()


def workload_config(w) -> dict:
    kind = "static" if w.T == 1 else f"dynamic {w.T}-frame"
    opt = f"Adam lr {w.lr:g}, TV_xy {w.tv_xy:g}" + (f", TV_t {w.tv_t:g}" if w.tv_t else "")
    return {"workload": f"{kind} {w.N}x{w.N} image, {w.Nf} bins over [{w.delta_lo:g},{w.delta_hi:g}] px, "
                        f"{w.B} blades x {w.L} lines x {w.R} readout",
            "N": w.N, "Nf": w.Nf, "blades": w.B, "lines": w.L, "readout": w.R, "frames": w.T,
            "oversampling": 2, "kb_width": 6, "optimizer": opt}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# --- oracle timing (CPU baseline and the reference arm) ------------------------

def oracle_sample(bins: int = 8):
    """The static problem restricted to its first `bins` of 32 spectral bins.

    The oracle's work per iteration is linear in the bin count (every bin is
    an independent exact sum of the same size), so a step on this sample
    costs bins/32 of a full step."""
    import numpy as np
    import oracle
    import synth
    w = synth.WORKLOADS[WORKLOAD]
    p = synth.make_problem(w)
    g = oracle.make_geometry(w.N, w.L, w.R, p["theta"], p["delta"][:bins], p["blade_frame"], w.T)
    prm = oracle.ReconParams(lr=w.lr, tv_xy=w.tv_xy, tv_t=w.tv_t, tv_eps=w.tv_eps)
    V = np.zeros((w.T, w.N, w.N, bins), dtype=np.complex128)
    y = p["y"].astype(np.complex128)
    return w, g, prm, V, y, w.Nf / bins


def oracle_steps(n_steps: int, max_seconds: float, bins: int = 8):
    import numpy as np
    import oracle
    w, g, prm, V, y, scale = oracle_sample(bins)
    m = np.zeros(V.shape + (2,))
    v = np.zeros(V.shape + (2,))
    done = 0
    t0 = time.perf_counter()
    for k in range(1, n_steps + 1):
        _, grad = oracle.loss_and_grad(V, y, g, prm)
        V, m, v = oracle.adam_step(V, grad, m, v, k, prm)
        done += 1
        if time.perf_counter() - t0 > max_seconds:
            break
    dt = time.perf_counter() - t0
    return done, dt, scale


def cpu_cores() -> int:
    try:
        from threadpoolctl import threadpool_info
        n = max((i.get("num_threads", 0) for i in threadpool_info()), default=0)
        if n:
            return int(n)
    except Exception:
        pass
    return os.cpu_count() or 1


def cpu_baseline_obj(seconds: float = 20.0) -> dict:
    done, dt, scale = oracle_steps(1000, seconds)
    return {"value": done / (dt * scale), "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
            "sample": f"{done} FP64 oracle iteration(s) (exact NDFT forward + explicit adjoint, TV, Adam) "
                      f"on 8 of the 32 spectral bins of the static workload, {dt:.1f} s; "
                      f"rate scaled by 8/32 (work is linear in bins)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    warm = min(args.warmup, 1)
    if warm:
        oracle_steps(warm, 60.0)
    done, dt, scale = oracle_steps(max(1, args.steps), 120.0)
    value = done / (dt * scale)
    import synth
    w = synth.WORKLOADS[WORKLOAD]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": done, "warmup": warm, "ms_per_step": 1000.0 / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                             "sample": f"{done} oracle iteration(s) on 8 of 32 bins ({dt:.1f} s), "
                                       f"scaled by 8/32; steps capped to fit 120 s"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --- GPU arm ---------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def stage_algo_bytes(plan) -> dict:
    """Algorithmic bytes per launch of each stage (one bin chunk = all bins here).

    |V| = 8 T N^2 Nf, |G| = 8 T (2N)^2 Nf, |y| = 8 B L R.  Per iteration they
    sum to 9|V| + 4|G| + 3|y|: forward FFT reads V and writes G (split over
    its row and column kernels as |V| and |G|), interpolation reads G and the
    data and writes the residual, spread reads the residual and writes G,
    the inverse FFT reads G and writes the gradient (|G| and |V|), TV + Adam
    reads V, g, m, v and writes V, m, v.  The fused row kernel of
    prop_reconstruct (inverse row FFT + TV + Adam + the next iteration's
    forward row FFT) carries the |V| + 7|V| + |V| of the three stages it
    replaces."""
    V = 8 * plan.T * plan.N * plan.N * plan.Nf
    G = 8 * plan.T * (2 * plan.N) ** 2 * plan.Nf
    y = 8 * plan.B * plan.L * plan.R
    return {"fft_fwd_rows": V, "fft_fwd_cols": G, "interp": G + 2 * y, "spread": y + G,
            "fft_adj_cols": G, "fft_adj_rows": V, "tv_adam": 7 * V,
            "rows_update": 9 * V}, 9 * V + 4 * G + 3 * y


def stage_alu_flops(plan, W: int = 6) -> dict:
    """FP32 flops per launch of the interpolation and the spread.

    Interpolation, per sample and bin: W x W taps of a real weight times a
    complex grid value (2 W^2 FMA), the W column weights (2 W FMA), the
    complex phase product (6 flops) and the bin sum (2 flops): 4 W^2 + 4 W + 8
    flops.  Spread, per sample and bin: the phased residual (6 flops) and W^2
    weighted complex accumulations (4 W^2 flops)."""
    sb = plan.B * plan.L * plan.R * plan.Nf
    return {"interp": sb * (4 * W * W + 4 * W + 8), "spread": sb * (4 * W * W + 6)}


def run_serving(n_req: int, iters: int, seed: int, device: int, slots: int = 8) -> dict:
    """Mixed-load serving: the request server against sequential lone solves.

    Requests draw N from {128, 192, 256, 384}, blades from {8, 16, 24, 32}
    (lines = N/8), Nf from {8, 16, 32, 64} and static or dynamic (16 frames),
    each with its own seeded phantom.  (1) sequential: each request solved
    alone in arrival order (plan build + reconstruction), giving mu_seq;
    (2) saturated: Poisson arrivals at 4 mu_seq, recons/s = requests /
    makespan; (3) latency: Poisson arrivals at 0.7 mu_seq through the server,
    latency = result time - submission time, against a FIFO queue of the lone
    solves over the same arrivals (their measured service times).  Every
    result of (2) is compared with its lone solve."""
    import numpy as np
    import torch
    import synth
    from paper_2311_13177_gb300 import Plan, ReconParams
    from paper_2311_13177_gb300.serve import Server

    reqs = synth.make_serve_requests(n_req, seed=seed, iters=iters)
    probs = [synth.make_problem(w) for w in reqs]

    def params(w):
        return ReconParams(iters=w.iters, lr=w.lr, tv_xy=w.tv_xy, tv_t=w.tv_t, tv_eps=w.tv_eps)

    dev = torch.device("cuda", device)
    lone, service = [], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for w, p in zip(reqs, probs):
        ts = time.perf_counter()
        plan = Plan(w.N, w.L, w.R, p["theta"], p["delta"], p["blade_frame"], w.T, device=device)
        V, _ = plan.reconstruct(torch.from_numpy(p["y"]).to(dev), params(w), trace=False)
        lone.append(V.cpu().numpy())
        plan.destroy()
        del V
        service.append(time.perf_counter() - ts)
    t_seq = time.perf_counter() - t0
    mu_seq = n_req / t_seq
    budget = int(min(torch.cuda.get_device_properties(device).total_memory * 0.6, 160e9))

    def serve(arrivals):
        srv = Server(budget, max_slots=slots, device=device)
        t_start = time.perf_counter()
        tickets = []
        for w, p, at in zip(reqs, probs, arrivals):
            delay = t_start + at - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.submit(w.N, w.L, w.R, p["theta"], p["delta"], p["y"], params(w),
                                      blade_frame=p["blade_frame"], T=w.T))
        outs = []
        for t in tickets:
            vol, lat, _ = srv.wait(t)
            outs.append((vol, lat))
        makespan = time.perf_counter() - t_start
        st = srv.stats()
        srv.close()
        return outs, makespan, st

    rng = np.random.default_rng(seed + 1)
    arr_sat = np.cumsum(rng.exponential(1.0 / (4.0 * mu_seq), n_req))
    outs, makespan, st = serve(list(arr_sat))
    mismatch = max(float(np.linalg.norm(o[0] - l) / max(np.linalg.norm(l), 1e-30)) for o, l in zip(outs, lone))
    arr = np.cumsum(rng.exponential(1.0 / (0.7 * mu_seq), n_req))
    outs_l, _, _ = serve(list(arr))
    lat = np.array([o[1] for o in outs_l]) * 1000.0
    fifo, done = [], 0.0
    for at, sv in zip(arr, service):
        done = max(done, at) + sv
        fifo.append(1000.0 * (done - at))
    return {"requests": n_req, "iters_per_request": iters, "slots": slots, "hbm_budget_bytes": budget,
            "sequential_recons_per_s": mu_seq, "batched_recons_per_s": n_req / makespan,
            "speedup_vs_sequential": (n_req / makespan) / mu_seq, "saturated_arrivals": "Poisson at 4 x sequential rate",
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "arrivals": "Poisson at 0.7 x sequential rate"},
            "sequential_fifo_latency_ms": {"p50": float(np.percentile(fifo, 50)),
                                           "p99": float(np.percentile(fifo, 99))},
            "max_rel_diff_mix_vs_alone": mismatch, "arena_peak_bytes": int(st["arena_peak_bytes"]),
            "mix": "N {128,192,256,384}, blades {8,16,24,32}, lines N/8, Nf {8,16,32,64}, static or dynamic T=16"}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2311_13177_gb300 import build as _b
    if rank == 0:
        _b.build()
    if world > 1:
        dist.barrier()
    import synth
    from paper_2311_13177_gb300 import Plan, ReconParams

    w = synth.WORKLOADS[args.workload]
    w_rank = synth.Workload(**{**w.__dict__, "seed": w.seed + rank})
    prob = synth.make_problem(w_rank)
    plan = Plan(w.N, w.L, w.R, prob["theta"], prob["delta"], prob["blade_frame"], w.T, device=local,
                bin_chunk=args.bin_chunk, row_kernel=args.row_kernel)
    params = ReconParams(iters=1, lr=w.lr, tv_xy=w.tv_xy, tv_t=w.tv_t, tv_eps=w.tv_eps)
    y = torch.from_numpy(prob["y"]).to(dev)
    Va = torch.zeros(plan.vol_shape, dtype=torch.complex64, device=dev)
    Vb = torch.empty_like(Va)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    # Warm-up, then the timed region: one prop_reconstruct call of K
    # iterations, back to back.  Each iteration streams a working set (grid,
    # row workspace, volumes, moments, lists) larger than the 129 MB L2, so
    # no flush is inserted between iterations.
    plan.reconstruct(y, dataclasses.replace(params, iters=args.warmup), Va, trace=False)
    torch.cuda.synchronize()
    K = args.steps
    Va.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    e0.record(stream)
    _, tr = plan.reconstruct(y, dataclasses.replace(params, iters=K), Va, trace=False)
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    t_run = e0.elapsed_time(e1) / 1000.0
    if world > 1:
        tt = torch.tensor([t_run], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
    else:
        t_max = t_run
    value = world * K / t_max

    # Stage breakdown: the same call again with every launch bracketed by
    # events (not part of the timed region above).
    Vp = torch.zeros_like(Va)
    plan.profile_read()
    plan.profile_enable(True)
    _, trace = plan.reconstruct(y, dataclasses.replace(params, iters=K), Vp, trace=True)
    plan.profile_enable(False)
    prof = plan.profile_read()
    final_loss = float(trace[-1])
    del Vp

    # Per-step rate with the L2 flushed before every step (prop_recon_step,
    # 256 MiB write in between, events around each step).
    Kf = min(K, 500)
    Va2 = torch.zeros_like(Va)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(Kf)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(Kf)]
    for i in range(Kf):
        flush.fill_(i & 0xFF)
        starts[i].record(stream)
        plan.recon_step(y, params, i + 1, Va2, Vb, loss)
        ends[i].record(stream)
        Va2, Vb = Vb, Va2
    torch.cuda.synchronize()
    flushed_rate = Kf / (sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)) / 1000.0)
    del Va2

    # End to end through the host-buffer API: pinned y and V, copies inside.
    y_h = torch.from_numpy(prob["y"]).pin_memory()
    V_h = torch.zeros(plan.vol_shape, dtype=torch.complex64).pin_memory()
    K_e2e = max(1, min(K, 2000))
    plan.reconstruct_host(y_h, dataclasses.replace(params, iters=3), V_h)  # staging warm-up
    V_h.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan.reconstruct_host(y_h, dataclasses.replace(params, iters=K_e2e), V_h)
    t_e2e = time.perf_counter() - t0
    if world > 1:
        tt = torch.tensor([t_e2e], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_e2e = float(tt.item())
    vol_bytes = 8 * int(np.prod(plan.vol_shape))
    y_bytes = 8 * int(np.prod(plan.data_shape))

    if rank == 0:
        algo, b_iter = stage_algo_bytes(plan)
        stages = {k_: v_ for k_, v_ in prof.items() if v_[1] > 0}
        dom = max(stages, key=lambda s: stages[s][0])
        dom_ms = stages[dom][0] / stages[dom][1]
        peak, peak_kind = measured_peaks()
        achieved = algo[dom] / (dom_ms / 1000.0) / 1e9
        traffic = None
        tr_path = os.path.join(ROOT, "profiles", "traffic.json")
        if os.path.exists(tr_path):
            with open(tr_path) as f:
                traffic = json.load(f).get(args.workload, {}).get(dom)
            if traffic is not None:
                traffic = float(traffic)
        launches = sum(v_[1] for v_ in prof.values())
        from paper_2311_13177_gb300.binding import prop_fp32_fma_peak
        fma = prop_fp32_fma_peak(local)
        flops = stage_alu_flops(plan)
        alu = {"fp32_fma_peak_tflops": fma, "peak_source": "measured by prop_fp32_fma_peak",
               "ridge_flop_per_byte": fma * 1e12 / (peak * 1e9)}
        for st_ in ("interp", "spread"):
            if st_ in stages:
                ms_ = stages[st_][0] / stages[st_][1]
                alu[st_] = {"tflops": flops[st_] / (ms_ / 1000.0) / 1e12,
                            "frac": flops[st_] / (ms_ / 1000.0) / 1e12 / fma,
                            "flop_per_byte": flops[st_] / algo[st_]}
        ws = plan.workspace_bytes() + 8 * int(np.prod(plan.vol_shape)) + 8 * int(np.prod(plan.data_shape))
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": 1000.0 * t_max / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "fp32", "data": "synthetic",
            "config": {**workload_config(w),
                       "l2": f"inputs larger than L2: each iteration streams a {ws / 1e6:.0f} MB working set "
                             f"(129 MB L2); K iterations back to back in one prop_reconstruct call",
                       "parallelism": f"replicas{world}" if world > 1 else "single"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": dom,
                         "peak_source": f"{peak_kind} hbm_gbs",
                         "kernel_ms": dom_ms, "algo_bytes_per_launch": algo[dom]},
            "alu_roofline": alu,
            "iteration_roofline": {"algo_bytes_per_iter": b_iter,
                                   "achieved_gbs": b_iter * value / world / 1e9,
                                   "frac": b_iter * value / world / 1e9 / peak,
                                   "roofline_iters_per_s": peak * 1e9 / b_iter},
            "stages_ms_per_step": {s: v_[0] / K for s, v_ in stages.items()},
            "l2_flushed_iters_per_s": flushed_rate,
            "l2_flushed_note": f"prop_recon_step with a 256 MiB write before each of {Kf} steps",
            "e2e": {"value": world * K_e2e / t_e2e, "unit": UNIT,
                    "h2d_bytes_per_step": (y_bytes + vol_bytes) / K_e2e,
                    "d2h_bytes_per_step": vol_bytes / K_e2e,
                    "note": f"prop_reconstruct_host: one call of {K_e2e} iterations per rank, "
                            f"pinned host y and V copied in and V copied out inside the timed region"},
            "gpu_launches": launches,
            "clocks": clk,
            "final_loss": final_loss,
            "wall_s": wall,
        }
        if world == 1 and not args.no_cpu_baseline and args.workload == WORKLOAD:
            line["cpu_baseline"] = cpu_baseline_obj()
        if world == 1 and not args.no_serving and args.serve_requests > 0 and args.workload == WORKLOAD:
            line["serving"] = run_serving(args.serve_requests, args.serve_iters, 7, local)
        if world == 1 and not args.no_projection and args.workload == WORKLOAD:
            line["projection_model"] = run_projection_model(plan, w, prob, dev, peak, K)
        print(json.dumps(line), flush=True)
    plan.destroy()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_projection_model(plan, w, prob, dev, peak, K):
    """The paper's own forward model (interpolated projection, Cartesian DFT
    and blade mask, image- plus k-space loss, one blade per iteration) on the
    same plan: Cartesian blade data of the same phantom, one
    prop_proj_reconstruct call of K iterations timed with CUDA events.
    Algorithmic bytes per iteration: the projected frame of V (|V| / T), V, m
    and v read and written by the update (6 |V|), and ten passes over an
    N x N complex image (projection, four transform passes, the gradient)."""
    import numpy as np
    import torch
    import synth
    from paper_2311_13177_gb300 import ProjParams
    rng = np.random.default_rng(w.seed + 1)
    yc = synth.simulate_cartesian_blades(prob["ellipses"], w.N, prob["theta"], w.fat_shift)
    yc = synth.add_noise(yc, w.rel_sigma, rng).astype(np.complex64)
    ycart = torch.from_numpy(yc).to(dev)
    q = dict(lr=w.lr, w_kspace=0.1, w_image=1.0, tv_xy=1e-3, tv_f=1e-3, l1=1e-4, tv_eps=w.tv_eps)
    V = torch.zeros(plan.vol_shape, dtype=torch.complex64, device=dev)
    plan.proj_reconstruct(ycart, ProjParams(iters=5, **q), V=V, trace=False)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    V.zero_()
    e0.record(s)
    plan.proj_reconstruct(ycart, ProjParams(iters=K, **q), V=V, trace=False)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    _, tr = plan.proj_reconstruct(ycart, ProjParams(iters=2 * w.B, **q), V=torch.zeros_like(V), trace=True)
    vol = 8.0 * float(np.prod(plan.vol_shape))
    b_iter = vol / w.T + 6.0 * vol + 10.0 * 8.0 * w.N * w.N
    rate = K / (ms / 1000.0)
    return {"value": rate, "unit": "iters/s", "ms_per_iter": ms / K, "iters": K,
            "config": f"{w.N}x{w.N}, {w.Nf} bins, {w.B} blades (Cartesian masks of {w.L} x {w.R}), one blade "
                      f"per iteration; w_k 0.1, w_i 1, TV_xy 1e-3, TV_f 1e-3, L1 1e-4",
            "roofline": {"bound": "hbm", "algo_bytes_per_iter": b_iter, "achieved_gbs": b_iter * rate / 1e9,
                         "peak": peak, "frac": b_iter * rate / 1e9 / peak,
                         "roofline_iters_per_s": peak * 1e9 / b_iter},
            "loss_first_pass": float(np.sum(tr[:w.B])), "loss_second_pass": float(np.sum(tr[w.B:]))}


def run_diff_study(args):
    """Forward + backward through the autograd op at the differentiation
    workload (384^2, 64 bins, 32 blades x 32 x 384) for several bin chunks.
    Chunk 64 keeps the oversampled grid of every bin resident at once
    ("store"); smaller chunks reuse one chunk-sized grid and recompute it per
    chunk in both directions ("recompute").  Reports the plan's device bytes
    and the time of one forward + backward (CUDA events, after warm-up)."""
    import torch
    import synth
    from paper_2311_13177_gb300 import build as _b
    _b.build()
    from paper_2311_13177_gb300 import Plan, prop_apply
    torch.cuda.set_device(0)
    w = synth.WORKLOADS["diff"]
    p = synth.make_problem(w)
    dev = torch.device("cuda", 0)
    y = torch.from_numpy(p["y"]).to(dev)
    rows = []
    for chunk in (8, 16, 32, 64):
        plan = Plan(w.N, w.L, w.R, p["theta"], p["delta"], p["blade_frame"], w.T, bin_chunk=chunk)
        V = torch.zeros(plan.vol_shape, dtype=torch.complex64, device=dev, requires_grad=True)

        def step():
            r = prop_apply(V, plan) - y
            loss = (r.real ** 2 + r.imag ** 2).sum()
            loss.backward()
        for _ in range(3):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 20
        e0.record()
        for _ in range(reps):
            step()
        e1.record()
        torch.cuda.synchronize()
        rows.append({"bin_chunk": chunk, "mode": "store" if chunk >= w.Nf else "recompute",
                     "plan_device_bytes": plan.workspace_bytes(),
                     "ms_forward_backward": e0.elapsed_time(e1) / reps})
        plan.destroy()
        del V
    print(json.dumps({"study": "differentiation grid store vs recompute",
                      "workload": "384x384, 64 bins, 32 blades x 32 lines x 384 readout, fp32",
                      "note": "forward + backward of sum |A V - y|^2 through torch.autograd (prop_forward, prop_adjoint)",
                      "rows": rows}), flush=True)


def main():
    args = parse()
    if args.diff_study:
        run_diff_study(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
