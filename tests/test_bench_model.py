"""The bench's algorithmic byte model (the denominators of its roofline
fractions): B_iter = 9|V| + 4|G| + 3|y| with |V| = 8 T N^2 Nf,
|G| = 8 T (2N)^2 Nf and |y| = 8 B L R, split over the iteration's stages.
Checked against the per-configuration sums worked out by hand from the
workload definitions (static 421.8 MB, dynamic 3779.6 MB) and against the
per-stage split summing to the iteration total."""
import importlib.util
import os
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_model_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("cfg,total_mb", [
    (dict(T=1, N=256, Nf=32, B=16, L=24, R=256), 421.789696),    # static
    (dict(T=32, N=192, Nf=16, B=64, L=16, R=192), 3779.592192),  # dynamic: 9 x 150.994944 + 4 x 603.979776 + 3 x 1.572864
])
def test_byte_model_matches_the_workload_sums(cfg, total_mb):
    bench = _bench()
    algo, b_iter = bench.stage_algo_bytes(types.SimpleNamespace(**cfg))
    assert b_iter == pytest.approx(total_mb * 1e6, rel=1e-9)
    V = 8 * cfg["T"] * cfg["N"] ** 2 * cfg["Nf"]
    G = 8 * cfg["T"] * (2 * cfg["N"]) ** 2 * cfg["Nf"]
    y = 8 * cfg["B"] * cfg["L"] * cfg["R"]
    # the fused iteration's five stages carry the whole model
    fused = algo["fft_fwd_cols"] + algo["interp"] + algo["spread"] + algo["fft_adj_cols"] + algo["rows_update"]
    assert fused == 9 * V + 4 * G + 3 * y == b_iter
    # the unfused split (forward rows, adjoint rows, TV + Adam) carries the same bytes
    unfused = (algo["fft_fwd_rows"] + algo["fft_fwd_cols"] + algo["interp"] + algo["spread"] + algo["fft_adj_cols"]
               + algo["fft_adj_rows"] + algo["tv_adam"])
    assert unfused == b_iter
