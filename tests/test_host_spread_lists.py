"""Host check of the grouped spread lists (the adjoint's plan-time tables).

The spread reads, for every 2 x 2-cell group, the samples whose footprint
meets it with their four weights; the spread is the transpose of the
interpolation (Sec. 3's forward model, its adjoint for the gradient) only
if every cell receives exactly its samples' terms in ascending sample
order.  tests/host/spread_lists_check.cu builds the lists with the plan's
own builder on the host for random geometries and compares the gather they
imply with a direct scatter, bit for bit (no GPU needed).
"""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HOST = os.path.join(ROOT, "tests", "host")


def test_grouped_spread_lists_equal_a_direct_scatter(tmp_path):
    from paper_2311_13177_gb300 import build as B
    try:
        nvcc = B.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "spread_lists_check")
    cmd = [nvcc, "-std=c++17", "-O1", "-x", "cu", "-I", B.CSRC, os.path.join(HOST, "spread_lists_check.cu"),
           os.path.join(HOST, "stubs.cu"), "-o", exe]
    b = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert b.returncode == 0, b.stderr[-3000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout[-3000:]
    assert "mismatching values 0" in r.stdout
