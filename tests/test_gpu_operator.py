"""GPU forward/adjoint through the C ABI against the FP64 oracle (<= 1e-4 rel L2)."""
import numpy as np
import pytest
import torch

import oracle
from helpers import rel, geometry, random_case, workload_case

pytestmark = pytest.mark.gpu

TOL = 1e-4   # forward and adjoint, relative L2 against the exact NDFT


def _plan(c, bin_chunk=0, kb_width=0):
    from paper_2311_13177_gb300 import Plan
    return Plan(c["N"], c["L"], c["R"], c["theta"], c["delta"], c["blade_frame"], c["T"], bin_chunk=bin_chunk,
                kb_width=kb_width)


def _check(c, bin_chunk=0, kb_width=0, tol=TOL):
    g = geometry(c["N"], c["L"], c["R"], c["theta"], c["delta"], c["blade_frame"], c["T"])
    plan = _plan(c, bin_chunk, kb_width)
    dev = torch.device("cuda")
    y = plan.forward(torch.from_numpy(c["V"]).to(dev)).cpu().numpy()
    y_ref = oracle.forward(c["V"].astype(np.complex128), g)
    e1 = rel(y, y_ref)
    V = plan.adjoint(torch.from_numpy(c["y"]).to(dev)).cpu().numpy()
    V_ref = oracle.adjoint(c["y"].astype(np.complex128), g)
    e2 = rel(V, V_ref)
    plan.destroy()
    assert e1 < tol and e2 < tol, (e1, e2)
    return e1, e2


@pytest.mark.parametrize("shape", [
    (32, 8, 5, 8, 32, 1),     # tiny workload's shape
    (64, 8, 8, 16, 64, 1),    # several tiles per side
    (48, 3, 4, 6, 48, 1),     # 2N = 96 (radix 3), odd bin count
    (24, 5, 3, 4, 24, 1),     # 2N = 48, ragged spread tiles are impossible (n % 16 == 0), odd R/L mix
    (16, 2, 2, 16, 16, 2),    # two frames, L = N
    (32, 1, 3, 5, 37, 1),     # single bin, odd readout count
    (40, 1, 3, 5, 37, 1),     # 2N = 80 is not 2^a 3^b: rejected by plan creation
])
def test_forward_adjoint_match_oracle(shape):
    N, Nf, B, L, R, T = shape
    c = random_case(N, Nf, B, L, R, T, seed=N + Nf)
    if 2 * N not in (16, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024):
        from paper_2311_13177_gb300._lib import PropError
        with pytest.raises(PropError):
            _plan(c)
        return
    _check(c)


@pytest.mark.parametrize("shape,kb_width", [
    ((256, 4, 3, 4, 256, 1), 8),   # 2N = 512: radix-32 and radix-16 column passes
    ((192, 3, 4, 4, 192, 2), 6),   # 2N = 384: radices 8, 8, 6 in the column passes, two frames
])
def test_large_transform_lengths_sampled(shape, kb_width):
    """The column passes' long-transform shapes: 2048 samples of A V and 256
    voxels of A^H y, each against the oracle's exact sum."""
    N, Nf, B, L, R, T = shape
    c = random_case(N, Nf, B, L, R, T, seed=N + 5)
    g = geometry(N, L, R, c["theta"], c["delta"], c["blade_frame"], T)
    plan = _plan(c, kb_width=kb_width)
    dev = torch.device("cuda")
    rng = np.random.default_rng(N)
    y = plan.forward(torch.from_numpy(c["V"]).to(dev)).cpu().numpy().reshape(-1)
    s = rng.choice(y.size, 2048, replace=False)
    assert rel(y[s], oracle.forward_at(c["V"].astype(np.complex128), g, s)) < TOL
    Va = plan.adjoint(torch.from_numpy(c["y"]).to(dev)).cpu().numpy().reshape(-1)
    q = rng.choice(Va.size, 256, replace=False)
    assert rel(Va[q], oracle.adjoint_at(c["y"].astype(np.complex128), g, q)) < TOL
    plan.destroy()


@pytest.mark.parametrize("shape", [(32, 8, 5, 8, 32, 1), (48, 3, 4, 6, 48, 2)])
def test_width8_kernel_is_more_accurate(shape):
    """Kernel width 8: same operators, error two orders of magnitude below width 6."""
    N, Nf, B, L, R, T = shape
    c = random_case(N, Nf, B, L, R, T, seed=31 + N)
    e6 = _check(c, kb_width=6)
    e8 = _check(c, kb_width=8, tol=1e-6)
    assert e8[0] < 0.05 * e6[0] and e8[1] < 0.05 * e6[1]


def test_chunked_grid_matches_unchunked():
    """Bin chunks of 4 over Nf = 10 (ragged last chunk) recompute the grid per chunk."""
    c = random_case(32, 10, 4, 6, 32, 2, seed=3)
    _check(c, bin_chunk=4)


@pytest.mark.parametrize("shape,bin_chunk", [
    ((32, 15, 5, 8, 32, 1), 0),    # bin stride 16, last lane's second bin dead
    ((32, 31, 4, 6, 32, 2), 0),    # bin stride 32, odd bin count, two frames
    ((32, 63, 4, 6, 32, 1), 64),   # bin stride 64 (8-cell interpolation tiles)
    ((32, 40, 4, 6, 32, 1), 32),   # chunks of 32 + 8: two-bin-per-lane then one-bin-per-lane kernels
    ((32, 20, 3, 5, 32, 1), 16),   # chunks of 16 + 4
])
def test_bin_strides_and_ragged_chunks(shape, bin_chunk):
    N, Nf, B, L, R, T = shape
    c = random_case(N, Nf, B, L, R, T, seed=Nf + 100)
    _check(c, bin_chunk=bin_chunk)


def test_dense_blade_overlap_uses_global_lists():
    """1400 blades through the k-space centre: the centre cells' spread lists
    outgrow a shared-memory stage, so the plan gathers from global memory."""
    c = random_case(16, 2, 1400, 2, 16, 1, seed=9)
    _check(c)


def test_tiny_workload_both_operators():
    w, p = workload_case("tiny")
    p["V"] = np.random.default_rng(11).standard_normal((1, 32, 32, 8)).astype(np.complex64)
    _check(p)


def test_gpu_adjoint_identity_fp32():
    from paper_2311_13177_gb300 import Plan
    c = random_case(64, 8, 6, 8, 64, 2, seed=5)
    plan = _plan(c)
    dev = torch.device("cuda")
    x = torch.from_numpy(c["V"]).to(dev)
    y = torch.from_numpy(c["y"]).to(dev)
    Ax = plan.forward(x)
    Ahy = plan.adjoint(y)
    lhs = torch.vdot(y.reshape(-1).to(torch.complex128), Ax.reshape(-1).to(torch.complex128))
    rhs = torch.vdot(Ahy.reshape(-1).to(torch.complex128), x.reshape(-1).to(torch.complex128))
    assert abs(complex(lhs - rhs)) < 1e-5 * abs(complex(lhs))
    plan.destroy()


@pytest.mark.parametrize("name", ["static", "dynamic"])
def test_full_size_sampled_against_oracle(name):
    """Full-size workloads in the bench's configuration: 4096 random samples of
    A V and 512 random voxels of A^H y, each an independent exact sum."""
    from paper_2311_13177_gb300 import Plan
    w, p = workload_case(name)
    g = geometry(w.N, w.L, w.R, p["theta"], p["delta"], p["blade_frame"], w.T)
    rng = np.random.default_rng(7)
    V = (rng.standard_normal((w.T, w.N, w.N, w.Nf)) + 1j * rng.standard_normal((w.T, w.N, w.N, w.Nf))).astype(np.complex64)
    plan = Plan(w.N, w.L, w.R, p["theta"], p["delta"], p["blade_frame"], w.T)
    dev = torch.device("cuda")
    y = plan.forward(torch.from_numpy(V).to(dev)).cpu().numpy().reshape(-1)
    s = rng.choice(g.M, 4096, replace=False)
    ref = oracle.forward_at(V.astype(np.complex128), g, s)
    assert rel(y[s], ref) < TOL
    yy = p["y"]
    Vt = plan.adjoint(torch.from_numpy(yy).to(dev))
    Va = Vt.cpu().numpy().reshape(-1)
    q = rng.choice(Va.size, 512, replace=False)
    refa = oracle.adjoint_at(yy.astype(np.complex128), g, q)
    assert rel(Va[q], refa) < TOL
    # a second launch (the dynamic plan's spread claims its items from a
    # counter that each launch must leave at zero) gives the same grid
    assert torch.equal(plan.adjoint(torch.from_numpy(yy).to(dev)), Vt)
    plan.destroy()


def test_render_sums_bins():
    from paper_2311_13177_gb300 import Plan
    c = random_case(32, 6, 3, 4, 32, 2, seed=9)
    plan = _plan(c)
    V = torch.from_numpy(c["V"]).cuda()
    img = plan.render(V).cpu().numpy()
    assert np.allclose(img, oracle.render(c["V"]), atol=1e-5)
    lo = plan.render(V, 0, 2).cpu().numpy()
    assert np.allclose(lo, oracle.render(c["V"], 0, 2), atol=1e-5)
    plan.destroy()


def test_psnr_matches_oracle():
    """prop_psnr on a noisy render of two frames against the oracle's PSNR;
    identical magnitudes give +inf."""
    c = random_case(32, 6, 3, 4, 32, 2, seed=10)
    plan = _plan(c)
    rng = np.random.default_rng(12)
    ref = oracle.render(c["V"])
    img = (ref + 0.05 * (rng.standard_normal(ref.shape) + 1j * rng.standard_normal(ref.shape))).astype(np.complex64)
    ref = ref.astype(np.complex64)
    got = plan.psnr(torch.from_numpy(img).cuda(), torch.from_numpy(ref).cuda())
    want = oracle.psnr(img.astype(np.complex128), ref.astype(np.complex128))
    assert abs(got - want) < 1e-6, (got, want)
    one = plan.psnr(torch.from_numpy(img[:1]).cuda(), torch.from_numpy(ref[:1]).cuda())
    assert abs(one - oracle.psnr(img[:1].astype(np.complex128), ref[:1].astype(np.complex128))) < 1e-6
    assert plan.psnr(torch.from_numpy(ref).cuda(), torch.from_numpy(ref).cuda()) == float("inf")
    plan.destroy()


@pytest.mark.gpu
def test_fp32_fma_peak_is_plausible():
    from paper_2311_13177_gb300.binding import prop_fp32_fma_peak
    tf = prop_fp32_fma_peak(0)
    # 152 SMs x 128 FP32 lanes x 2 flops x ~2 GHz is about 80 TFLOP/s
    assert 10.0 < tf < 200.0, tf


def test_bounded_wait_gives_up_and_device_stays_usable():
    """The staged kernels' mbarrier waits are bounded: a wait on a barrier
    nobody arrives at gives up after its cycle budget, the kernel returns,
    and the device keeps working."""
    from paper_2311_13177_gb300.binding import prop_check_bounded_wait
    expired, ms = prop_check_bounded_wait(20_000_000)   # about 10 ms of SM clock
    assert expired == 1
    assert 1.0 < ms < 1000.0, ms
    x = torch.ones(4096, device="cuda")
    assert float(x.sum()) == 4096.0
