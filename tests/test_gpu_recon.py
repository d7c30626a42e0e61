"""GPU loss, gradient and Adam reconstruction against the FP64 oracle.

Bar: the volume after the same iterations within 1e-3 relative L2 of the
oracle's; loss values within 1e-4; gradients within 1e-4.
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import rel, geometry, random_case, workload_case

pytestmark = pytest.mark.gpu

TOL_RECON = 1e-3
TOL_GRAD = 1e-4


def _params(w, iters):
    from paper_2311_13177_gb300 import ReconParams
    return (ReconParams(iters=iters, lr=w.lr, tv_xy=w.tv_xy, tv_t=w.tv_t, tv_eps=w.tv_eps),
            oracle.ReconParams(iters=iters, lr=w.lr, tv_xy=w.tv_xy, tv_t=w.tv_t, tv_eps=w.tv_eps))


# The small dynamic problem runs at kernel width 8: with width 6 the NUFFT's
# ~6e-6 operator error is amplified by Adam's sign-like early steps to ~1.6e-3
# after 20 iterations even in exact arithmetic (an FP64 emulation of the
# width-6 NUFFT trajectory against the exact-NDFT oracle gives 1.6e-3; width
# 8 gives 1e-6), so only width 8 tests the temporal path at the 1e-3 bar.
@pytest.mark.parametrize("name,iters,kbw", [("tiny", 20, 6), ("tiny", 20, 8), ("dyn_small", 20, 8),
                                            ("small64", 100, 6)])
def test_reconstruction_matches_oracle(name, iters, kbw):
    from paper_2311_13177_gb300 import Plan
    w, p = workload_case(name)
    g = geometry(w.N, w.L, w.R, p["theta"], p["delta"], p["blade_frame"], w.T)
    pg, po = _params(w, iters)
    plan = Plan(w.N, w.L, w.R, p["theta"], p["delta"], p["blade_frame"], w.T, kb_width=kbw)
    V, tr = plan.reconstruct(torch.from_numpy(p["y"]).cuda(), pg)
    Vo, tro = oracle.reconstruct(p["y"].astype(np.complex128), g, po)
    e = rel(V.cpu().numpy(), Vo)
    et = np.max(np.abs(tr - tro) / np.abs(tro))
    plan.destroy()
    assert e < TOL_RECON, e
    assert et < 1e-4, et
    assert tro[-1] < tro[0]


@pytest.mark.parametrize("kbw", [8])
def test_full_static_workload_three_iterations_match_oracle(kbw):
    """The benchmark's own configuration (256^2, 32 bins, 16 blades x 24 x
    256, kernel width 8 as benchmarked): 3 iterations of prop_reconstruct
    against the FP64 oracle's exact-NDFT iterations (about 20 s each on the
    host cores).  Width 6 misses this bar here (3.3e-3 after 3 iterations):
    Adam's first step is the sign of each gradient component, and the
    width-6 operator error (~8e-6) flips the components whose gradient is
    that close to zero."""
    from paper_2311_13177_gb300 import Plan
    w, p = workload_case("static")
    g = geometry(w.N, w.L, w.R, p["theta"], p["delta"], p["blade_frame"], w.T)
    pg, po = _params(w, 3)
    plan = Plan(w.N, w.L, w.R, p["theta"], p["delta"], p["blade_frame"], w.T, kb_width=kbw)
    V, tr = plan.reconstruct(torch.from_numpy(p["y"]).cuda(), pg)
    V = V.cpu().numpy()
    plan.destroy()
    Vo, tro = _oracle_static_3iters(p, g, po)
    e = rel(V, Vo)
    et = np.max(np.abs(tr - tro) / np.abs(tro))
    print(f"width {kbw}: volume rel {e:.3e}, trace rel {et:.3e}")
    assert e < TOL_RECON, e
    assert et < 1e-4, et


_ORACLE_CACHE = {}


def _oracle_static_3iters(p, g, po):
    if "static3" not in _ORACLE_CACHE:
        _ORACLE_CACHE["static3"] = oracle.reconstruct(p["y"].astype(np.complex128), g, po)
    return _ORACLE_CACHE["static3"]


def test_multi_chunk_reconstruction_matches_oracle():
    """Bins in two grid passes (chunk 4 of 8): the separate adjoint-row and
    TV + Adam kernels instead of the fused row kernel."""
    from paper_2311_13177_gb300 import Plan
    w, p = workload_case("tiny")
    g = geometry(w.N, w.L, w.R, p["theta"], p["delta"], p["blade_frame"], w.T)
    pg, po = _params(w, 20)
    plan = Plan(w.N, w.L, w.R, p["theta"], p["delta"], p["blade_frame"], w.T, bin_chunk=4)
    V, tr = plan.reconstruct(torch.from_numpy(p["y"]).cuda(), pg)
    Vo, tro = oracle.reconstruct(p["y"].astype(np.complex128), g, po)
    plan.destroy()
    assert rel(V.cpu().numpy(), Vo) < TOL_RECON
    assert np.max(np.abs(tr - tro) / np.abs(tro)) < 1e-4


@pytest.mark.parametrize("name,bin_chunk", [("tiny", 0), ("dyn_small", 0), ("tiny", 4)])
def test_reconstruct_equals_step_sequence(name, bin_chunk):
    """prop_reconstruct hands each iteration's forward row transform to the
    next one; prop_recon_step recomputes it.  Same iterates, bit for bit."""
    from paper_2311_13177_gb300 import Plan
    w, p = workload_case(name)
    pg, _ = _params(w, 9)
    plan = Plan(w.N, w.L, w.R, p["theta"], p["delta"], p["blade_frame"], w.T, bin_chunk=bin_chunk)
    y = torch.from_numpy(p["y"]).cuda()
    V, tr = plan.reconstruct(y, pg)
    a = torch.zeros(plan.vol_shape, dtype=torch.complex64, device="cuda")
    b = torch.empty_like(a)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    trs = []
    for k in range(1, 10):
        plan.recon_step(y, pg, k, a, b, loss)
        trs.append(float(loss.item()))
        a, b = b, a
    plan.destroy()
    assert torch.equal(V, a)
    assert np.array_equal(np.array(trs), tr)


def test_loss_and_gradient_match_oracle():
    """Random volume, three frames of which the middle one has no blades."""
    from paper_2311_13177_gb300 import Plan, ReconParams
    c = random_case(48, 6, 5, 8, 48, T=3, seed=4)
    c["blade_frame"] = np.array([0, 0, 2, 2, 2], dtype=np.int32)
    g = geometry(48, 8, 48, c["theta"], c["delta"], c["blade_frame"], 3)
    V = (c["V"] * np.float32(0.1)).astype(np.complex64)
    pg = ReconParams(tv_xy=3e-2, tv_t=2e-2, tv_eps=5e-2)
    po = oracle.ReconParams(tv_xy=3e-2, tv_t=2e-2, tv_eps=5e-2)
    plan = Plan(48, 8, 48, c["theta"], c["delta"], c["blade_frame"], 3)
    loss, grad = plan.loss_grad(torch.from_numpy(c["y"]).cuda(), pg, torch.from_numpy(V).cuda())
    lo, go = oracle.loss_and_grad(V.astype(np.complex128), c["y"].astype(np.complex128), g, po)
    plan.destroy()
    assert abs(loss - lo) / abs(lo) < 1e-5
    assert rel(grad.cpu().numpy(), go) < TOL_GRAD


def test_host_api_matches_device_api():
    from paper_2311_13177_gb300 import Plan, ReconParams
    w, p = workload_case("tiny")
    plan = Plan(w.N, w.L, w.R, p["theta"], p["delta"], p["blade_frame"], w.T)
    pg = ReconParams(iters=7, lr=w.lr, tv_xy=w.tv_xy)
    Vd, trd = plan.reconstruct(torch.from_numpy(p["y"]).cuda(), pg)
    Vh, trh = plan.reconstruct_host(p["y"].copy(), pg, trace=True)
    plan.destroy()
    assert rel(Vh, Vd.cpu().numpy()) < 1e-6
    assert np.allclose(trh, trd, rtol=1e-6)


def _row_kernel_plan(c, T, row_kernel):
    from paper_2311_13177_gb300 import Plan
    return Plan(c["N"], c["L"], c["R"], c["theta"], c["delta"], c["blade_frame"], T, kb_width=8,
                row_kernel=row_kernel)


def test_row_kernels_same_iterates_and_match_oracle():
    """row_kernel 1 (one CTA per image row and 16 bins) and 2 (persistent,
    warp-specialised): the same iterates bit for bit, both within the
    reconstruction bar of the oracle.  Two frames (temporal TV), 16 bins."""
    from paper_2311_13177_gb300 import ReconParams
    c = random_case(32, 16, 4, 6, 32, T=2, seed=21)
    g = geometry(32, 6, 32, c["theta"], c["delta"], c["blade_frame"], 2)
    pg = ReconParams(iters=10, lr=1e-2, tv_xy=1e-3, tv_t=1e-2)
    po = oracle.ReconParams(iters=10, lr=1e-2, tv_xy=1e-3, tv_t=1e-2)
    y = torch.from_numpy(c["y"]).cuda()
    out = {}
    for rk in (1, 2):
        plan = _row_kernel_plan(c, 2, rk)
        out[rk] = plan.reconstruct(y, pg)
        plan.destroy()
    assert torch.equal(out[1][0], out[2][0])
    # the TV partial sums are grouped per CTA: the loss traces agree to rounding
    assert np.max(np.abs(out[1][1] - out[2][1]) / np.abs(out[1][1])) < 1e-6
    Vo, tro = oracle.reconstruct(c["y"].astype(np.complex128), g, po)
    assert rel(out[2][0].cpu().numpy(), Vo) < TOL_RECON
    assert np.max(np.abs(out[2][1] - tro) / np.abs(tro)) < 1e-4


def test_warp_specialised_reconstruct_equals_step_sequence():
    from paper_2311_13177_gb300 import ReconParams
    c = random_case(48, 31, 5, 6, 48, T=3, seed=22)   # 2N = 96 (radix 3), ragged second bin group
    pg = ReconParams(iters=6, lr=1e-2, tv_xy=1e-3, tv_t=1e-2)
    plan = _row_kernel_plan(c, 3, 2)
    y = torch.from_numpy(c["y"]).cuda()
    V, tr = plan.reconstruct(y, pg)
    a = torch.zeros(plan.vol_shape, dtype=torch.complex64, device="cuda")
    b = torch.empty_like(a)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    trs = []
    for k in range(1, 7):
        plan.recon_step(y, pg, k, a, b, loss)
        trs.append(float(loss.item()))
        a, b = b, a
    plan.destroy()
    assert torch.equal(V, a)
    assert np.array_equal(np.array(trs), tr)


@pytest.mark.parametrize("shape", [(32, 8, 3, 4, 32), (32, 4, 2, 4, 32)])
def test_warp_specialised_row_kernel_rejected_where_impossible(shape):
    """Bin strides of 8 and 4 (less than the 16-bin unit) cannot run it."""
    from paper_2311_13177_gb300._lib import PropError
    N, Nf, B, L, R = shape
    c = random_case(N, Nf, B, L, R, seed=3)
    with pytest.raises(PropError):
        _row_kernel_plan(c, 1, 2)

