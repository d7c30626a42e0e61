"""GPU projection model (the paper's own forward model, Sec. 4.2-4.3) through
the C ABI against the FP64 oracle.

Bars: forward and adjoint within 1e-5 relative L2 (FP32 bilinear taps and
FFTs against FP64); the volume after the same Adam iterations within 1e-3,
the loss trace within 1e-4.
"""
import numpy as np
import pytest
import torch

from oracle import projection as pj
from oracle.geometry import make_geometry
from helpers import rel

pytestmark = pytest.mark.gpu

TOL = 1e-5
TOL_RECON = 1e-3


def _case(N, Nf, B, L, R, T, seed):
    rng = np.random.default_rng(seed)
    theta = np.pi * np.arange(B) / B + rng.uniform(-0.05, 0.05, B)
    delta = np.linspace(-3.3, 2.9, Nf) if Nf > 1 else np.array([1.4])
    frames = (np.arange(B) * T // B).astype(np.int32)
    V = (rng.standard_normal((T, N, N, Nf)) + 1j * rng.standard_normal((T, N, N, Nf))).astype(np.complex64)
    return theta, delta, frames, V


def _plan(N, L, R, theta, delta, frames, T):
    from paper_2311_13177_gb300 import Plan
    return Plan(N, L, R, theta, delta, frames, T)


@pytest.mark.parametrize("shape", [
    (16, 2, 2, 4, 16, 1),     # smallest transform length
    (32, 5, 3, 8, 32, 2),     # two frames, odd bin count
    (48, 3, 2, 6, 40, 1),     # N = 48: radix-3 transforms, R != N
    (64, 8, 4, 16, 64, 1),
    (256, 32, 2, 24, 256, 1),  # the static workload's image and bins
])
def test_forward_and_adjoint_match_oracle(shape):
    N, Nf, B, L, R, T = shape
    theta, delta, frames, V = _case(N, Nf, B, L, R, T, seed=N + Nf)
    g = make_geometry(N, L, R, theta, delta, frames, T)
    plan = _plan(N, L, R, theta, delta, frames, T)
    Vd = torch.from_numpy(V).cuda()
    rng = np.random.default_rng(1)
    for b in range(B):
        z = plan.proj_forward(b, Vd).cpu().numpy()
        zr = pj.forward(V.astype(np.complex128), g, b)
        assert rel(z, zr) < TOL, (b, rel(z, zr))
        assert np.all(z[~pj.blade_mask(N, float(theta[b]), L, R)] == 0)
        y = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))).astype(np.complex64)
        Va = plan.proj_adjoint(b, torch.from_numpy(y).cuda()).cpu().numpy()
        Vr = pj.adjoint(y.astype(np.complex128), g, b)
        assert rel(Va, Vr) < TOL, (b, rel(Va, Vr))
    plan.destroy()


@pytest.mark.parametrize("with_image", [False, True])
def test_reconstruction_matches_oracle(with_image):
    """12 iterations over 4 blades and 2 frames with every term on: both data
    terms (an image that is not the k-space data's inverse DFT when given),
    TV along x-y, the spectrum and time, and L1."""
    from paper_2311_13177_gb300 import ProjParams
    N, Nf, B, L, R, T = 32, 4, 4, 8, 32, 2
    theta, delta, frames, _ = _case(N, Nf, B, L, R, T, seed=7)
    g = make_geometry(N, L, R, theta, delta, frames, T)
    rng = np.random.default_rng(8)
    Vt = np.zeros((T, N, N, Nf), dtype=np.complex128)
    Vt[:, 8:22, 10:24, 1] = 1.0
    Vt[:, 12:18, 12:16, 3] = 0.6 + 0.3j
    ycart = np.stack([pj.forward(Vt, g, b) for b in range(B)])
    ycart = (ycart + 0.01 * (rng.standard_normal(ycart.shape) + 1j * rng.standard_normal(ycart.shape))).astype(np.complex64)
    img = None
    if with_image:
        img = np.stack([pj.image_of(ycart, g, b) for b in range(B)])
        img = (img + 0.02 * rng.standard_normal(img.shape)).astype(np.complex64)
    kw = dict(iters=12, lr=2e-2, w_kspace=0.3, w_image=1.0, tv_xy=2e-3, tv_f=1e-3, tv_t=5e-3, l1=1e-3, tv_eps=1e-2)
    plan = _plan(N, L, R, theta, delta, frames, T)
    V, tr = plan.proj_reconstruct(torch.from_numpy(ycart).cuda(), ProjParams(**kw),
                                  img=None if img is None else torch.from_numpy(img).cuda())
    Vo, tro = pj.reconstruct(ycart.astype(np.complex128), None if img is None else img.astype(np.complex128), g,
                             pj.ProjParams(**kw))
    plan.destroy()
    e = rel(V.cpu().numpy(), Vo)
    et = np.max(np.abs(tr - tro) / np.abs(tro))
    assert e < TOL_RECON, e
    assert et < 1e-4, et
    assert tro[-4:].sum() < tro[:4].sum()


def test_blade_index_is_checked():
    from paper_2311_13177_gb300._lib import PropError
    theta, delta, frames, V = _case(16, 2, 2, 4, 16, 1, seed=3)
    plan = _plan(16, 4, 16, theta, delta, frames, 1)
    with pytest.raises(PropError):
        plan.proj_forward(2, torch.from_numpy(V).cuda())
    plan.destroy()


@pytest.mark.parametrize("lo,hi", [(0, 4), (1, 3)])
def test_baseline_matches_oracle(lo, hi):
    N, Nf, B, L, R, T = 32, 2, 4, 8, 32, 1
    theta, delta, frames, _ = _case(N, Nf, B, L, R, T, seed=31)
    g = make_geometry(N, L, R, theta, delta, frames, T)
    rng = np.random.default_rng(32)
    ycart = (rng.standard_normal((B, N, N)) + 1j * rng.standard_normal((B, N, N))).astype(np.complex64)
    plan = _plan(N, L, R, theta, delta, frames, T)
    img = plan.proj_baseline(torch.from_numpy(ycart).cuda(), lo, hi).cpu().numpy()
    plan.destroy()
    ref = pj.baseline(ycart.astype(np.complex128), g, lo, hi)
    assert rel(img, ref) < TOL
