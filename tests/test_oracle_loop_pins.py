"""Pins of the oracle's three reconstruction loops (Sec. 4.3: Adam on the
data term plus regularisers; one blade per iteration for the paper's own
forward model) against independent torch implementations (no GPU).

Each loop is compared, on the iterate and on the loss trace, with
``torch.optim.Adam`` (float64, complex parameters) driving a loss written
separately in torch (``independent_models``: dense operators assembled entry
by entry, TV and L1 as torch expressions, gradients by autograd).  A slip in
the loop itself -- the Adam step counter starting at 0, the trace taken after
the update, V_0 not zero, the blade schedule off by one, one parameter
array's moments stepping out of turn -- fails these, which the per-function
pins cannot see.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import kplanes as kp
from oracle import projection as pj
from oracle.geometry import make_geometry

import independent_models as im

TOL = 1e-12


def _rand_c(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("start", ["zero", "given"])
def test_volume_reconstruction_loop_matches_torch_adam(start):
    """oracle.reconstruct (full-batch Adam on sum|AV - y|^2 + TV_xy + TV_t)."""
    N, L, R, T = 8, 2, 8, 2
    theta = [0.3, 1.2, 2.4]
    delta = [-1.0, 0.4, 1.7]
    frames = [0, 1, 1]
    g = make_geometry(N, L, R, theta, delta, frames, T=T)
    rng = np.random.default_rng(11)
    y = _rand_c(rng, (3, L, R))
    V0 = None if start == "zero" else 0.3 * _rand_c(rng, (T, N, N, 3))
    p = oracle.ReconParams(iters=12, lr=2e-2, tv_xy=3e-2, tv_t=5e-2, tv_eps=1e-2)
    V_o, tr_o = oracle.reconstruct(y, g, p, V0=V0)

    A = torch.tensor(im.nonuniform_matrix(N, L, R, theta, delta, frames, T))
    yt = torch.tensor(y)
    V = torch.zeros((T, N, N, 3), dtype=torch.complex128) if V0 is None else torch.tensor(V0)
    V.requires_grad_(True)
    tr_t = im.run_adam([V], lambda k: im.volume_loss(V, A, yt, p.tv_xy, p.tv_t, p.tv_eps), p.iters, p.lr,
                       (p.beta1, p.beta2), p.eps)
    assert _rel(V_o, V.detach().numpy()) < TOL
    assert np.max(np.abs(tr_o - tr_t) / np.abs(tr_t)) < TOL
    # the iterate really moved: a loop that skipped updates would fail above,
    # but make the size of the motion explicit
    start_v = np.zeros_like(V_o) if V0 is None else V0
    assert np.linalg.norm((V_o - start_v).ravel()) > 1e-2 * np.linalg.norm(V_o.ravel())


@pytest.mark.parametrize("with_images", [False, True])
def test_projection_reconstruction_loop_matches_torch_adam(with_images):
    """oracle.projection.reconstruct: Adam over the blades in turn, blade
    (k - 1) mod B in iteration k, on the k-space + image-space data terms,
    TV along x1, x2, the spectral axis and frames, and L1."""
    N, L, R, T, Nf = 8, 4, 8, 2, 3
    theta = [0.25, 1.3, 2.2]
    delta = [-1.3, 0.0, 1.6]
    frames = [0, 1, 1]
    g = make_geometry(N, L, R, theta, delta, frames, T=T)
    rng = np.random.default_rng(12)
    ycart = _rand_c(rng, (3, N, N))
    img = _rand_c(rng, (3, N, N)) if with_images else None
    p = pj.ProjParams(iters=8, lr=2e-2, w_kspace=0.3, w_image=1.0, tv_xy=2e-2, tv_f=1e-2, tv_t=3e-2, l1=1e-2,
                      tv_eps=1e-2)
    V_o, tr_o = pj.reconstruct(ycart, img, g, p)

    Ps = [torch.tensor(im.projection_matrix(N, Nf, theta[b], delta)).to(torch.complex128) for b in range(3)]
    Ms = [torch.tensor(im.blade_support(N, theta[b], L, R)) for b in range(3)]
    yc = torch.tensor(ycart)
    V = torch.zeros((T, N, N, Nf), dtype=torch.complex128, requires_grad=True)

    def loss(k):
        b = (k - 1) % 3
        t = frames[b]
        Z = im.centred_dft((Ps[b] @ V[t].reshape(-1)).reshape(N, N))
        Mz = torch.where(Ms[b], Z, torch.zeros_like(Z))
        rk = torch.where(Ms[b], Z - yc[b], torch.zeros_like(Z))
        ref_img = torch.tensor(img[b]) if with_images else im.centred_idft(torch.where(Ms[b], yc[b],
                                                                                         torch.zeros_like(Z)))
        ri = im.centred_idft(Mz) - ref_img
        out = p.w_kspace * (rk.real ** 2 + rk.imag ** 2).sum() + p.w_image * (ri.real ** 2 + ri.imag ** 2).sum()
        out = out + p.tv_xy * (im.smoothed_tv(V, 2, p.tv_eps) + im.smoothed_tv(V, 1, p.tv_eps))
        out = out + p.tv_f * im.smoothed_tv(V, 3, p.tv_eps) + p.tv_t * im.smoothed_tv(V, 0, p.tv_eps)
        return out + p.l1 * im.smoothed_l1(V, p.tv_eps)

    tr_t = im.run_adam([V], loss, p.iters, p.lr, (p.beta1, p.beta2), p.eps)
    assert _rel(V_o, V.detach().numpy()) < TOL
    assert np.max(np.abs(tr_o - tr_t) / np.abs(tr_t)) < TOL


def test_projection_schedule_is_detectably_cyclic():
    """The trace of a loop that starts at blade 1 instead of blade 0 differs,
    so the comparison above resolves the schedule."""
    N, L, R = 8, 4, 8
    g = make_geometry(N, L, R, [0.25, 1.3, 2.2], [-1.3, 0.0, 1.6])
    rng = np.random.default_rng(13)
    ycart = _rand_c(rng, (3, N, N))
    p = pj.ProjParams(iters=3, lr=2e-2)
    _, tr = pj.reconstruct(ycart, None, g, p)
    g_rot = make_geometry(N, L, R, [1.3, 2.2, 0.25], [-1.3, 0.0, 1.6])
    _, tr_rot = pj.reconstruct(np.roll(ycart, -1, axis=0), None, g_rot, p)
    assert abs(tr[0] - tr_rot[0]) / abs(tr[0]) > 1e-3


def test_kplanes_reconstruction_loop_matches_torch_adam():
    """oracle.kplanes.reconstruct: Adam on every plane and weighting vector
    (one step counter), loss = data term of the rendered volume + TV."""
    N, L, R, T, Nf, F = 8, 2, 8, 2, 3, 4
    theta = [0.3, 1.2, 2.4]
    delta = [-1.0, 0.4, 1.7]
    frames = [0, 1, 1]
    g = make_geometry(N, L, R, theta, delta, frames, T=T)
    rng = np.random.default_rng(14)
    y = 0.05 * _rand_c(rng, (3, L, R))
    prm0 = kp.init_params(N, Nf, T, rng, F=F, scales=2, spread=0.3)
    p = oracle.ReconParams(iters=10, lr=1e-2, tv_xy=1e-2, tv_t=2e-2, tv_eps=1e-2)
    prm_o, tr_o = kp.reconstruct(y, g, p, prm0)

    A = torch.tensor(im.nonuniform_matrix(N, L, R, theta, delta, frames, T))
    yt = torch.tensor(y)
    planes = [{c: torch.tensor(v).requires_grad_(True) for c, v in d.items()} for d in prm0["planes"]]
    avec = [torch.tensor(a).requires_grad_(True) for a in prm0["a"]]
    params = [P[c] for P in planes for c in kp.PLANES] + avec

    def loss(k):
        V = im.kplanes_volume(planes, avec, N, Nf, T)
        return im.volume_loss(V, A, yt, p.tv_xy, p.tv_t, p.tv_eps)

    tr_t = im.run_adam(params, loss, p.iters, p.lr, (p.beta1, p.beta2), p.eps)
    assert np.max(np.abs(tr_o - tr_t) / np.abs(tr_t)) < TOL
    for s in range(2):
        for c in kp.PLANES:
            assert _rel(prm_o["planes"][s][c], planes[s][c].detach().numpy()) < TOL, (s, c)
        assert _rel(prm_o["a"][s], avec[s].detach().numpy()) < TOL
    assert tr_o[-1] < tr_o[0]


def test_kplanes_independent_render_matches_oracle():
    """The torch K-Planes volume used above equals the oracle's render (so the
    loop comparison is not comparing two different models)."""
    rng = np.random.default_rng(15)
    N, Nf, T = 8, 3, 2
    prm = kp.init_params(N, Nf, T, rng, F=3, scales=2, spread=0.5)
    planes = [{c: torch.tensor(v) for c, v in d.items()} for d in prm["planes"]]
    avec = [torch.tensor(a) for a in prm["a"]]
    V_t = im.kplanes_volume(planes, avec, N, Nf, T).numpy()
    assert _rel(kp.render(prm, N, Nf, T), V_t) < 1e-13


def test_independent_operators_match_the_oracle_operators():
    """The dense torch-side operators equal the oracle's operators on random
    inputs (one call each), so a failure above points at the loop."""
    rng = np.random.default_rng(16)
    N, L, R, T = 8, 2, 8, 2
    theta, delta, frames = [0.3, 1.2, 2.4], [-1.0, 0.4, 1.7], [0, 1, 1]
    g = make_geometry(N, L, R, theta, delta, frames, T=T)
    V = _rand_c(rng, (T, N, N, 3))
    A = im.nonuniform_matrix(N, L, R, theta, delta, frames, T)
    assert _rel(A @ V.reshape(-1), oracle.forward(V, g).reshape(-1)) < 1e-12
    for b in range(3):
        P = im.projection_matrix(N, 3, theta[b], delta)
        assert _rel((P @ V[frames[b]].reshape(-1)).reshape(N, N), pj.project(V[frames[b]], pj.shifts(g, b))) < 1e-12
        assert np.array_equal(im.blade_support(N, theta[b], 4, R), pj.blade_mask(N, theta[b], 4, R))
