"""GPU K-Planes volume model (Sec. 4.1, Eq. 3) through the C ABI against the
FP64 oracle: rendering, the parameter gradients of a given grad V, and a
short reconstruction through the non-uniform data term."""
import numpy as np
import pytest
import torch

import oracle
from oracle import kplanes as kp
from helpers import rel, geometry, random_case, kplanes_pack, kplanes_unpack

pytestmark = pytest.mark.gpu


def _setup(N=16, Nf=3, B=4, L=4, R=16, T=2, F=4, S=2, seed=40):
    from paper_2311_13177_gb300 import Plan
    c = random_case(N, Nf, B, L, R, T, seed=seed)
    plan = Plan(N, L, R, c["theta"], c["delta"], c["blade_frame"], T, kb_width=8)
    prm = kp.init_params(N, Nf, T, np.random.default_rng(seed + 1), F=F, scales=S, spread=0.3)
    return c, plan, prm


def test_param_count_matches_layout():
    c, plan, prm = _setup()
    assert plan.kplanes_param_count(4, 2) == kplanes_pack(prm).size
    plan.destroy()


def test_render_matches_oracle():
    c, plan, prm = _setup()
    flat = torch.from_numpy(kplanes_pack(prm).astype(np.complex64)).cuda()
    V = plan.kplanes_render(flat, 4, 2).cpu().numpy()
    plan.destroy()
    ref = kp.render(prm, 16, 3, 2)
    assert rel(V, ref) < 1e-5, rel(V, ref)


def test_parameter_gradients_match_oracle():
    c, plan, prm = _setup()
    rng = np.random.default_rng(41)
    gV = (rng.standard_normal((2, 16, 16, 3)) + 1j * rng.standard_normal((2, 16, 16, 3))).astype(np.complex64)
    flat = torch.from_numpy(kplanes_pack(prm).astype(np.complex64)).cuda()
    G = plan.kplanes_vjp(flat, torch.from_numpy(gV).cuda(), 4, 2).cpu().numpy()
    plan.destroy()
    ref = kplanes_pack(kp.vjp(prm, gV.astype(np.complex128), 16, 3, 2))
    assert rel(G, ref) < 1e-4, rel(G, ref)


def test_reconstruction_matches_oracle():
    """5 Adam iterations on the model's parameters through the non-uniform
    data term with TV in x-y and time (two frames)."""
    from paper_2311_13177_gb300 import ReconParams
    c, plan, prm = _setup()
    g = geometry(16, 4, 16, c["theta"], c["delta"], c["blade_frame"], 2)
    y = (0.1 * c["y"]).astype(np.complex64)
    pg = ReconParams(iters=5, lr=1e-2, tv_xy=1e-3, tv_t=1e-2)
    po = oracle.ReconParams(iters=5, lr=1e-2, tv_xy=1e-3, tv_t=1e-2)
    flat = torch.from_numpy(kplanes_pack(prm).astype(np.complex64)).cuda()
    flat, tr = plan.kplanes_reconstruct(torch.from_numpy(y).cuda(), pg, flat, 4, 2)
    V = plan.kplanes_render(flat, 4, 2).cpu().numpy()
    plan.destroy()
    prm_o, tro = kp.reconstruct(y.astype(np.complex128), g, po, prm)
    Vo = kp.render(prm_o, 16, 3, 2)
    assert rel(V, Vo) < 1e-3, rel(V, Vo)
    assert np.max(np.abs(tr - tro) / np.abs(tro)) < 1e-4
    assert rel(kplanes_unpack(flat.cpu().numpy(), prm)["a"][0], prm_o["a"][0]) < 1e-3


def _setup_paper(seed=50):
    """The paper's settings (F = 8 features, two scales) on a mid-size
    dynamic grid: 64^2, 16 bins, 8 frames, 8 golden-angle blades of 8 x 64."""
    from paper_2311_13177_gb300 import Plan
    N, Nf, B, L, R, T = 64, 16, 8, 8, 64, 8
    c = random_case(N, Nf, B, L, R, T, seed=seed)
    c["theta"] = np.deg2rad((np.arange(B) * 111.246) % 180.0)
    plan = Plan(N, L, R, c["theta"], c["delta"], c["blade_frame"], T, kb_width=8)
    prm = kp.init_params(N, Nf, T, np.random.default_rng(seed + 1), F=8, scales=2, spread=0.3)
    return c, plan, prm, (N, Nf, B, L, R, T)


def test_paper_settings_render_and_gradients_match_oracle():
    c, plan, prm, (N, Nf, B, L, R, T) = _setup_paper()
    flat = torch.from_numpy(kplanes_pack(prm).astype(np.complex64)).cuda()
    V = plan.kplanes_render(flat, 8, 2).cpu().numpy()
    assert rel(V, kp.render(prm, N, Nf, T)) < 1e-5
    rng = np.random.default_rng(51)
    gV = (rng.standard_normal((T, N, N, Nf)) + 1j * rng.standard_normal((T, N, N, Nf))).astype(np.complex64)
    G = plan.kplanes_vjp(flat, torch.from_numpy(gV).cuda(), 8, 2).cpu().numpy()
    plan.destroy()
    ref = kplanes_pack(kp.vjp(prm, gV.astype(np.complex128), N, Nf, T))
    assert rel(G, ref) < 1e-4, rel(G, ref)


def test_paper_settings_reconstruction_matches_oracle():
    """3 Adam iterations of the F = 8, two-scale model through the
    non-uniform data term with TV in x-y and time (8 frames)."""
    from paper_2311_13177_gb300 import ReconParams
    c, plan, prm, (N, Nf, B, L, R, T) = _setup_paper(seed=52)
    g = geometry(N, L, R, c["theta"], c["delta"], c["blade_frame"], T)
    y = (0.05 * c["y"]).astype(np.complex64)
    pg = ReconParams(iters=3, lr=1e-2, tv_xy=1e-3, tv_t=1e-2)
    po = oracle.ReconParams(iters=3, lr=1e-2, tv_xy=1e-3, tv_t=1e-2)
    flat = torch.from_numpy(kplanes_pack(prm).astype(np.complex64)).cuda()
    flat, tr = plan.kplanes_reconstruct(torch.from_numpy(y).cuda(), pg, flat, 8, 2)
    V = plan.kplanes_render(flat, 8, 2).cpu().numpy()
    plan.destroy()
    prm_o, tro = kp.reconstruct(y.astype(np.complex128), g, po, prm)
    assert rel(V, kp.render(prm_o, N, Nf, T)) < 1e-3
    assert np.max(np.abs(tr - tro) / np.abs(tro)) < 1e-4

