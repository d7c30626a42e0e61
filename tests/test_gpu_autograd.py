"""torch.autograd through the operator: backward = prop_adjoint.

* 64^2: the gradient of the k-space loss sum|A V - y|^2 taken by autograd
  equals the oracle's 2 A^H (A V - y) (<= 1e-4 relative L2).
* 384^2, 64 bins, 32 blades x 32 x 384 (the differentiation workload):
  central finite differences with h = 1e-3 along 64 random unit directions,
  each error measured against the largest possible directional derivative
  ||grad|| (random directions in ~10^7 dimensions make single derivatives
  tiny), and the 64 derivatives compared as a vector.
  The loss is quadratic in V, so the central difference is exact in exact
  arithmetic; the volume is scaled to 1e-3 so that FP32 rounding of the
  forward stays well below the h-sized signal, and the loss is summed in FP64.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import rel, geometry, random_case

pytestmark = pytest.mark.gpu


def _loss(plan, V, y):
    from paper_2311_13177_gb300 import prop_apply
    r = prop_apply(V, plan) - y
    return (r.real.double() ** 2 + r.imag.double() ** 2).sum()


def test_autograd_gradient_matches_oracle_adjoint():
    from paper_2311_13177_gb300 import Plan
    c = random_case(64, 8, 6, 8, 64, T=2, seed=12)
    g = geometry(64, 8, 64, c["theta"], c["delta"], c["blade_frame"], 2)
    plan = Plan(64, 8, 64, c["theta"], c["delta"], c["blade_frame"], 2)
    V = torch.from_numpy(c["V"]).cuda().requires_grad_(True)
    y = torch.from_numpy(c["y"]).cuda()
    loss = _loss(plan, V, y)
    loss.backward()
    Vd = c["V"].astype(np.complex128)
    ref = 2 * oracle.adjoint(oracle.forward(Vd, g) - c["y"].astype(np.complex128), g)
    assert rel(V.grad.cpu().numpy(), ref) < 1e-4
    plan.destroy()


def test_finite_differences_at_384():
    from paper_2311_13177_gb300 import Plan
    w = synth.WORKLOADS["diff"]
    p = synth.make_problem(w)
    plan = Plan(w.N, w.L, w.R, p["theta"], p["delta"], p["blade_frame"], w.T)
    gen = torch.Generator(device="cuda").manual_seed(0)
    shape = plan.vol_shape
    V = (torch.randn(shape, generator=gen, device="cuda", dtype=torch.complex64) * 1e-3).requires_grad_(True)
    y = torch.from_numpy(p["y"]).cuda() * 1e-3
    loss = _loss(plan, V, y)
    loss.backward()
    G = V.grad.detach()
    gnorm = torch.linalg.vector_norm(G).item()
    h = 1e-3
    fds, ans = [], []
    with torch.no_grad():
        for _ in range(64):
            D = torch.randn(shape, generator=gen, device="cuda", dtype=torch.complex64)
            D /= torch.linalg.vector_norm(D)
            lp = _loss(plan, V + h * D, y).item()
            lm = _loss(plan, V - h * D, y).item()
            fd = (lp - lm) / (2 * h)
            an = (G.real.double() * D.real.double() + G.imag.double() * D.imag.double()).sum().item()
            fds.append(fd)
            ans.append(an)
    plan.destroy()
    fds, ans = np.array(fds), np.array(ans)
    # |<G, D>| <= ||G|| for unit D: scale each error by the largest possible
    # directional derivative, and compare the 64 derivatives as a vector.
    assert np.max(np.abs(fds - ans)) < 1e-5 * gnorm
    assert np.linalg.norm(fds - ans) < 5e-3 * np.linalg.norm(ans)
