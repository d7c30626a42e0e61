"""The allocation-free TV entry point (prop_tv_grad_static) against the plan-based one.

prop_tv_grad_static serves callers that cannot allocate device memory (for
example code running inside a host framework's memory arena, or a real-time
loop under a no-allocation rule): its reduction scratch is a static device
array instead of plan memory.  Its output must equal what prop_loss_grad
computes for the same TV terms: with blade data y = A V the data term of
prop_loss_grad is exactly zero (same kernels, same order), so its loss and
gradient are the TV loss and gradient alone.  Two calls in a row with
different volumes check that the shared scratch carries nothing over.
This file is collected last so that a failure here stops a run only after
every other test has run.
"""
import numpy as np
import pytest
import torch

from helpers import rel, random_case

pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-4   # gradient tolerance of the other gradient tests
TOL_LOSS = 1e-5


def test_static_scratch_tv_matches_plan_entry_point_twice():
    from paper_2311_13177_gb300 import Plan, ReconParams
    from paper_2311_13177_gb300.binding import prop_tv_grad_static
    c = random_case(48, 6, 5, 8, 48, T=3, seed=44)
    plan = Plan(48, 8, 48, c["theta"], c["delta"], c["blade_frame"], 3)
    dev = torch.device("cuda")
    params = ReconParams(tv_xy=3e-2, tv_t=2e-2, tv_eps=5e-2)
    rng = np.random.default_rng(45)
    grad = torch.empty(plan.vol_shape, dtype=torch.complex64, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    for call in range(2):
        V = torch.from_numpy((c["V"] * np.float32(0.1 * (call + 1)) +
                              rng.standard_normal(plan.vol_shape).astype(np.float32) * 0.01)
                             .astype(np.complex64)).to(dev)
        y = plan.forward(V)
        ref_loss, ref_grad = plan.loss_grad(y, params, V)
        prop_tv_grad_static(V, params.tv_xy, params.tv_t, params.tv_eps, grad, loss)
        torch.cuda.synchronize()
        assert abs(float(loss.item()) - ref_loss) <= TOL_LOSS * abs(ref_loss), (call, float(loss.item()), ref_loss)
        assert rel(grad.cpu().numpy(), ref_grad.cpu().numpy()) < TOL_GRAD, call
    plan.destroy()


def test_static_scratch_rejects_oversized_problem():
    from paper_2311_13177_gb300._lib import PropError
    from paper_2311_13177_gb300.binding import prop_tv_grad_static
    dev = torch.device("cuda")
    V = torch.zeros((65, 256, 256, 1), dtype=torch.complex64, device=dev)   # 16640 rows > 16384
    g = torch.empty_like(V)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(PropError, match="static scratch limit"):
        prop_tv_grad_static(V, 1e-3, 1e-2, 1e-3, g, loss)
