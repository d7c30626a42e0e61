"""Multi-problem launches (prop_reconstruct_batch, and the request server's
batched iterations): several reconstructions of one kernel class (same 2N,
bin stride, kernel width) advanced together, each stage one launch for all
of them, give every problem's volume bit for bit as its own
prop_reconstruct, with different blade counts, lines, frames, angles, bins,
data and iteration counts in the batch."""
import numpy as np
import pytest
import torch

import oracle
from helpers import rel, geometry, random_case

pytestmark = pytest.mark.gpu


def _case(N, Nf, B, L, R, T, seed, kbw=6, row_kernel=0):
    from paper_2311_13177_gb300 import Plan
    c = random_case(N, Nf, B, L, R, T, seed=seed)
    plan = Plan(N, L, R, c["theta"], c["delta"], c["blade_frame"], T, kb_width=kbw, row_kernel=row_kernel)
    return c, plan


def _params(iters, tv_t=0.0):
    from paper_2311_13177_gb300 import ReconParams
    return ReconParams(iters=iters, lr=1e-2, tv_xy=1e-3, tv_t=tv_t)


@pytest.mark.parametrize("kbw", [6, 8])
def test_batch_equals_lone_reconstructions(kbw):
    from paper_2311_13177_gb300 import prop_reconstruct_batch
    # one kernel class: 2N = 96, 8 bins (stride 8); everything else differs
    specs = [(48, 8, 5, 6, 48, 1, 1, 9), (48, 7, 3, 8, 40, 2, 2, 7), (48, 8, 7, 4, 48, 3, 3, 11)]
    cases, plans, params = [], [], []
    for N, Nf, B, L, R, T, seed, iters in specs:
        c, pl = _case(N, Nf, B, L, R, T, seed, kbw)
        cases.append(c)
        plans.append(pl)
        params.append(_params(iters, tv_t=1e-2 if T > 1 else 0.0))
    ys = [torch.from_numpy(c["y"]).cuda() for c in cases]
    Vb, trb = prop_reconstruct_batch(plans, ys, params)
    for c, pl, y, q, V, tr in zip(cases, plans, ys, params, Vb, trb):
        Vl, trl = pl.reconstruct(y, q)
        assert torch.equal(V, Vl)
        assert np.max(np.abs(tr - trl) / np.abs(trl)) < 1e-12
    for pl in plans:
        pl.destroy()


def test_batch_matches_oracle_and_mixes_row_kernels():
    """A member that runs the warp-specialised row kernel is launched on its
    own inside the batch; the result is still its lone reconstruction, and
    the batched reconstruction meets the oracle bar."""
    from paper_2311_13177_gb300 import prop_reconstruct_batch
    c1, p1 = _case(32, 16, 4, 6, 32, 2, 21, kbw=8, row_kernel=2)
    c2, p2 = _case(32, 16, 6, 4, 32, 1, 22, kbw=8, row_kernel=1)
    q1, q2 = _params(8, tv_t=1e-2), _params(6)
    ys = [torch.from_numpy(c["y"]).cuda() for c in (c1, c2)]
    (V1, V2), (t1, t2) = prop_reconstruct_batch([p1, p2], ys, [q1, q2])
    assert torch.equal(V1, p1.reconstruct(ys[0], q1)[0])
    assert torch.equal(V2, p2.reconstruct(ys[1], q2)[0])
    g = geometry(32, 6, 32, c1["theta"], c1["delta"], c1["blade_frame"], 2)
    Vo, tro = oracle.reconstruct(c1["y"].astype(np.complex128), g,
                                 oracle.ReconParams(iters=8, lr=1e-2, tv_xy=1e-3, tv_t=1e-2))
    assert rel(V1.cpu().numpy(), Vo) < 1e-3
    assert np.max(np.abs(t1 - tro) / np.abs(tro)) < 1e-4
    p1.destroy()
    p2.destroy()


def test_batch_rejects_incompatible_plans():
    from paper_2311_13177_gb300 import prop_reconstruct_batch
    from paper_2311_13177_gb300._lib import PropError
    c1, p1 = _case(32, 8, 3, 4, 32, 1, 1)
    c2, p2 = _case(48, 8, 3, 4, 48, 1, 2)     # different 2N
    c3, p3 = _case(32, 16, 3, 4, 32, 1, 3)    # different bin stride
    ys = [torch.from_numpy(c["y"]).cuda() for c in (c1, c2, c3)]
    for other, y in ((p2, ys[1]), (p3, ys[2])):
        with pytest.raises(PropError):
            prop_reconstruct_batch([p1, other], [ys[0], y], [_params(2), _params(2)])
    with pytest.raises(PropError):
        prop_reconstruct_batch([p1, p1], [ys[0], ys[0]], [_params(2), _params(2)])
    for p in (p1, p2, p3):
        p.destroy()
