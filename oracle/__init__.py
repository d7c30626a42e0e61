"""FP64 CPU oracle for volumetric PROPELLER reconstruction -- TEST INFRASTRUCTURE.

This package is the plain, slow, obviously-correct statement of what the GPU
path computes.  It exists to check the CUDA library: only the test-suite,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import or
run it.  The product path (``paper_2311_13177_gb300``) never imports it, and
it imports nothing from the product path; the two share only the seeded input
generators in ``synth/``.

Contents
  geometry  sample positions k of every blade sample (Sec. 4.2 "Blur", and
            the non-uniform blade lines of Sec. 7 "Limitations")
  ndft      the exact volumetric forward operator, a direct non-uniform DFT
            with the spectral displacement phase (Sec. 3 Eq. 1-2, Sec. 4.2),
            and its explicit adjoint
  recon     data-consistency loss, smoothed TV in x-y and in time, Adam, and
            the full-batch reconstruction loop (Sec. 4.3), plus the phi = 0
            render, the fat/water split and PSNR (Sec. 4.3, Sec. 6)
  kplanes   the dynamic K-Planes volume model (Sec. 4.1, Eq. 3): six planes
            of feature vectors, bilinear lookups, Hadamard product, weighting
            vector, two scales; rendering on the volume grid and the
            parameter gradients
  projection  the paper's own forward model (Sec. 4.2): interpolated
            projection at the blade's tilt, centred DFT and blade mask; its
            adjoint; the image- plus k-space loss with TV (x-y, spectral,
            time) and L1, and Adam over the blades in turn (Sec. 4.3)

Every function is pinned by a ``-m "not gpu"`` test against something other
than itself (library special cases, closed forms, invariants, brute force,
torch.optim.Adam).  The three reconstruction loops (``recon.reconstruct``,
``projection.reconstruct``, ``kplanes.reconstruct``) are pinned as wholes
against independent torch statements of the same problems driven by
torch.optim.Adam (iterates and loss traces to 1e-12).
"""
from .geometry import Geometry, make_geometry, sample_coords, phase_table
from .ndft import forward, adjoint, forward_at, adjoint_at
from .recon import (ReconParams, data_loss, tv_xy, tv_t, loss_and_grad,
                    adam_step, reconstruct, render, psnr)
from . import projection
from . import kplanes

__all__ = [
    "Geometry", "make_geometry", "sample_coords", "phase_table", "forward", "adjoint",
    "forward_at", "adjoint_at", "ReconParams", "data_loss", "tv_xy", "tv_t",
    "loss_and_grad", "adam_step", "reconstruct", "render", "psnr", "projection", "kplanes",
]
