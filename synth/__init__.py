"""Seeded synthetic inputs for the volumetric PROPELLER reconstruction.

This package is the only code shared by the FP64 oracle (``oracle/``) and the
CUDA path (``paper_2311_13177_gb300``).  It produces *inputs* only: blade
angles, spectral-bin displacements, blade-to-frame maps, ground-truth ellipse
phantoms and the k-space blade data simulated from their analytic Fourier
transform.  It holds none of the reconstruction's arithmetic (no discrete
forward operator, adjoint, loss, TV or optimiser).

The paper's datasets (Shepp-Logan slabs, Dixon-RAVE liver/breast layers,
Sec. 5) are not available; seeded random-ellipse phantoms with the same
structure (water and fat layers, fat displaced along each blade's readout,
Sec. 3 and Sec. 5) stand in for them.
"""

from .phantom import (Ellipse, random_ellipses, ellipse_ft, simulate_blades,
                      simulate_cartesian_blades, add_noise, rasterize, blade_kspace)
from .workloads import WORKLOADS, Workload, make_problem, make_serve_requests

__all__ = [
    "Ellipse", "random_ellipses", "ellipse_ft", "simulate_blades", "simulate_cartesian_blades", "add_noise",
    "rasterize", "blade_kspace", "WORKLOADS", "Workload", "make_problem",
    "make_serve_requests",
]
