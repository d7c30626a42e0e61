"""Named workloads: shapes, sizes and seeds of the synthetic problems.

Each workload mirrors one of the paper's acquisition settings (Sec. 5):
water/fat phantoms imaged by rotating PROPELLER blades, static or dynamic.
Spectral bins are an inclusive linspace over [delta_lo, delta_hi] pixels;
uniform blade angles are theta_b = pi b / B, golden-angle ones
theta_b = (b * 180 (sqrt 5 - 1)/2 degrees) mod 180; blade b belongs to frame
t(b) = floor(b T / B).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

from .phantom import random_ellipses, simulate_blades, add_noise, rasterize


@dataclass(frozen=True)
class Workload:
    name: str
    N: int                 # matrix size (square image, even)
    Nf: int                # spectral bins
    delta_lo: float        # displacement of bin 0 (pixels along readout)
    delta_hi: float        # displacement of bin Nf-1
    B: int                 # blades
    L: int                 # lines per blade
    R: int                 # readout samples per line
    T: int = 1             # frames (1 = static)
    angles: str = "uniform"
    n_ellipses: int = 20
    fat_shift: float = 1.7
    rel_sigma: float = 1e-3
    iters: int = 100
    lr: float = 1e-2
    tv_xy: float = 1e-3
    tv_t: float = 0.0
    tv_eps: float = 1e-3
    seed: int = 0
    motion: tuple = field(default=None)   # (ellipse index, amplitude px, period frames)

    @property
    def M(self) -> int:
        return self.B * self.L * self.R

    def voxels(self) -> int:
        return self.T * self.N * self.N * self.Nf


GOLDEN_DEG = 180.0 * (math.sqrt(5.0) - 1.0) / 2.0   # 111.246...


def blade_angles(w: Workload) -> np.ndarray:
    b = np.arange(w.B, dtype=np.float64)
    if w.angles == "uniform":
        return math.pi * b / w.B
    if w.angles == "golden":
        return np.deg2rad(np.mod(b * GOLDEN_DEG, 180.0))
    raise ValueError(w.angles)


def bin_displacements(w: Workload) -> np.ndarray:
    if w.Nf == 1:
        return np.array([w.delta_lo], dtype=np.float64)
    return np.linspace(w.delta_lo, w.delta_hi, w.Nf, dtype=np.float64)


def blade_frames(w: Workload) -> np.ndarray:
    return (np.arange(w.B, dtype=np.int64) * w.T // w.B).astype(np.int32)


WORKLOADS = {
    # 32x32, 6 ellipses, Nf=8 over [-2, 2], 5 blades at 0..144 deg, 8 lines x 32.
    "tiny": Workload("tiny", N=32, Nf=8, delta_lo=-2.0, delta_hi=2.0, B=5, L=8, R=32,
                     n_ellipses=6, iters=20, lr=1e-2, tv_xy=1e-3),
    # Small dynamic series the oracle runs in full: 32^2, Nf 4, 8 golden-angle
    # blades over 4 frames (2 per frame), moving ellipse, temporal TV.
    "dyn_small": Workload("dyn_small", N=32, Nf=4, delta_lo=-2.0, delta_hi=2.0, B=8, L=8, R=32,
                          T=4, angles="golden", n_ellipses=6, iters=20, lr=1e-2, tv_xy=1e-3,
                          tv_t=1e-2, motion=(0, 3.0, 4.0)),
    # Reduced static problem the oracle runs in full: 64^2, Nf 8, 8 blades.
    "small64": Workload("small64", N=64, Nf=8, delta_lo=-4.0, delta_hi=4.0, B=8, L=16, R=64,
                        n_ellipses=10, iters=100, lr=1e-2, tv_xy=1e-3),
    # Static abdomen-like problem: 256^2, Nf 32 over [-4, 4], 16 blades x 24 x 256.
    "static": Workload("static", N=256, Nf=32, delta_lo=-4.0, delta_hi=4.0, B=16, L=24, R=256,
                       n_ellipses=20, iters=500, lr=1e-2, tv_xy=1e-3),
    # Dynamic series: 192^2, Nf 16, 64 golden-angle blades x 16 x 192, 32 frames.
    "dynamic": Workload("dynamic", N=192, Nf=16, delta_lo=-4.0, delta_hi=4.0, B=64, L=16, R=192,
                        T=32, angles="golden", n_ellipses=12, iters=800, lr=1e-2,
                        tv_xy=1e-3, tv_t=1e-2, motion=(0, 8.0, 16.0)),
    # Differentiation problem: 384^2, Nf 64, 32 blades x 32 x 384.
    "diff": Workload("diff", N=384, Nf=64, delta_lo=-4.0, delta_hi=4.0, B=32, L=32, R=384,
                     n_ellipses=20, iters=0),
}


def make_problem(w: Workload, with_truth: bool = False) -> dict:
    """Geometry and noisy blade data for workload ``w`` (seeded).

    Returns theta [B] f64, delta [Nf] f64, blade_frame [B] i32 and y [B, L, R]
    complex64 (the stored measurement; consumers needing FP64 upcast it
    exactly).  With ``with_truth`` also the water/fat rasters per frame.
    """
    rng = np.random.default_rng(w.seed)
    ell = random_ellipses(rng, w.n_ellipses, w.N, liver=w.motion is not None)
    theta = blade_angles(w)
    delta = bin_displacements(w)
    frames = blade_frames(w)
    y = simulate_blades(ell, w.N, w.L, w.R, theta, w.fat_shift, frames, w.motion)
    y = add_noise(y, w.rel_sigma, rng).astype(np.complex64)
    out = dict(workload=w, theta=theta, delta=delta, blade_frame=frames, y=y,
               ellipses=ell)
    if with_truth:
        layers = [rasterize(ell, w.N, 4, t, w.motion) for t in range(w.T)]
        out["water"] = np.stack([a for a, _ in layers])
        out["fat"] = np.stack([b for _, b in layers])
    return out


def make_serve_requests(n: int = 256, seed: int = 0, iters: int = 300):
    """Mixed request stream: N, blades, Nf and static/dynamic drawn per request.

    N in {128, 192, 256, 384}, blades in {8, 16, 24, 32}, lines = N/8,
    Nf in {8, 16, 32, 64}, static or dynamic (T = 16).
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        N = int(rng.choice([128, 192, 256, 384]))
        B = int(rng.choice([8, 16, 24, 32]))
        Nf = int(rng.choice([8, 16, 32, 64]))
        dyn = bool(rng.integers(0, 2))
        out.append(Workload(f"req{i}", N=N, Nf=Nf, delta_lo=-4.0, delta_hi=4.0, B=B,
                            L=N // 8, R=N, T=16 if dyn else 1,
                            angles="golden" if dyn else "uniform", n_ellipses=8,
                            iters=iters, tv_t=1e-2 if dyn else 0.0,
                            motion=(0, 8.0, 16.0) if dyn else None, seed=1000 + i))
    return out
