"""Blade sample geometry of the volumetric PROPELLER model (oracle, FP64).

Test infrastructure: see the package docstring.

Readings of the paper (which leaves these conventions open):
  * Sec. 4.2 "Blur" masks the image's DFT by the blade support; Sec. 7
    "Limitations" states that real blades are blade-aligned lines needing a
    non-uniform DFT.  Here blade b is the rotated Cartesian patch
    k = k_r d_b + k_p d_b^perp, d_b = (cos th_b, sin th_b),
    d_b^perp = (-sin th_b, cos th_b), k_r = (j - R/2)/N, k_p = (l - L/2)/N,
    for line l < L and readout sample j < R (cycles per pixel).
  * Sample order: m = (b L + l) R + j.
  * Sec. 3 (Eq. 2 and the text after it): a material displaced by Delta_f
    along the blade picks up exp(-2 pi i k.(Delta_f d_b)) = exp(-2 pi i k_r
    Delta_f), because k.d_b = k_r.  The phase table P[m, f] holds that factor.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Geometry:
    """Problem geometry.

    N: image size (x_i in {-N/2..N/2-1}); L, R: lines and readout samples per
    blade; theta [B] (rad); delta [Nf] spectral displacements (pixels);
    blade_frame [B] frame of each blade; T: number of frames.
    """
    N: int
    L: int
    R: int
    theta: np.ndarray
    delta: np.ndarray
    blade_frame: np.ndarray
    T: int = 1

    @property
    def B(self) -> int:
        return len(self.theta)

    @property
    def Nf(self) -> int:
        return len(self.delta)

    @property
    def M(self) -> int:
        return self.B * self.L * self.R

    @property
    def scale(self) -> float:
        """Operator scale s = 1/N (orthonormal 2-D DFT when Delta = 0, theta = 0, L = N)."""
        return 1.0 / self.N

    def pixel_coords(self) -> np.ndarray:
        return np.arange(self.N, dtype=np.float64) - self.N // 2


def make_geometry(N, L, R, theta, delta, blade_frame=None, T=1) -> Geometry:
    theta = np.asarray(theta, dtype=np.float64)
    delta = np.asarray(delta, dtype=np.float64)
    if blade_frame is None:
        blade_frame = np.zeros(len(theta), dtype=np.int64)
    return Geometry(int(N), int(L), int(R), theta, delta,
                    np.asarray(blade_frame, dtype=np.int64), int(T))


def sample_coords(g: Geometry):
    """k1, k2, k_r of every sample, each a flat [M] float64 array (order m = (b L + l) R + j)."""
    j = np.arange(g.R, dtype=np.float64)
    l = np.arange(g.L, dtype=np.float64)
    kr = (j - g.R / 2.0) / g.N
    kp = (l - g.L / 2.0) / g.N
    k1 = np.empty((g.B, g.L, g.R))
    k2 = np.empty((g.B, g.L, g.R))
    for b, th in enumerate(g.theta):
        d = (np.cos(th), np.sin(th))
        dp = (-np.sin(th), np.cos(th))
        k1[b] = kr[None, :] * d[0] + kp[:, None] * dp[0]
        k2[b] = kr[None, :] * d[1] + kp[:, None] * dp[1]
    KR = np.broadcast_to(kr, (g.B, g.L, g.R))
    return k1.reshape(-1), k2.reshape(-1), np.array(KR).reshape(-1)


def phase_table(kr: np.ndarray, delta: np.ndarray) -> np.ndarray:
    """P[m, f] = exp(-2 pi i k_r(m) Delta_f), complex128 [M, Nf]."""
    return np.exp(-2j * np.pi * np.outer(kr, delta))


def sample_frame(g: Geometry) -> np.ndarray:
    """Frame index of every sample, [M]."""
    return np.repeat(np.asarray(g.blade_frame, dtype=np.int64), g.L * g.R)
