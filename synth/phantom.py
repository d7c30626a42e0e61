"""Seeded ellipse phantoms and their k-space PROPELLER blade data.

The measurement model follows the paper's physics (Sec. 3, Eq. 1-2): each
material is imaged through the Fourier transform of the object, and a
material with off-resonance displacement ``delta`` (pixels) is translated by
``delta`` along the blade's readout direction d_b, i.e. its k-space signal is
multiplied by exp(-2 pi i k_r delta) with k_r = k . d_b.  Water sits at
delta = 0 and fat at a fixed, continuous ``fat_shift`` (which is deliberately
not one of the volume's spectral bins).

Conventions (shared with every consumer of these inputs):
  * pixel coordinates x_i in {-N/2, ..., N/2-1}; continuous objects live in
    the same pixel units, one pixel = unit area;
  * blade b has angle theta_b, readout direction d_b = (cos, sin) and phase
    direction d_b^perp = (-sin, cos);
  * sample (b, l, j) sits at k = k_r d_b + k_p d_b^perp with
    k_r = (j - R/2)/N and k_p = (l - L/2)/N (cycles per pixel);
  * blade data carry the scale s = 1/N of the discrete operator they will be
    compared against, so that y ~ s * FT(object).

Nothing here evaluates the discrete operator on a voxel grid; the data come
from the closed-form Fourier transform of ellipse indicators.
"""
from __future__ import annotations

from dataclasses import dataclass, replace
import math

import numpy as np
from scipy.special import j1


@dataclass(frozen=True)
class Ellipse:
    """One ellipse of the phantom.

    center: (c1, c2) in pixels; axes: semi-axes (a, b) in pixels;
    angle: rotation of the a-axis from x1 (radians); rho: complex intensity;
    fat: fat fraction in [0, 1] (the rest is water).
    """
    center: tuple
    axes: tuple
    angle: float
    rho: complex
    fat: float


def random_ellipses(rng: np.random.Generator, n: int, N: int,
                    liver: bool = False) -> list:
    """Draw ``n`` random ellipses inside an N x N field of view.

    Centres U(-0.35N, 0.35N), semi-axes U(0.05N, 0.3N), rotation U(0, pi),
    magnitude U[0.2, 1], phase U[0, 2 pi), fat fraction U[0, 1].
    With ``liver=True`` the first ellipse is a large, mostly-water ellipse
    near the centre (the organ that moves in the dynamic series).
    """
    out = []
    for i in range(n):
        c = rng.uniform(-0.35 * N, 0.35 * N, size=2)
        ax = rng.uniform(0.05 * N, 0.3 * N, size=2)
        ang = rng.uniform(0.0, math.pi)
        mag = rng.uniform(0.2, 1.0)
        ph = rng.uniform(0.0, 2 * math.pi)
        ff = rng.uniform(0.0, 1.0)
        if liver and i == 0:
            c = rng.uniform(-0.05 * N, 0.05 * N, size=2)
            ax = np.array([0.22 * N, 0.15 * N]) * rng.uniform(0.9, 1.1, size=2)
            ff = 0.1 * ff
        out.append(Ellipse((float(c[0]), float(c[1])), (float(ax[0]), float(ax[1])),
                           float(ang), complex(mag * np.exp(1j * ph)), float(ff)))
    return out


def moved(e: Ellipse, dx: float) -> Ellipse:
    return replace(e, center=(e.center[0] + dx, e.center[1]))


def ellipse_ft(k1: np.ndarray, k2: np.ndarray, e: Ellipse) -> np.ndarray:
    """Closed-form continuous Fourier transform of the unit ellipse indicator.

    FT(k) = a b J1(2 pi kappa)/kappa * exp(-2 pi i k.c),
    kappa = |diag(a, b) R(angle)^T k|; the kappa -> 0 limit is pi a b.
    """
    a, b = e.axes
    ca, sa = math.cos(e.angle), math.sin(e.angle)
    q1 = a * (ca * k1 + sa * k2)
    q2 = b * (-sa * k1 + ca * k2)
    kap = np.sqrt(q1 * q1 + q2 * q2)
    small = kap < 1e-12
    kap_safe = np.where(small, 1.0, kap)
    amp = np.where(small, math.pi * a * b, a * b * j1(2 * math.pi * kap_safe) / kap_safe)
    return amp * np.exp(-2j * math.pi * (k1 * e.center[0] + k2 * e.center[1]))


def blade_kspace(N: int, L: int, R: int, theta: np.ndarray):
    """Sample positions of every blade: (k1, k2, kr), each [B, L, R] float64."""
    theta = np.asarray(theta, dtype=np.float64)
    kr = (np.arange(R, dtype=np.float64) - R / 2) / N
    kp = (np.arange(L, dtype=np.float64) - L / 2) / N
    c = np.cos(theta)[:, None, None]
    s = np.sin(theta)[:, None, None]
    KR = np.broadcast_to(kr[None, None, :], (len(theta), L, R))
    KP = np.broadcast_to(kp[None, :, None], (len(theta), L, R))
    k1 = KR * c - KP * s
    k2 = KR * s + KP * c
    return k1, k2, np.ascontiguousarray(KR)


def simulate_blades(ellipses: list, N: int, L: int, R: int, theta: np.ndarray,
                    fat_shift: float, blade_frame=None, motion=None) -> np.ndarray:
    """Clean blade data y[b, l, j] (complex128) from the analytic ellipse FT.

    ``motion`` = (index, amplitude_px, period_frames) moves that ellipse along
    x1 as amplitude * sin(2 pi t / period) in frame t = blade_frame[b].
    """
    k1, k2, kr = blade_kspace(N, L, R, theta)
    B = len(theta)
    if blade_frame is None:
        blade_frame = np.zeros(B, dtype=np.int64)
    y = np.zeros((B, L, R), dtype=np.complex128)
    fat_phase = np.exp(-2j * math.pi * kr * fat_shift)
    for b in range(B):
        t = int(blade_frame[b])
        acc_w = np.zeros((L, R), dtype=np.complex128)
        acc_f = np.zeros((L, R), dtype=np.complex128)
        for i, e in enumerate(ellipses):
            if motion is not None and i == motion[0]:
                e = moved(e, motion[1] * math.sin(2 * math.pi * t / motion[2]))
            ft = ellipse_ft(k1[b], k2[b], e) * e.rho
            acc_w += (1.0 - e.fat) * ft
            acc_f += e.fat * ft
        y[b] = (acc_w + fat_phase[b] * acc_f) / N
    return y


def simulate_cartesian_blades(ellipses: list, N: int, theta: np.ndarray, fat_shift: float) -> np.ndarray:
    """Per-blade k-space on the whole Cartesian grid, ycart[b, u2, u1]
    (complex128), k = (u - N/2)/N: the analytic ellipse FT with the fat
    component displaced by ``fat_shift`` along the blade's readout direction
    (the same physics as ``simulate_blades``, sampled on the Cartesian grid;
    which cells a blade measured is for the consumer to decide)."""
    k = (np.arange(N, dtype=np.float64) - N / 2) / N
    K2, K1 = np.meshgrid(k, k, indexing="ij")
    out = np.zeros((len(theta), N, N), dtype=np.complex128)
    for b, th in enumerate(np.asarray(theta, dtype=np.float64)):
        kr = K1 * math.cos(th) + K2 * math.sin(th)
        acc_w = np.zeros((N, N), dtype=np.complex128)
        acc_f = np.zeros((N, N), dtype=np.complex128)
        for e in ellipses:
            ft = ellipse_ft(K1, K2, e) * e.rho
            acc_w += (1.0 - e.fat) * ft
            acc_f += e.fat * ft
        out[b] = (acc_w + np.exp(-2j * math.pi * kr * fat_shift) * acc_f) / N
    return out


def add_noise(y: np.ndarray, rel_sigma: float, rng: np.random.Generator) -> np.ndarray:
    """Complex Gaussian noise, Re and Im ~ N(0, sigma^2/2), sigma = rel_sigma * max|y|."""
    sigma = rel_sigma * float(np.abs(y).max())
    n = rng.standard_normal(y.shape) + 1j * rng.standard_normal(y.shape)
    return y + n * (sigma / math.sqrt(2.0))


def rasterize(ellipses: list, N: int, supersample: int = 4, frame: int = 0,
              motion=None):
    """Box-averaged raster of the water and fat layers, each [N, N] complex128.

    Pixel (i2, i1) covers x in [x_i - 1/2, x_i + 1/2) with x_i = i - N/2.
    """
    s = supersample
    sub = (np.arange(s) + 0.5) / s - 0.5
    xs = (np.arange(N) - N / 2)[:, None] + sub[None, :]
    xs = xs.reshape(-1)
    X2, X1 = np.meshgrid(xs, xs, indexing="ij")
    water = np.zeros_like(X1, dtype=np.complex128)
    fat = np.zeros_like(X1, dtype=np.complex128)
    for i, e in enumerate(ellipses):
        if motion is not None and i == motion[0]:
            e = moved(e, motion[1] * math.sin(2 * math.pi * frame / motion[2]))
        ca, sa = math.cos(e.angle), math.sin(e.angle)
        d1 = X1 - e.center[0]
        d2 = X2 - e.center[1]
        u = (ca * d1 + sa * d2) / e.axes[0]
        v = (-sa * d1 + ca * d2) / e.axes[1]
        inside = (u * u + v * v) <= 1.0
        water += inside * ((1.0 - e.fat) * e.rho)
        fat += inside * (e.fat * e.rho)
    water = water.reshape(N, s, N, s).mean(axis=(1, 3))
    fat = fat.reshape(N, s, N, s).mean(axis=(1, 3))
    return water, fat
