"""The paper's own forward model: interpolated projection, Cartesian DFT and
blade mask, image- and k-space loss, one blade per iteration (oracle, FP64).

Test infrastructure: see the package docstring.

Sec. 4.2 "Projection" casts one ray per image pixel through the (x, y, omega)
volume, tilted by phi from the spectral axis in the plane of that axis and the
blade's readout direction, samples the volume along it by interpolation and
sums the samples.  Sec. 4.2 "Blur" takes the 2-D DFT of the projected image
and masks it by the blade's k-space support.  Sec. 4.3 fits the volume with
Adam, one blade per iteration, on the squared L2 error in k-space and in
image space plus TV and L1 terms along the spatial and spectral axes.

Readings where the paper is silent:
  * the ray meets spectral slice f (height h_f) at the in-plane point
    p - Delta_f d_b with Delta_f = h_f tan(phi), so a voxel at x in bin f lands
    on pixel x + Delta_f d_b: the same direction as the displacement phase of
    the non-uniform model.  Samples are taken at the slice heights, where the
    trilinear interpolation reduces to bilinear interpolation in the slice;
    samples outside the image read zero;
  * the DFT is the centred unitary one, Z(k) = (1/N) sum_x I(x)
    exp(-2 pi i k.x), k = (u - N/2)/N, x = i - N/2 on both axes;
  * the mask of blade b keeps the Cartesian cells whose rotated coordinates
    rho = N k.d_b and pi = N k.d_b^perp satisfy -R/2 - 1/2 <= rho < R/2 - 1/2
    and -L/2 - 1/2 <= pi < L/2 - 1/2: the unit cells around the blade's own
    sample lattice (at theta = 0 exactly the blade's samples); rho and pi
    within 1e-9 of a half-integer are taken as that half-integer, so that
    cos/sin rounding cannot decide a boundary cell;
  * measurements: per blade the Cartesian k-space data ycart[b] (cells
    outside the mask are ignored) and an image img[b]; when no image is
    given it is the inverse DFT of the masked k-space data;
  * data term of blade b: w_k sum_{mask} |Z - ycart|^2
    + w_i sum_pixels |U^H(M Z) - img|^2, Z = U P_b V_t(b);
  * regularisers: smoothed anisotropic TV along x1, x2 (tv_xy), along the
    spectral axis (tv_f) and along time (tv_t), each sqrt(|d|^2 + eps^2) per
    forward difference, and L1 sparsity l1 * sum sqrt(|V|^2 + eps^2);
  * schedule: iteration k (1-based) uses blade (k - 1) mod B; Adam as in
    ``recon.adam_step``; V_0 = 0; loss_trace[k - 1] is the iteration's loss
    before its update;
  * baseline (Sec. 6): the coverage-weighted k-space average of a range of
    blades (all blades, or the most recent ones of a dynamic series), each
    cell averaging the blades whose mask holds it, then the inverse DFT.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .geometry import Geometry
from .recon import _tv_axis, adam_step


@dataclass
class ProjParams:
    iters: int = 20
    lr: float = 1e-2
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    w_kspace: float = 0.1
    w_image: float = 1.0
    tv_xy: float = 1e-3
    tv_f: float = 0.0
    tv_t: float = 0.0
    l1: float = 0.0
    tv_eps: float = 1e-3


def shifts(g: Geometry, b: int) -> np.ndarray:
    """In-plane displacement Delta_f d_b of every bin for blade b: [Nf, 2] (along x1, x2)."""
    th = float(g.theta[b])
    return np.stack([g.delta * np.cos(th), g.delta * np.sin(th)], axis=1)


def project(Vt: np.ndarray, s: np.ndarray) -> np.ndarray:
    """I[i2, i1] = sum_f bilinear(Vt[:, :, f], (i1 - s[f, 0], i2 - s[f, 1])), zero outside."""
    N = Vt.shape[0]
    out = np.zeros((N, N), dtype=np.complex128)
    idx = np.arange(N, dtype=np.float64)
    for f in range(Vt.shape[2]):
        q1 = idx - s[f, 0]
        q2 = idx - s[f, 1]
        a1 = np.floor(q1)
        a2 = np.floor(q2)
        w1 = q1 - a1   # weight of the upper tap along x1
        w2 = q2 - a2
        a1 = a1.astype(np.int64)
        a2 = a2.astype(np.int64)
        for d2, c2 in ((0, 1.0 - w2), (1, w2)):
            j2 = a2 + d2
            ok2 = (j2 >= 0) & (j2 < N)
            for d1, c1 in ((0, 1.0 - w1), (1, w1)):
                j1 = a1 + d1
                ok1 = (j1 >= 0) & (j1 < N)
                vals = np.zeros((N, N), dtype=np.complex128)
                sub = Vt[np.clip(j2, 0, N - 1)][:, np.clip(j1, 0, N - 1), f]
                vals[:] = sub * (ok2[:, None] & ok1[None, :])
                out += (c2[:, None] * c1[None, :]) * vals
    return out


def project_adjoint(img: np.ndarray, s: np.ndarray, Nf: int) -> np.ndarray:
    """Transpose of ``project``: every pixel scatters its value with the same
    bilinear weights onto the taps it read (np.add.at)."""
    N = img.shape[0]
    out = np.zeros((N, N, Nf), dtype=np.complex128)
    idx = np.arange(N, dtype=np.float64)
    I2, I1 = np.meshgrid(idx, idx, indexing="ij")
    for f in range(Nf):
        q1 = I1 - s[f, 0]
        q2 = I2 - s[f, 1]
        a1 = np.floor(q1)
        a2 = np.floor(q2)
        w1 = q1 - a1
        w2 = q2 - a2
        a1 = a1.astype(np.int64)
        a2 = a2.astype(np.int64)
        for d2 in (0, 1):
            c2 = w2 if d2 else 1.0 - w2
            for d1 in (0, 1):
                c1 = w1 if d1 else 1.0 - w1
                j1 = a1 + d1
                j2 = a2 + d2
                ok = (j1 >= 0) & (j1 < N) & (j2 >= 0) & (j2 < N)
                np.add.at(out[:, :, f], (j2[ok], j1[ok]), (c1 * c2 * img)[ok])
    return out


def dft(I: np.ndarray) -> np.ndarray:
    """Centred unitary 2-D DFT (numpy's FFT as the step)."""
    N = I.shape[-1]
    return np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(I, axes=(-2, -1))), axes=(-2, -1)) / N


def idft(Z: np.ndarray) -> np.ndarray:
    """Inverse (= adjoint) of ``dft``."""
    N = Z.shape[-1]
    return np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(Z, axes=(-2, -1))), axes=(-2, -1)) * N


def _snap(a: np.ndarray) -> np.ndarray:
    """Rotated coordinates within 1e-9 of a half-integer become that
    half-integer, so that rounding in cos/sin cannot move a cell across a
    boundary at axis-aligned angles."""
    h = np.round(2.0 * a) / 2.0
    return np.where(np.abs(a - h) < 1e-9, h, a)


def blade_mask(N: int, theta: float, L: int, R: int) -> np.ndarray:
    """Boolean [u2, u1] support of a blade on the Cartesian k grid."""
    c = np.arange(N, dtype=np.float64) - N / 2.0
    C2, C1 = np.meshgrid(c, c, indexing="ij")
    rho = _snap(C1 * np.cos(theta) + C2 * np.sin(theta))
    pi = _snap(-C1 * np.sin(theta) + C2 * np.cos(theta))
    return ((rho >= -R / 2.0 - 0.5) & (rho < R / 2.0 - 0.5) &
            (pi >= -L / 2.0 - 0.5) & (pi < L / 2.0 - 0.5))


def forward(V: np.ndarray, g: Geometry, b: int) -> np.ndarray:
    """Masked Cartesian k-space of blade b: M_b U P_b V_t(b), [N, N]."""
    t = int(g.blade_frame[b])
    Z = dft(project(np.asarray(V, dtype=np.complex128)[t], shifts(g, b)))
    return Z * blade_mask(g.N, float(g.theta[b]), g.L, g.R)


def adjoint(z: np.ndarray, g: Geometry, b: int) -> np.ndarray:
    """P_b^H U^H M_b z placed in frame t(b) of a zero [T, N, N, Nf] volume."""
    out = np.zeros((g.T, g.N, g.N, g.Nf), dtype=np.complex128)
    zm = np.asarray(z, dtype=np.complex128) * blade_mask(g.N, float(g.theta[b]), g.L, g.R)
    out[int(g.blade_frame[b])] = project_adjoint(idft(zm), shifts(g, b), g.Nf)
    return out


def image_of(ycart: np.ndarray, g: Geometry, b: int) -> np.ndarray:
    """The measured image of blade b when none is given: U^H (M_b ycart_b)."""
    return idft(np.asarray(ycart[b], dtype=np.complex128) * blade_mask(g.N, float(g.theta[b]), g.L, g.R))


def baseline(ycart: np.ndarray, g: Geometry, lo: int = 0, hi=None) -> np.ndarray:
    """The results section's baseline: the coverage-weighted average of the
    blades lo .. hi-1 in k-space (each Cartesian cell averages the blades
    whose mask holds it; uncovered cells are zero), then the inverse DFT."""
    hi = g.B if hi is None else hi
    acc = np.zeros((g.N, g.N), dtype=np.complex128)
    cnt = np.zeros((g.N, g.N))
    for b in range(lo, hi):
        m = blade_mask(g.N, float(g.theta[b]), g.L, g.R)
        acc += m * np.asarray(ycart[b], dtype=np.complex128)
        cnt += m
    return idft(np.where(cnt > 0, acc / np.maximum(cnt, 1.0), 0.0))


def l1(V: np.ndarray, eps: float):
    """sum sqrt(|V|^2 + eps^2) and its gradient."""
    mag = np.sqrt(np.abs(V) ** 2 + eps * eps)
    return float(mag.sum()), V / mag


def loss_and_grad(V: np.ndarray, ycart: np.ndarray, img, g: Geometry, b: int, p: ProjParams):
    """Loss of iteration on blade b and dL/dRe V + i dL/dIm V."""
    V = np.asarray(V, dtype=np.complex128)
    t = int(g.blade_frame[b])
    s = shifts(g, b)
    M = blade_mask(g.N, float(g.theta[b]), g.L, g.R)
    y = np.asarray(ycart[b], dtype=np.complex128)
    im = image_of(ycart, g, b) if img is None else np.asarray(img[b], dtype=np.complex128)
    Z = dft(project(V[t], s))
    rk = M * (Z - y)                      # k-space residual on the mask
    ri = idft(M * Z) - im                 # image-space residual
    loss = p.w_kspace * float(np.sum(np.abs(rk) ** 2)) + p.w_image * float(np.sum(np.abs(ri) ** 2))
    # chain rule written step by step: d/dZ of both terms, then U^H, then P^H
    dZ = p.w_kspace * rk + p.w_image * (M * dft(ri))
    grad = np.zeros_like(V)
    grad[t] = 2.0 * project_adjoint(idft(dZ), s, g.Nf)
    for w, fn in ((p.tv_xy, lambda: _tv_axis(V, 2, p.tv_eps)), (p.tv_xy, lambda: _tv_axis(V, 1, p.tv_eps)),
                  (p.tv_f, lambda: _tv_axis(V, 3, p.tv_eps)), (p.tv_t, lambda: _tv_axis(V, 0, p.tv_eps)),
                  (p.l1, lambda: l1(V, p.tv_eps))):
        if w != 0.0:
            v, gr = fn()
            loss += w * v
            grad += w * gr
    return loss, grad


def reconstruct(ycart: np.ndarray, img, g: Geometry, p: ProjParams, V0=None):
    """Adam over the blades in turn: returns (V_K, loss_trace[K])."""
    shape = (g.T, g.N, g.N, g.Nf)
    V = np.zeros(shape, dtype=np.complex128) if V0 is None else np.array(V0, dtype=np.complex128)
    m = np.zeros(shape + (2,))
    v = np.zeros(shape + (2,))
    trace = np.zeros(p.iters)
    for k in range(1, p.iters + 1):
        b = (k - 1) % g.B
        loss, grad = loss_and_grad(V, ycart, img, g, b, p)
        trace[k - 1] = loss
        V, m, v = adam_step(V, grad, m, v, k, p)
    return V, trace
