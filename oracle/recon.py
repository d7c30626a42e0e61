"""Loss, regularisers, Adam and the reconstruction loop (oracle, FP64).

Test infrastructure: see the package docstring.

Sec. 4.3 optimises the volume's grid values with Adam on a squared-L2 data
term plus total-variation regularisation (and, for dynamic series, temporal
smoothness).  Readings where the paper is silent:
  * data term: the plain sum sum_m |(A V)_m - y_m|^2 over all blade samples
    (full batch, k-space term only), so its gradient is 2 A^H (A V - y);
  * TV: anisotropic and smoothed, per complex difference d,
    sqrt(|d|^2 + eps^2), forward differences with no wrap-around, along x1 and
    x2 (TV_xy) and along the frame axis (TV_t);
  * gradient convention: dL/dRe V + i dL/dIm V (torch's convention for
    complex parameters), so real and imaginary parts are separate parameters;
  * Adam as in Kingma & Ba with bias correction (beta1, beta2, eps), per real
    component; V_0 = 0 unless a start is given;
  * loss_trace[k] is L(V_k), evaluated in iteration k+1 before its update.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .geometry import Geometry
from .ndft import forward, adjoint


@dataclass
class ReconParams:
    iters: int = 20
    lr: float = 1e-2
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    tv_xy: float = 1e-3
    tv_t: float = 0.0
    tv_eps: float = 1e-3


def data_loss(V: np.ndarray, y: np.ndarray, g: Geometry):
    """sum |A V - y|^2 and the residual r = A V - y."""
    r = forward(V, g) - np.asarray(y, dtype=np.complex128).reshape(g.B, g.L, g.R)
    return float(np.sum(np.abs(r) ** 2)), r


def _tv_axis(V: np.ndarray, axis: int, eps: float):
    """sum over forward differences along ``axis`` of sqrt(|d|^2 + eps^2), and its gradient."""
    grad = np.zeros_like(V)
    if V.shape[axis] < 2:
        return 0.0, grad
    d = np.diff(V, axis=axis)
    mag = np.sqrt(np.abs(d) ** 2 + eps * eps)
    q = d / mag
    lo = [slice(None)] * V.ndim
    hi = [slice(None)] * V.ndim
    lo[axis] = slice(0, -1)
    hi[axis] = slice(1, None)
    grad[tuple(lo)] -= q
    grad[tuple(hi)] += q
    return float(mag.sum()), grad


def tv_xy(V: np.ndarray, eps: float):
    """Spatial TV of V[t, i2, i1, f] (axes 2 = x1 and 1 = x2) and its gradient."""
    v1, g1 = _tv_axis(V, 2, eps)
    v2, g2 = _tv_axis(V, 1, eps)
    return v1 + v2, g1 + g2


def tv_t(V: np.ndarray, eps: float):
    """Temporal TV of V[t, i2, i1, f] (axis 0) and its gradient."""
    return _tv_axis(V, 0, eps)


def loss_and_grad(V: np.ndarray, y: np.ndarray, g: Geometry, p: ReconParams):
    """L(V) = sum|A V - y|^2 + tv_xy TV_xy(V) + tv_t TV_t(V), and dL/dRe + i dL/dIm."""
    dl, r = data_loss(V, y, g)
    grad = 2.0 * adjoint(r, g)
    loss = dl
    if p.tv_xy != 0.0:
        v, gr = tv_xy(V, p.tv_eps)
        loss += p.tv_xy * v
        grad += p.tv_xy * gr
    if p.tv_t != 0.0:
        v, gr = tv_t(V, p.tv_eps)
        loss += p.tv_t * v
        grad += p.tv_t * gr
    return loss, grad


def adam_step(V, grad, m, v, k: int, p: ReconParams):
    """One Adam update (step k >= 1) on the real and imaginary parts of V.

    m and v have V's shape plus a trailing axis of 2 (real, imaginary).
    Returns the new (V, m, v).
    """
    gr = np.stack([grad.real, grad.imag], axis=-1)
    m = p.beta1 * m + (1.0 - p.beta1) * gr
    v = p.beta2 * v + (1.0 - p.beta2) * gr * gr
    mhat = m / (1.0 - p.beta1 ** k)
    vhat = v / (1.0 - p.beta2 ** k)
    step = p.lr * mhat / (np.sqrt(vhat) + p.eps)
    V = V - (step[..., 0] + 1j * step[..., 1])
    return V, m, v


def reconstruct(y: np.ndarray, g: Geometry, p: ReconParams, V0=None):
    """Full-batch Adam reconstruction: returns (V_K, loss_trace[K])."""
    shape = (g.T, g.N, g.N, g.Nf)
    V = np.zeros(shape, dtype=np.complex128) if V0 is None else np.array(V0, dtype=np.complex128)
    m = np.zeros(shape + (2,))
    v = np.zeros(shape + (2,))
    trace = np.zeros(p.iters)
    for k in range(1, p.iters + 1):
        loss, grad = loss_and_grad(V, y, g, p)
        trace[k - 1] = loss
        V, m, v = adam_step(V, grad, m, v, k, p)
    return V, trace


def render(V: np.ndarray, f_lo: int = 0, f_hi=None) -> np.ndarray:
    """phi = 0 projection: image[t, i2, i1] = sum_{f_lo <= f < f_hi} V[t, i2, i1, f].

    The full range is the final render of Sec. 4.3; a lower or upper part of
    the spectral axis gives the water-only or fat-only image of Sec. 6.
    """
    V = np.asarray(V)
    if f_hi is None:
        f_hi = V.shape[-1]
    return V[..., f_lo:f_hi].sum(axis=-1)


def psnr(image: np.ndarray, ref: np.ndarray) -> float:
    """Peak signal-to-noise ratio of |image| against |ref| in dB (the quality
    figure of the results, Sec. 6, Table 1): 10 log10(max|ref|^2 / mean
    (|image| - |ref|)^2) over the whole array; +inf when the magnitudes agree."""
    a = np.abs(np.asarray(image, dtype=np.complex128))
    b = np.abs(np.asarray(ref, dtype=np.complex128))
    mse = float(np.mean((a - b) ** 2))
    if mse == 0.0:
        return float("inf")
    return float(10.0 * np.log10(float(np.max(b)) ** 2 / mse))
