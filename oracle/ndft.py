"""Exact volumetric forward operator and its adjoint (oracle, FP64).

Test infrastructure: see the package docstring.

The paper lifts the image to a volume V(x, f) over space and a spectral axis
(Sec. 4.1) and explains off-resonance as a translation of each spectral layer
along the blade's readout direction (Sec. 3, Eq. 2, and Fig. 2's projection
picture).  Sampling the Fourier transform on the blade's lines (Sec. 4.2
"Blur", with the non-uniform blade-aligned lines of Sec. 7 "Limitations")
gives the operator written out here as its plain definition:

    y_b(k) = s * sum_f sum_x V_t(b)(x, f) exp(-2 pi i k.(x + Delta_f d_b))
           = s * sum_f P[m, f] sum_x V_t(b)(x, f) exp(-2 pi i k.x),

with s = 1/N, P[m, f] = exp(-2 pi i k_r Delta_f) and x over the integer pixel
grid {-N/2..N/2-1}^2.  The inner sum is evaluated exactly as two dense
complex matrix products per blade (library zgemm as a step, no
approximation).  The adjoint is the conjugate transpose of each step.

Array layout: V[t, i2, i1, f] with x_a = i_a - N/2; y[b, l, j].
"""
from __future__ import annotations

import numpy as np

from .geometry import Geometry, sample_coords, phase_table, sample_frame

_CHUNK = 2048   # samples per matrix-product chunk (bounds temporary memory)


def _exp_rows(k: np.ndarray, x: np.ndarray, sign: float) -> np.ndarray:
    return np.exp(sign * 2j * np.pi * np.outer(k, x))


def _forward_samples(V, g: Geometry, idx: np.ndarray) -> np.ndarray:
    """y at flat sample indices ``idx`` (all in one frame or mixed)."""
    k1, k2, kr = sample_coords(g)
    fr = sample_frame(g)
    x = g.pixel_coords()
    N, Nf = g.N, g.Nf
    out = np.zeros(len(idx), dtype=np.complex128)
    for t in np.unique(fr[idx]):
        sel = np.nonzero(fr[idx] == t)[0]
        # Vt[i1, (i2, f)] so that E1 @ Vt sums over x1.
        Vt = np.ascontiguousarray(V[t].transpose(1, 0, 2)).reshape(N, N * Nf)
        for c0 in range(0, len(sel), _CHUNK):
            s = sel[c0:c0 + _CHUNK]
            m = idx[s]
            E1 = _exp_rows(k1[m], x, -1.0)                     # [S, N] over x1
            E2 = _exp_rows(k2[m], x, -1.0)                     # [S, N] over x2
            Tm = (E1 @ Vt).reshape(len(m), N, Nf)              # sum_x1 -> [S, i2, f]
            inner = np.einsum("si,sif->sf", E2, Tm)            # sum_x2 -> [S, f]
            P = phase_table(kr[m], g.delta)                    # [S, f]
            out[s] = g.scale * np.sum(P * inner, axis=1)
    return out


def forward(V: np.ndarray, g: Geometry) -> np.ndarray:
    """A V: y[b, l, j] complex128 from V[t, i2, i1, f]."""
    V = np.asarray(V, dtype=np.complex128)
    assert V.shape == (g.T, g.N, g.N, g.Nf), V.shape
    y = _forward_samples(V, g, np.arange(g.M))
    return y.reshape(g.B, g.L, g.R)


def forward_at(V: np.ndarray, g: Geometry, samples: np.ndarray) -> np.ndarray:
    """(A V) at the flat sample indices ``samples`` (each output is an independent sum)."""
    V = np.asarray(V, dtype=np.complex128)
    return _forward_samples(V, g, np.asarray(samples, dtype=np.int64))


def adjoint(y: np.ndarray, g: Geometry) -> np.ndarray:
    """A^H y: V[t, i2, i1, f] complex128 from y[b, l, j] (no factor 2)."""
    y = np.asarray(y, dtype=np.complex128).reshape(-1)
    assert y.size == g.M
    k1, k2, kr = sample_coords(g)
    fr = sample_frame(g)
    x = g.pixel_coords()
    N, Nf = g.N, g.Nf
    V = np.zeros((g.T, N, N, Nf), dtype=np.complex128)
    for t in np.unique(fr):
        sel = np.nonzero(fr == t)[0]
        acc = np.zeros((N, N * Nf), dtype=np.complex128)       # [i2, (i1, f)]
        for c0 in range(0, len(sel), _CHUNK):
            m = sel[c0:c0 + _CHUNK]
            E1c = _exp_rows(k1[m], x, +1.0)                    # conj(E1) [S, N]
            E2c = _exp_rows(k2[m], x, +1.0)                    # conj(E2) [S, N]
            c = np.conj(phase_table(kr[m], g.delta)) * y[m][:, None]   # [S, f]
            W = (E1c[:, :, None] * c[:, None, :]).reshape(len(m), N * Nf)
            acc += E2c.T @ W                                   # sum over samples
        V[t] = g.scale * acc.reshape(N, N, Nf)
    return V


def adjoint_at(y: np.ndarray, g: Geometry, voxels: np.ndarray) -> np.ndarray:
    """(A^H y) at flat voxel indices into V[t, i2, i1, f] (each an independent sum)."""
    y = np.asarray(y, dtype=np.complex128).reshape(-1)
    voxels = np.asarray(voxels, dtype=np.int64)
    k1, k2, kr = sample_coords(g)
    fr = sample_frame(g)
    N, Nf = g.N, g.Nf
    t, rem = np.divmod(voxels, N * N * Nf)
    i2, rem = np.divmod(rem, N * Nf)
    i1, f = np.divmod(rem, Nf)
    x1 = i1 - N // 2
    x2 = i2 - N // 2
    out = np.zeros(len(voxels), dtype=np.complex128)
    c = np.conj(phase_table(kr, g.delta)) * y[:, None]           # [M, f]
    for tt in np.unique(t):
        q = np.nonzero(t == tt)[0]
        m = np.nonzero(fr == tt)[0]
        for c0 in range(0, len(q), 256):
            qq = q[c0:c0 + 256]
            E = np.exp(2j * np.pi * (np.outer(k1[m], x1[qq]) + np.outer(k2[m], x2[qq])))
            out[qq] = g.scale * np.sum(E * c[m][:, f[qq]], axis=0)
    return out
