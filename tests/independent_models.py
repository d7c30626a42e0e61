"""Independent torch statements of the three reconstruction problems.

These exist only to pin the oracle's optimisation loops (``oracle.reconstruct``,
``oracle.projection.reconstruct``, ``oracle.kplanes.reconstruct``) against an
implementation that shares none of their code: every operator here is a dense
matrix assembled entry by entry from its definition, every regulariser is
written with torch ops, gradients come from ``torch.autograd`` and the
optimiser is ``torch.optim.Adam`` (float64, complex parameters).  Sizes are
tiny (8 x 8 images) so that the dense matrices stay small.

Definitions restated (all from the paper's model, with the readings the
oracle documents):
  * non-uniform model (Sec. 3 Eq. 2, Sec. 4.2): entry (m, voxel) of A is
    exp(-2 pi i k_m . (x + Delta_f d_b)) / N for the voxels of frame t(b);
  * projection model (Sec. 4.2): pixel p of blade b's image sums, over the
    bins, the bilinear interpolation of bin f at p - Delta_f d_b (zero
    outside the image); the blur is the centred unitary DFT masked by the
    blade's support;
  * K-Planes (Sec. 4.1 Eq. 3): the volume is sum_k a_k times the product of
    the six bilinearly interpolated plane features, summed over scales;
  * losses as in Sec. 4.3, TV smoothed as sqrt(|d|^2 + eps^2) over forward
    differences; Adam with the step counter starting at 1.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def nonuniform_matrix(N, L, R, theta, delta, blade_frame, T) -> np.ndarray:
    """Dense A [B L R, T N N Nf] from the displaced-position form, one entry at a time."""
    Nf = len(delta)
    B = len(theta)
    A = np.zeros((B * L * R, T * N * N * Nf), dtype=np.complex128)
    row = 0
    for b in range(B):
        c, s = math.cos(theta[b]), math.sin(theta[b])
        for l in range(L):
            for j in range(R):
                kr, kp = (j - R / 2) / N, (l - L / 2) / N
                k1, k2 = kr * c - kp * s, kr * s + kp * c
                for i2 in range(N):
                    for i1 in range(N):
                        for f in range(Nf):
                            p1 = (i1 - N // 2) + delta[f] * c
                            p2 = (i2 - N // 2) + delta[f] * s
                            col = ((int(blade_frame[b]) * N + i2) * N + i1) * Nf + f
                            A[row, col] = complex(math.cos(-2 * math.pi * (k1 * p1 + k2 * p2)),
                                                  math.sin(-2 * math.pi * (k1 * p1 + k2 * p2))) / N
                row += 1
    return A


def _abs2(z: torch.Tensor) -> torch.Tensor:
    return z.real * z.real + z.imag * z.imag


def smoothed_tv(V: torch.Tensor, dim: int, eps: float) -> torch.Tensor:
    """sum over forward differences along ``dim`` of sqrt(|d|^2 + eps^2)."""
    if V.shape[dim] < 2:
        return V.real.sum() * 0.0
    n = V.shape[dim]
    d = V.narrow(dim, 1, n - 1) - V.narrow(dim, 0, n - 1)
    return torch.sqrt(_abs2(d) + eps * eps).sum()


def smoothed_l1(V: torch.Tensor, eps: float) -> torch.Tensor:
    return torch.sqrt(_abs2(V) + eps * eps).sum()


def volume_loss(V, A, y, tv_xy, tv_t, eps):
    """sum |A vec(V) - y|^2 + tv_xy (TV along x1 and x2) + tv_t TV along frames; V[t, i2, i1, f]."""
    r = A @ V.reshape(-1) - y.reshape(-1)
    loss = _abs2(r).sum()
    if tv_xy:
        loss = loss + tv_xy * (smoothed_tv(V, 2, eps) + smoothed_tv(V, 1, eps))
    if tv_t:
        loss = loss + tv_t * smoothed_tv(V, 0, eps)
    return loss


def run_adam(params, loss_fn, iters, lr, betas=(0.9, 0.999), eps=1e-8):
    """torch.optim.Adam over ``params``; loss_fn(k) is the loss of iteration k
    (1-based).  Returns the loss of every iteration taken before its step."""
    opt = torch.optim.Adam(params, lr=lr, betas=betas, eps=eps)
    trace = []
    for k in range(1, iters + 1):
        opt.zero_grad()
        loss = loss_fn(k)
        trace.append(float(loss.detach()))
        loss.backward()
        opt.step()
    return np.array(trace)


# --- projection model ---------------------------------------------------------

def projection_matrix(N, Nf, theta, delta) -> np.ndarray:
    """Dense P_b [N N, N N Nf] (pixel (i2, i1) <- voxel (j2, j1, f)), by explicit taps."""
    P = np.zeros((N * N, N * N * Nf))
    c, s = math.cos(theta), math.sin(theta)
    for i2 in range(N):
        for i1 in range(N):
            for f in range(Nf):
                q1, q2 = i1 - delta[f] * c, i2 - delta[f] * s
                a1, a2 = math.floor(q1), math.floor(q2)
                t1, t2 = q1 - a1, q2 - a2
                for j2, w2 in ((a2, 1.0 - t2), (a2 + 1, t2)):
                    for j1, w1 in ((a1, 1.0 - t1), (a1 + 1, t1)):
                        if 0 <= j1 < N and 0 <= j2 < N:
                            P[i2 * N + i1, (j2 * N + j1) * Nf + f] += w1 * w2
    return P


def blade_support(N, theta, L, R) -> np.ndarray:
    """[u2, u1] cells whose rotated coordinates lie in the blade's unit cells."""
    M = np.zeros((N, N), dtype=bool)
    c, s = math.cos(theta), math.sin(theta)
    for u2 in range(N):
        for u1 in range(N):
            a1, a2 = u1 - N / 2, u2 - N / 2
            rho, pi_ = a1 * c + a2 * s, -a1 * s + a2 * c
            rho = round(2 * rho) / 2 if abs(rho - round(2 * rho) / 2) < 1e-9 else rho
            pi_ = round(2 * pi_) / 2 if abs(pi_ - round(2 * pi_) / 2) < 1e-9 else pi_
            M[u2, u1] = (-R / 2 - 0.5 <= rho < R / 2 - 0.5) and (-L / 2 - 0.5 <= pi_ < L / 2 - 0.5)
    return M


def centred_dft(I: torch.Tensor) -> torch.Tensor:
    N = I.shape[-1]
    return torch.fft.fftshift(torch.fft.fft2(torch.fft.ifftshift(I, dim=(-2, -1))), dim=(-2, -1)) / N


def centred_idft(Z: torch.Tensor) -> torch.Tensor:
    N = Z.shape[-1]
    return torch.fft.fftshift(torch.fft.ifft2(torch.fft.ifftshift(Z, dim=(-2, -1))), dim=(-2, -1)) * N


# --- K-Planes -----------------------------------------------------------------

def axis_weights(N: int, R: int) -> np.ndarray:
    """[N, R] linear interpolation weights of voxel index i on R cell-centred
    nodes spanning the N voxels (coordinate (i + 1/2) R / N - 1/2, clamped)."""
    W = np.zeros((N, R))
    for i in range(N):
        if R == 1:
            W[i, 0] = 1.0
            continue
        u = min(max((i + 0.5) * R / N - 0.5, 0.0), R - 1.0)
        lo = min(math.floor(u), R - 2)
        W[i, lo] += 1.0 - (u - lo)
        W[i, lo + 1] += u - lo
    return W


def kplanes_volume(planes, avec, N, Nf, T):
    """V[t, y, x, w] from per-scale dicts of torch planes and torch a vectors."""
    dt = torch.complex128
    V = torch.zeros((T, N, N, Nf), dtype=dt)
    for P, a in zip(planes, avec):
        n = P["xy"].shape[1]
        Wx = torch.tensor(axis_weights(N, n), dtype=dt)
        Ww = torch.tensor(axis_weights(Nf, Nf), dtype=dt)
        Wt = torch.tensor(axis_weights(T, T), dtype=dt)
        hxy = torch.einsum("ir,jc,rck->ijk", Wx, Wx, P["xy"])   # [y][x]
        hxw = torch.einsum("ir,jc,rck->ijk", Ww, Wx, P["xw"])   # [w][x]
        hxt = torch.einsum("ir,jc,rck->ijk", Wt, Wx, P["xt"])   # [t][x]
        hyw = torch.einsum("ir,jc,rck->ijk", Ww, Wx, P["yw"])   # [w][y]
        hyt = torch.einsum("ir,jc,rck->ijk", Wt, Wx, P["yt"])   # [t][y]
        hwt = torch.einsum("ir,jc,rck->ijk", Wt, Ww, P["wt"])   # [t][w]
        V = V + torch.einsum("yxk,wxk,txk,wyk,tyk,twk,k->tyxw", hxy, hxw, hxt, hyw, hyt, hwt, a)
    return V
