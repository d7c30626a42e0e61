"""The dynamic K-Planes volume model (Sec. 4.1, Eq. 3) -- oracle, FP64.

Test infrastructure: see the package docstring.

Eq. 3 models the complex signal at (x, y, omega, t) as the inner product of
a weighting vector a with the elementwise product of six feature vectors,
each bilinearly interpolated in one of the planes xy, x-omega, x-t,
y-omega, y-t and omega-t; two scales (full and half spatial resolution) are
summed.  This module renders that model on the volume grid and carries
gradients back to the plane parameters; the volume then enters either
forward model unchanged.

Readings where the paper is silent:
  * feature dimension F = 8 (stated), complex parameters and a complex a per
    scale; the inner product is sum_k a_k h_k (no conjugation);
  * plane shapes [rows][cols][F]: xy [Ny][Nx], x-omega [Nf][Nx], x-t [T][Nx],
    y-omega [Nf][Ny], y-t [T][Ny], omega-t [T][Nf], with Nx = Ny = N at scale
    0 and N/2 at scale 1 (spectral and time resolutions unchanged);
  * coordinates: plane nodes are cell centres spanning the same extent as the
    volume's voxels, so voxel index i maps to the node coordinate
    (i + 1/2) R / N - 1/2 for a spatial axis of R nodes (i itself at full
    resolution, i/2 - 1/4 at half); spectral and time indices map to nodes
    directly; bilinear interpolation clamps coordinates to [0, R - 1];
  * gradients: dL/dRe + i dL/dIm for every complex parameter, so for a
    parameter z that the volume depends on holomorphically,
    grad z = sum conj(dV/dz) grad V.
"""
from __future__ import annotations

import numpy as np

PLANES = ("xy", "xw", "xt", "yw", "yt", "wt")   # w = omega


def plane_shapes(N: int, Nf: int, T: int, F: int = 8, scale: int = 0) -> dict:
    n = N >> scale
    return {"xy": (n, n, F), "xw": (Nf, n, F), "xt": (T, n, F),
            "yw": (Nf, n, F), "yt": (T, n, F), "wt": (T, Nf, F)}


def node_coord(i: np.ndarray, R: int, N: int) -> np.ndarray:
    """Continuous node coordinate of voxel index i on an axis of R plane nodes."""
    return (np.asarray(i, dtype=np.float64) + 0.5) * R / N - 0.5


def _taps(u: np.ndarray, R: int):
    """Lower node, upper node and upper weight of each coordinate, clamped."""
    u = np.clip(u, 0.0, R - 1.0)
    lo = np.minimum(np.floor(u).astype(np.int64), max(R - 2, 0))
    w = u - lo
    hi = np.minimum(lo + 1, R - 1)
    return lo, hi, w


def _axes(N: int, Nf: int, T: int, n: int):
    """Per plane: (row coordinates over the voxel axis, col coordinates), as
    tap triples, for spatial planes of n nodes per axis."""
    ix = _taps(node_coord(np.arange(N), n, N), n)     # x and y axes share the mapping
    iw = _taps(np.arange(Nf, dtype=np.float64), Nf)
    it = _taps(np.arange(T, dtype=np.float64), T)
    return {"xy": (ix, ix), "xw": (iw, ix), "xt": (it, ix), "yw": (iw, ix), "yt": (it, ix), "wt": (it, iw)}


def _interp(P: np.ndarray, rows, cols) -> np.ndarray:
    """Bilinear interpolation of plane P [R][C][F] at every (row, col) pair: [len(rows)][len(cols)][F]."""
    r0, r1, wr = rows
    c0, c1, wc = cols
    A = P[r0][:, c0] * (1 - wr)[:, None, None] * (1 - wc)[None, :, None]
    A = A + P[r0][:, c1] * (1 - wr)[:, None, None] * wc[None, :, None]
    A = A + P[r1][:, c0] * wr[:, None, None] * (1 - wc)[None, :, None]
    A = A + P[r1][:, c1] * wr[:, None, None] * wc[None, :, None]
    return A


def _interp_T(G: np.ndarray, rows, cols, shape) -> np.ndarray:
    """Transpose of ``_interp``: scatter G [len(rows)][len(cols)][F] onto the plane nodes."""
    r0, r1, wr = rows
    c0, c1, wc = cols
    out = np.zeros(shape, dtype=np.complex128)
    for rr, fr in ((r0, 1 - wr), (r1, wr)):
        for cc, fc in ((c0, 1 - wc), (c1, wc)):
            W = G * fr[:, None, None] * fc[None, :, None]
            R_, C_ = np.meshgrid(rr, cc, indexing="ij")
            np.add.at(out, (R_, C_), W)
    return out


def _features(params: dict, N: int, Nf: int, T: int, scale: int) -> dict:
    """Interpolated features of every plane broadcast to [T][N(y)][N(x)][Nf][F]."""
    p = params["planes"][scale]
    ax = _axes(N, Nf, T, p["xy"].shape[1])
    hxy = _interp(p["xy"], *ax["xy"])                 # [y][x][F]
    hxw = _interp(p["xw"], *ax["xw"])                 # [w][x][F]
    hxt = _interp(p["xt"], *ax["xt"])                 # [t][x][F]
    hyw = _interp(p["yw"], *ax["yw"])                 # [w][y][F]
    hyt = _interp(p["yt"], *ax["yt"])                 # [t][y][F]
    hwt = _interp(p["wt"], *ax["wt"])                 # [t][w][F]
    return {
        "xy": hxy[None, :, :, None, :],
        "xw": np.transpose(hxw, (1, 0, 2))[None, None, :, :, :],
        "xt": hxt[:, None, :, None, :],
        "yw": np.transpose(hyw, (1, 0, 2))[None, :, None, :, :],
        "yt": hyt[:, :, None, None, :],
        "wt": hwt[:, None, None, :, :],
    }


def render(params: dict, N: int, Nf: int, T: int) -> np.ndarray:
    """V[t, i2, i1, f] = sum over scales of sum_k a_k prod_c psi_c,k (Eq. 3)."""
    V = np.zeros((T, N, N, Nf), dtype=np.complex128)
    for s in range(len(params["planes"])):
        h = _features(params, N, Nf, T, s)
        prod = np.ones((T, N, N, Nf, h["xy"].shape[-1]), dtype=np.complex128)
        for c in PLANES:
            prod = prod * h[c]
        V += prod @ params["a"][s]
    return V


def vjp(params: dict, gV: np.ndarray, N: int, Nf: int, T: int) -> dict:
    """Gradients of a real loss with respect to every parameter, given
    gV = dL/dRe V + i dL/dIm V: grad z = sum conj(dV/dz) gV."""
    out = {"planes": [], "a": []}
    for s in range(len(params["planes"])):
        ax = _axes(N, Nf, T, params["planes"][s]["xy"].shape[1])
        h = _features(params, N, Nf, T, s)
        full = {c: np.broadcast_to(h[c], (T, N, N, Nf, h["xy"].shape[-1])) for c in PLANES}
        prod = np.ones_like(full["xy"])
        for c in PLANES:
            prod = prod * full[c]
        a = params["a"][s]
        out["a"].append(np.einsum("tyxwk,tyxw->k", np.conj(prod), gV))
        gs = {}
        for c in PLANES:
            others = np.ones_like(prod)
            for c2 in PLANES:
                if c2 != c:
                    others = others * full[c2]
            gh = np.conj(a[None, None, None, None, :] * others) * gV[..., None]   # [t][y][x][w][F]
            # sum over the axes the plane does not have, in the plane's (row, col) order
            red = {"xy": np.einsum("tyxwk->yxk", gh), "xw": np.einsum("tyxwk->wxk", gh),
                   "xt": np.einsum("tyxwk->txk", gh), "yw": np.einsum("tyxwk->wyk", gh),
                   "yt": np.einsum("tyxwk->tyk", gh), "wt": np.einsum("tyxwk->twk", gh)}[c]
            gs[c] = _interp_T(red, *ax[c], params["planes"][s][c].shape)
        out["planes"].append(gs)
    return out


def init_params(N: int, Nf: int, T: int, rng: np.random.Generator, F: int = 8, scales: int = 2,
                spread: float = 0.1) -> dict:
    """Planes near one (the product starts near the weighting), small random a."""
    planes, avec = [], []
    for s in range(scales):
        planes.append({c: (1.0 + spread * (rng.standard_normal(sh) + 1j * rng.standard_normal(sh)))
                       for c, sh in plane_shapes(N, Nf, T, F, s).items()})
        avec.append(spread * (rng.standard_normal(F) + 1j * rng.standard_normal(F)))
    return {"planes": planes, "a": avec}


def loss_and_grad(params: dict, y: np.ndarray, g, p):
    """The main path's loss (data term of the non-uniform model plus TV, as
    ``recon.loss_and_grad``) of the rendered volume, and the parameter
    gradients by ``vjp``."""
    from .recon import loss_and_grad as volume_loss
    V = render(params, g.N, g.Nf, g.T)
    loss, gV = volume_loss(V, y, g, p)
    return loss, vjp(params, gV, g.N, g.Nf, g.T)


def reconstruct(y: np.ndarray, g, p, params0: dict):
    """Adam on every parameter array (``recon.adam_step``, step k for all)
    for ``loss_and_grad``: returns (params_K, loss_trace[K])."""
    from .recon import adam_step
    prm = {"planes": [{c: np.array(v, dtype=np.complex128) for c, v in d.items()} for d in params0["planes"]],
           "a": [np.array(v, dtype=np.complex128) for v in params0["a"]]}
    mom = {"planes": [{c: [np.zeros(v.shape + (2,)), np.zeros(v.shape + (2,))] for c, v in d.items()}
                      for d in prm["planes"]],
           "a": [[np.zeros(v.shape + (2,)), np.zeros(v.shape + (2,))] for v in prm["a"]]}
    trace = np.zeros(p.iters)
    for k in range(1, p.iters + 1):
        loss, G = loss_and_grad(prm, y, g, p)
        trace[k - 1] = loss
        for s in range(len(prm["planes"])):
            for c in PLANES:
                mm, vv = mom["planes"][s][c]
                prm["planes"][s][c], mm, vv = adam_step(prm["planes"][s][c], G["planes"][s][c], mm, vv, k, p)
                mom["planes"][s][c] = [mm, vv]
            mm, vv = mom["a"][s]
            prm["a"][s], mm, vv = adam_step(prm["a"][s], G["a"][s], mm, vv, k, p)
            mom["a"][s] = [mm, vv]
    return prm, trace
