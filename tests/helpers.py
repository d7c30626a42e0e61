"""Shared test helpers: build matching oracle geometries and GPU plans."""
import math

import numpy as np

import oracle
import synth


def rel(a, b) -> float:
    """Relative L2 error ||a - b|| / ||b|| over the whole tensor (b = reference)."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def geometry(N, L, R, theta, delta, blade_frame=None, T=1):
    return oracle.make_geometry(N, L, R, theta, delta, blade_frame, T)


def random_case(N, Nf, B, L, R, T=1, seed=0, delta_range=(-3.0, 3.0)):
    """Random geometry (uniform-ish angles with jitter), random volume and data."""
    rng = np.random.default_rng(seed)
    theta = np.pi * np.arange(B) / B + rng.uniform(-0.05, 0.05, B)
    delta = np.linspace(delta_range[0], delta_range[1], Nf) if Nf > 1 else np.array([0.7])
    frames = (np.arange(B) * T // B).astype(np.int32)
    V = (rng.standard_normal((T, N, N, Nf)) + 1j * rng.standard_normal((T, N, N, Nf))).astype(np.complex64)
    y = (rng.standard_normal((B, L, R)) + 1j * rng.standard_normal((B, L, R))).astype(np.complex64)
    return dict(theta=theta, delta=delta, blade_frame=frames, V=V, y=y, N=N, L=L, R=R, T=T)


def workload_case(name):
    w = synth.WORKLOADS[name]
    p = synth.make_problem(w)
    p.update(N=w.N, L=w.L, R=w.R, T=w.T)
    return w, p


def kplanes_pack(params):
    """Flat parameter vector in the C ABI's K-Planes layout (per scale: the six
    planes in oracle order, then a)."""
    from oracle.kplanes import PLANES
    parts = []
    for s in range(len(params["planes"])):
        for c in PLANES:
            parts.append(np.asarray(params["planes"][s][c]).reshape(-1))
        parts.append(np.asarray(params["a"][s]).reshape(-1))
    return np.concatenate(parts)


def kplanes_unpack(flat, like):
    """Inverse of ``kplanes_pack`` with the shapes of ``like``."""
    from oracle.kplanes import PLANES
    out = {"planes": [], "a": []}
    o = 0
    for s in range(len(like["planes"])):
        d = {}
        for c in PLANES:
            sh = like["planes"][s][c].shape
            n = int(np.prod(sh))
            d[c] = np.asarray(flat[o:o + n]).reshape(sh)
            o += n
        out["planes"].append(d)
        n = like["a"][s].size
        out["a"].append(np.asarray(flat[o:o + n]))
        o += n
    assert o == len(flat)
    return out
