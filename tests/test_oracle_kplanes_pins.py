"""Pins of the K-Planes volume model oracle (Sec. 4.1, Eq. 3) against
things other than itself (no GPU): plane lookups at full resolution equal
direct indexing, the six-way product and the weighting by a, exact
reproduction of linear planes by the half-resolution interpolation (with
clamping at the borders), additivity over scales, and the parameter
gradients against finite differences.
"""
import numpy as np
import pytest

from oracle import kplanes as kp


def _rand_c(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _ones(N, Nf, T, F, scales=1):
    return {"planes": [{c: np.ones(sh, dtype=complex) for c, sh in kp.plane_shapes(N, Nf, T, F, s).items()}
                       for s in range(scales)],
            "a": [np.zeros(F, dtype=complex) for _ in range(scales)]}


def test_full_resolution_planes_are_looked_up_directly():
    """One scale, random planes, a = e_k: V equals the product of the six
    planes indexed at the voxel's own coordinates."""
    rng = np.random.default_rng(1)
    N, Nf, T, F = 6, 3, 2, 4
    prm = _ones(N, Nf, T, F)
    for c in kp.PLANES:
        prm["planes"][0][c] = _rand_c(rng, prm["planes"][0][c].shape)
    for k in range(F):
        prm["a"][0] = np.eye(F)[k].astype(complex)
        V = kp.render(prm, N, Nf, T)
        P = prm["planes"][0]
        t, y, x, w = 1, 4, 2, 2
        ref = (P["xy"][y, x, k] * P["xw"][w, x, k] * P["xt"][t, x, k] * P["yw"][w, y, k] * P["yt"][t, y, k]
               * P["wt"][t, w, k])
        assert abs(V[t, y, x, w] - ref) < 1e-12
        full = np.einsum("yx,wx,tx,wy,ty,tw->tyxw", P["xy"][..., k], P["xw"][..., k], P["xt"][..., k],
                         P["yw"][..., k], P["yt"][..., k], P["wt"][..., k])
        assert np.allclose(V, full, atol=1e-12)


def test_weighting_vector_is_a_plain_inner_product():
    rng = np.random.default_rng(2)
    N, Nf, T, F = 4, 2, 1, 5
    prm = _ones(N, Nf, T, F)
    prm["planes"][0]["xy"] = _rand_c(rng, (N, N, F))
    prm["a"][0] = _rand_c(rng, F)
    V = kp.render(prm, N, Nf, T)
    ref = prm["planes"][0]["xy"] @ prm["a"][0]      # no conjugation of a
    assert np.allclose(V[0, :, :, 0], ref, atol=1e-12)
    assert np.allclose(V[0, :, :, 1], ref, atol=1e-12)


def test_half_resolution_reproduces_linear_planes_and_clamps():
    """A half-resolution xy plane that is linear in its node coordinates is
    reproduced exactly inside; beyond the outer node centres the value is
    held (clamping)."""
    N, F = 8, 1
    n = N // 2
    prm = _ones(N, 1, 1, F, scales=2)
    prm["a"] = [np.zeros(F, dtype=complex), np.ones(F, dtype=complex)]
    j = np.arange(n, dtype=float)
    prm["planes"][1]["xy"] = (0.7 * j[None, :] - 1.3j * j[:, None])[..., None]
    V = kp.render(prm, N, 1, 1)[0, :, :, 0]
    u = np.clip((np.arange(N) + 0.5) / 2 - 0.5, 0, n - 1)
    ref = 0.7 * u[None, :] - 1.3j * u[:, None]
    assert np.allclose(V, ref, atol=1e-12)
    assert np.isclose(V[0, 0], 0.0) and np.isclose(V[0, 1], 0.7 * 0.25)


def test_scales_add():
    rng = np.random.default_rng(3)
    N, Nf, T = 8, 2, 2
    prm = kp.init_params(N, Nf, T, rng, F=3)
    both = kp.render(prm, N, Nf, T)
    s0 = kp.render({"planes": prm["planes"][:1], "a": prm["a"][:1]}, N, Nf, T)
    s1 = kp.render({"planes": prm["planes"][1:], "a": prm["a"][1:]}, N, Nf, T)
    assert np.allclose(both, s0 + s1, atol=1e-12)


def test_parameter_gradients_match_finite_differences():
    rng = np.random.default_rng(4)
    N, Nf, T, F = 6, 3, 2, 3
    prm = kp.init_params(N, Nf, T, rng, F=F, spread=0.3)
    W = _rand_c(rng, (T, N, N, Nf))

    def loss(q):
        V = kp.render(q, N, Nf, T)
        return float(np.sum(np.abs(V - W) ** 2))

    V = kp.render(prm, N, Nf, T)
    G = kp.vjp(prm, 2.0 * (V - W), N, Nf, T)
    h = 1e-6
    for s in range(2):
        for c in kp.PLANES + ("a",):
            base = prm["a"][s] if c == "a" else prm["planes"][s][c]
            D = _rand_c(rng, base.shape)
            g = G["a"][s] if c == "a" else G["planes"][s][c]

            def shifted(sign):
                q = {"planes": [dict(d) for d in prm["planes"]], "a": list(prm["a"])}
                if c == "a":
                    q["a"][s] = base + sign * h * D
                else:
                    q["planes"][s][c] = base + sign * h * D
                return q

            fd = (loss(shifted(+1)) - loss(shifted(-1))) / (2 * h)
            an = float(np.sum(g.real * D.real + g.imag * D.imag))
            assert abs(fd - an) < 1e-5 * max(1.0, abs(an)), (s, c, fd, an)


def test_gradients_through_the_data_loss():
    """The model composed with the non-uniform data term and TV: parameter
    gradients against central differences along random directions."""
    import oracle
    from oracle.geometry import make_geometry
    rng = np.random.default_rng(5)
    N, Nf, T, F = 8, 2, 2, 3
    g = make_geometry(N, 4, 8, [0.2, 1.4], [-1.0, 1.5], [0, 1], T)
    y = _rand_c(rng, (2, 4, 8))
    p = oracle.ReconParams(tv_xy=0.05, tv_t=0.03, tv_eps=0.1)
    prm = kp.init_params(N, Nf, T, rng, F=F, spread=0.3)
    L0, G = kp.loss_and_grad(prm, y, g, p)
    h = 1e-6
    for s, c in ((0, "xy"), (1, "wt"), (0, "yt")):
        D = _rand_c(rng, prm["planes"][s][c].shape)

        def at(sign):
            q = {"planes": [dict(d) for d in prm["planes"]], "a": list(prm["a"])}
            q["planes"][s][c] = prm["planes"][s][c] + sign * h * D
            return kp.loss_and_grad(q, y, g, p)[0]

        fd = (at(+1) - at(-1)) / (2 * h)
        gg = G["planes"][s][c]
        an = float(np.sum(gg.real * D.real + gg.imag * D.imag))
        assert abs(fd - an) < 1e-5 * max(1.0, abs(an)), (s, c, fd, an)
