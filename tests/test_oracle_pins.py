"""Pins of the FP64 oracle against things other than itself (no GPU).

Each test checks one part of the oracle against a library special case, a
closed form, an invariant or brute force, chosen so that a plausible mistake
(a dropped term, a wrong sign or index, a transposed operand, a wrong scale)
fails at least one of them.
"""
import cmath
import math

import numpy as np
import pytest
import torch
from scipy.integrate import dblquad

import oracle
from oracle.geometry import make_geometry
from synth.phantom import Ellipse, ellipse_ft, rasterize


def _rand_c(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# --- forward: sign, centring and scale -------------------------------------

@pytest.mark.parametrize("N", [8, 16])
def test_forward_is_centred_fft2_at_theta0(N):
    """Delta = 0, theta = 0, L = R = N: the operator is the centred, orthonormal 2-D DFT."""
    rng = np.random.default_rng(0)
    img = _rand_c(rng, (N, N))
    g = make_geometry(N, N, N, [0.0], [0.0])
    y = oracle.forward(img[None, :, :, None], g)[0]          # [l, j]
    ref = np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(img))) / N   # [q2, q1]
    # theta = 0: k1 = k_r (column j), k2 = k_p (line l).
    assert np.max(np.abs(y - ref)) < 1e-12 * np.max(np.abs(ref))


def test_forward_is_transposed_fft2_at_theta90():
    """theta = 90 deg: readout runs along +x2 and the line axis along -x1."""
    N = 16
    rng = np.random.default_rng(1)
    img = _rand_c(rng, (N, N))
    g = make_geometry(N, N, N, [math.pi / 2], [0.0])
    y = oracle.forward(img[None, :, :, None], g)[0]
    F = np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(img))) / N     # F[q2 + N/2, q1 + N/2]
    l = np.arange(N)[:, None]
    j = np.arange(N)[None, :]
    ref = F[j, (N - l) % N]            # k2 = k_r -> q2 = j - N/2 ; k1 = -k_p -> q1 = N/2 - l
    assert np.max(np.abs(y - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("theta,axis", [(0.0, 2), (math.pi / 2, 1)])
def test_integer_displacement_translates_along_readout(theta, axis):
    """Shift theorem: a bin displaced by Delta = +3 px equals the undisplaced image
    rolled by +3 px along the readout direction (x1 at 0 deg, x2 at 90 deg).
    With L = R = N every sample frequency is a multiple of 1/N, so the roll is exact."""
    N = 16
    rng = np.random.default_rng(2)
    img = _rand_c(rng, (N, N))
    g3 = make_geometry(N, N, N, [theta], [3.0])
    g0 = make_geometry(N, N, N, [theta], [0.0])
    y3 = oracle.forward(img[None, :, :, None], g3)
    rolled = np.roll(img, 3, axis=axis - 1)
    y0 = oracle.forward(rolled[None, :, :, None], g0)
    assert np.max(np.abs(y3 - y0)) < 1e-11 * np.max(np.abs(y0))
    # and the opposite sign is detectably different
    y0m = oracle.forward(np.roll(img, -3, axis=axis - 1)[None, :, :, None], g0)
    assert np.max(np.abs(y3 - y0m)) > 1e-2 * np.max(np.abs(y0))


def test_single_voxel_is_pure_phase_ramp():
    """A single voxel a at (x0, f0) gives y_b(k) = a/N exp(-2 pi i k.(x0 + Delta_f0 d_b))."""
    N, L, R = 16, 4, 16
    theta = [0.37, 2.1]
    delta = [-1.5, 0.25, 2.0]
    g = make_geometry(N, L, R, theta, delta)
    V = np.zeros((1, N, N, 3), dtype=complex)
    a = 0.7 - 0.4j
    i2, i1, f0 = 11, 3, 2
    V[0, i2, i1, f0] = a
    y = oracle.forward(V, g)
    x0 = (i1 - N / 2, i2 - N / 2)
    for b, th in enumerate(theta):
        for l in range(L):
            for j in range(R):
                kr, kp = (j - R / 2) / N, (l - L / 2) / N
                k = (kr * math.cos(th) - kp * math.sin(th), kr * math.sin(th) + kp * math.cos(th))
                p = (x0[0] + delta[f0] * math.cos(th), x0[1] + delta[f0] * math.sin(th))
                ref = a / N * cmath.exp(-2j * math.pi * (k[0] * p[0] + k[1] * p[1]))
                assert abs(y[b, l, j] - ref) < 1e-13


# --- brute force: the whole matrix on an 8 x 8 grid -------------------------

def test_bruteforce_matrix_8x8():
    """Assemble A entry by entry from the displaced-position form
    exp(-2 pi i k.(x + Delta_f d_b)) and compare both operators with it."""
    N, L, R = 8, 2, 8
    theta = [0.3, 1.9]
    delta = [-1.0, 0.4, 1.7]
    frames = [0, 1]
    g = make_geometry(N, L, R, theta, delta, frames, T=2)
    nvox = 2 * N * N * 3
    A = np.zeros((g.M, nvox), dtype=complex)
    m = 0
    for b, th in enumerate(theta):
        d = (math.cos(th), math.sin(th))
        dp = (-math.sin(th), math.cos(th))
        for l in range(L):
            for j in range(R):
                kr, kp = (j - R / 2) / N, (l - L / 2) / N
                k = (kr * d[0] + kp * dp[0], kr * d[1] + kp * dp[1])
                for i2 in range(N):
                    for i1 in range(N):
                        for f in range(3):
                            p1 = (i1 - N // 2) + delta[f] * d[0]
                            p2 = (i2 - N // 2) + delta[f] * d[1]
                            col = ((frames[b] * N + i2) * N + i1) * 3 + f
                            A[m, col] = cmath.exp(-2j * math.pi * (k[0] * p1 + k[1] * p2)) / N
                m += 1
    rng = np.random.default_rng(3)
    V = _rand_c(rng, (2, N, N, 3))
    y = _rand_c(rng, (2, L, R))
    assert np.allclose(oracle.forward(V, g).reshape(-1), A @ V.reshape(-1), rtol=0, atol=1e-12)
    assert np.allclose(oracle.adjoint(y, g).reshape(-1), A.conj().T @ y.reshape(-1), rtol=0, atol=1e-12)


# --- invariants ---------------------------------------------------------------

@pytest.mark.parametrize("T", [1, 3])
def test_adjoint_identity(T):
    """<A x, y> = <x, A^H y> for random complex x, y (static and multi-frame)."""
    N, L, R = 24, 6, 24
    rng = np.random.default_rng(4 + T)
    B = 5
    g = make_geometry(N, L, R, rng.uniform(0, math.pi, B), np.linspace(-3, 3, 4),
                      rng.integers(0, T, B), T=T)
    x = _rand_c(rng, (T, N, N, 4))
    y = _rand_c(rng, (B, L, R))
    lhs = np.vdot(y.reshape(-1), oracle.forward(x, g).reshape(-1))
    rhs = np.vdot(oracle.adjoint(y, g).reshape(-1), x.reshape(-1))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_sampled_evaluations_match_full_operators():
    N, L, R = 16, 4, 16
    rng = np.random.default_rng(5)
    g = make_geometry(N, L, R, [0.1, 0.9, 2.5], [-1.0, 1.0], [0, 1, 1], T=2)
    V = _rand_c(rng, (2, N, N, 2))
    y = _rand_c(rng, (3, L, R))
    s = rng.choice(g.M, 40, replace=False)
    assert np.allclose(oracle.forward_at(V, g, s), oracle.forward(V, g).reshape(-1)[s], atol=1e-12)
    q = rng.choice(V.size, 50, replace=False)
    assert np.allclose(oracle.adjoint_at(y, g, q), oracle.adjoint(y, g).reshape(-1)[q], atol=1e-12)


# --- data generator vs operator conventions ------------------------------------

def test_ellipse_closed_form_matches_quadrature():
    """The Bessel closed form of the ellipse FT against direct 2-D quadrature."""
    e = Ellipse((5.3, -7.1), (14.2, 9.7), 0.6, 1.0, 0.0)
    ca, sa = math.cos(e.angle), math.sin(e.angle)
    for k in [(0.0, 0.0), (0.03, -0.05), (0.11, 0.07)]:
        def f(v, u, part):
            x1 = e.center[0] + ca * e.axes[0] * u - sa * e.axes[1] * v
            x2 = e.center[1] + sa * e.axes[0] * u + ca * e.axes[1] * v
            ph = -2 * math.pi * (k[0] * x1 + k[1] * x2)
            return (math.cos(ph) if part == 0 else math.sin(ph)) * e.axes[0] * e.axes[1]
        lo = lambda u: -math.sqrt(1 - u * u)
        hi = lambda u: math.sqrt(1 - u * u)
        ref = dblquad(f, -1, 1, lo, hi, args=(0,), epsabs=1e-10)[0] + \
            1j * dblquad(f, -1, 1, lo, hi, args=(1,), epsabs=1e-10)[0]
        val = complex(ellipse_ft(np.array(k[0]), np.array(k[1]), e))
        assert abs(val - ref) < 1e-8 * max(1.0, abs(ref))


def test_operator_matches_analytic_ellipse_ft_with_supersampling():
    """NDFT of a box-averaged raster -> (1/N) FT(ellipse) sinc(k1) sinc(k2) at low |k|,
    with the error shrinking as the raster is supersampled (convention check: a
    wrong sign, centre or scale is off by O(1))."""
    N = 64
    e = Ellipse((5.3, -7.1), (14.2, 9.7), 0.6, 0.8 * np.exp(0.7j), 0.0)
    g = make_geometry(N, 8, N, [0.3, 1.9], [0.0])
    k1, k2, _ = oracle.sample_coords(g)
    sel = np.nonzero(np.hypot(k1, k2) < 0.12)[0]
    ref = ellipse_ft(k1[sel], k2[sel], e) * e.rho / N * np.sinc(k1[sel]) * np.sinc(k2[sel])
    errs = []
    for s in (1, 8):
        w, _ = rasterize([e], N, s)
        y = oracle.forward_at(w[None, :, :, None], g, sel)
        errs.append(np.linalg.norm(y - ref) / np.linalg.norm(ref))
    assert errs[1] < 5e-3 and errs[1] < 0.5 * errs[0]
    w, _ = rasterize([e], N, 8)
    y = oracle.forward_at(w[None, :, :, None], g, sel)
    assert np.linalg.norm(np.conj(y) - ref) / np.linalg.norm(ref) > 0.5


# --- regularisers, loss gradient, Adam ----------------------------------------------

def test_tv_gradients_match_central_differences():
    rng = np.random.default_rng(6)
    V = _rand_c(rng, (3, 5, 6, 2)) * 0.1
    eps = 1e-3
    for fn in (oracle.tv_xy, oracle.tv_t):
        _, grad = fn(V, eps)
        h = 1e-6
        for _ in range(12):
            idx = tuple(rng.integers(0, n) for n in V.shape)
            for unit, part in ((1.0, grad[idx].real), (1j, grad[idx].imag)):
                Vp = V.copy(); Vp[idx] += h * unit
                Vm = V.copy(); Vm[idx] -= h * unit
                fd = (fn(Vp, eps)[0] - fn(Vm, eps)[0]) / (2 * h)
                assert abs(fd - part) < 1e-6 * max(1.0, abs(part))


def test_tv_values_closed_form():
    """Constant volume: every difference is 0, so TV = eps * (number of differences)."""
    V = np.full((2, 4, 5, 3), 0.3 + 0.2j)
    eps = 1e-3
    assert abs(oracle.tv_xy(V, eps)[0] - eps * 2 * 3 * (4 * 4 + 3 * 5)) < 1e-15
    assert abs(oracle.tv_t(V, eps)[0] - eps * 1 * 4 * 5 * 3) < 1e-15
    # one nonzero voxel (|3+4i| = 5) in a 2 x 3 image: one x1 difference and one
    # x2 difference of magnitude 5, the other 3 + 2 differences are 0
    W = np.zeros((1, 2, 3, 1), dtype=complex)
    W[0, 0, 2, 0] = 3 + 4j
    v = oracle.tv_xy(W, eps)[0]
    terms_x1 = [abs(W[0, r, c + 1, 0] - W[0, r, c, 0]) for r in range(2) for c in range(2)]
    terms_x2 = [abs(W[0, 1, c, 0] - W[0, 0, c, 0]) for c in range(3)]
    ref = sum(math.hypot(t, eps) for t in terms_x1 + terms_x2)
    assert abs(v - ref) < 1e-12 and abs(v - (2 * math.hypot(5, eps) + 5 * eps)) < 1e-12


def test_loss_gradient_matches_finite_differences():
    """dL/dRe + i dL/dIm against central differences along random directions
    (the data term is quadratic, so its central difference is exact up to rounding)."""
    N, L, R = 12, 4, 12
    rng = np.random.default_rng(7)
    g = make_geometry(N, L, R, [0.2, 1.3, 2.2], [-1.0, 0.5], [0, 0, 1], T=2)
    V = _rand_c(rng, (2, N, N, 2)) * 0.2
    y = _rand_c(rng, (3, L, R))
    p = oracle.ReconParams(tv_xy=0.05, tv_t=0.02, tv_eps=0.1)
    loss, grad = oracle.loss_and_grad(V, y, g, p)
    for _ in range(4):
        D = _rand_c(rng, V.shape)
        D /= np.linalg.norm(D)
        h = 1e-4
        lp, _ = oracle.loss_and_grad(V + h * D, y, g, p)
        lm, _ = oracle.loss_and_grad(V - h * D, y, g, p)
        fd = (lp - lm) / (2 * h)
        an = float(np.sum(grad.real * D.real + grad.imag * D.imag))
        assert abs(fd - an) < 1e-6 * max(1.0, abs(an))
    # data term alone: gradient is 2 A^H (A V - y) (closed form)
    p0 = oracle.ReconParams(tv_xy=0.0, tv_t=0.0)
    _, g0 = oracle.loss_and_grad(V, y, g, p0)
    r = oracle.forward(V, g) - y
    assert np.allclose(g0, 2 * oracle.adjoint(r, g), atol=1e-12)


def test_adam_matches_torch_optim_adam():
    """The oracle's Adam against torch.optim.Adam (float64, complex parameter)."""
    rng = np.random.default_rng(8)
    V0 = _rand_c(rng, (1, 3, 4, 2))
    p = oracle.ReconParams(lr=3e-2, beta1=0.85, beta2=0.99, eps=1e-6)
    prm = torch.nn.Parameter(torch.tensor(V0, dtype=torch.complex128))
    opt = torch.optim.Adam([prm], lr=p.lr, betas=(p.beta1, p.beta2), eps=p.eps)
    V = V0.copy()
    m = np.zeros(V.shape + (2,))
    v = np.zeros(V.shape + (2,))
    for k in range(1, 6):
        G = _rand_c(rng, V.shape)
        opt.zero_grad()
        prm.grad = torch.tensor(G, dtype=torch.complex128)
        opt.step()
        V, m, v = oracle.adam_step(V, G, m, v, k, p)
        assert np.max(np.abs(V - prm.detach().numpy())) < 1e-13
    # first step moves each real component by -lr * g/(|g| + eps)
    G = _rand_c(rng, V0.shape)
    V1, _, _ = oracle.adam_step(V0, G, np.zeros(V0.shape + (2,)), np.zeros(V0.shape + (2,)), 1, p)
    step = V0 - V1
    assert np.allclose(step.real, p.lr * G.real / (np.abs(G.real) + p.eps), atol=1e-15)
    assert np.allclose(step.imag, p.lr * G.imag / (np.abs(G.imag) + p.eps), atol=1e-15)


def test_render_and_split():
    rng = np.random.default_rng(9)
    V = _rand_c(rng, (2, 3, 3, 5))
    assert np.allclose(oracle.render(V), V.sum(-1))
    assert np.allclose(oracle.render(V, 0, 2) + oracle.render(V, 2, 5), oracle.render(V))


# --- PSNR (Sec. 6, Table 1) -------------------------------------------------

def test_psnr_closed_form():
    """|image| = (1 + d) |ref| on a constant-magnitude reference c: the error is
    c d everywhere, so PSNR = 10 log10(c^2 / (c d)^2) = -20 log10 d exactly;
    a phase change alone leaves the magnitudes equal (PSNR at the rounding
    floor, and +inf for identical magnitudes)."""
    rng = np.random.default_rng(10)
    phase = np.exp(2j * np.pi * rng.uniform(size=(3, 16, 16)))
    c = 2.5
    ref = c * phase
    for d in (0.1, 0.01, 3e-4):
        assert abs(oracle.psnr((1 + d) * ref, ref) - (-20.0 * math.log10(d))) < 1e-9
    assert oracle.psnr(ref * np.exp(0.7j), ref) > 250.0
    assert oracle.psnr(ref, ref) == float("inf")


def test_psnr_brute_force_and_peak_of_reference():
    """Against a loop over the pixels; the peak is the reference's, not the image's."""
    rng = np.random.default_rng(11)
    ref = _rand_c(rng, (5, 7))
    img = ref + 0.1 * _rand_c(rng, (5, 7))
    se, pk = 0.0, 0.0
    for a, b in zip(img.ravel(), ref.ravel()):
        se += (abs(a) - abs(b)) ** 2
        pk = max(pk, abs(b))
    ref_val = 10 * math.log10(pk * pk / (se / ref.size))
    assert abs(oracle.psnr(img, ref) - ref_val) < 1e-10
    assert abs(oracle.psnr(img, ref) - oracle.psnr(ref, img)) > 1e-3   # not symmetric: the peak is the reference's
