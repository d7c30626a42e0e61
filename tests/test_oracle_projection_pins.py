"""Pins of the projection-model oracle (the paper's own forward model, Sec.
4.2-4.3) against things other than itself (no GPU): shifts that reduce to
rolls and averages, the independent gather/scatter pair as an adjoint
identity, numpy's FFT against the non-uniform DFT oracle on a Cartesian
blade, the blade mask's lattice and area, the two models agreeing where they
must, and the loss gradient against finite differences.
"""
import numpy as np
import pytest

import oracle
from oracle import projection as pj
from oracle.geometry import make_geometry


def _rand_c(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_zero_shift_projection_sums_the_bins():
    rng = np.random.default_rng(1)
    V = _rand_c(rng, (8, 8, 3))
    I = pj.project(V, np.zeros((3, 2)))
    assert np.allclose(I, V.sum(axis=2), atol=1e-14)


@pytest.mark.parametrize("d", [3, -2])
def test_integer_shift_is_a_zero_filled_translation(d):
    """theta = 0 moves bin contents by +Delta along x1, theta = 90 deg along x2;
    what enters from outside the image is zero (no wrap-around)."""
    rng = np.random.default_rng(2)
    N = 10
    V = _rand_c(rng, (N, N, 1))
    g0 = make_geometry(N, 4, N, [0.0], [float(d)])
    I = pj.project(V, pj.shifts(g0, 0))
    ref = np.zeros((N, N), dtype=complex)
    if d > 0:
        ref[:, d:] = V[:, :-d, 0]
    else:
        ref[:, :d] = V[:, -d:, 0]
    assert np.allclose(I, ref, atol=1e-12)
    g90 = make_geometry(N, 4, N, [np.pi / 2], [float(d)])
    I = pj.project(V, pj.shifts(g90, 0))
    ref = np.zeros((N, N), dtype=complex)
    if d > 0:
        ref[d:, :] = V[:-d, :, 0]
    else:
        ref[:d, :] = V[-d:, :, 0]
    assert np.allclose(I, ref, atol=1e-12)


def test_half_pixel_shift_averages_neighbours():
    rng = np.random.default_rng(3)
    N = 9
    V = _rand_c(rng, (N, N, 1))
    I = pj.project(V, np.array([[0.5, 0.0]]))
    ref = 0.5 * V[:, :, 0]
    ref[:, 1:] += 0.5 * V[:, :-1, 0]
    assert np.allclose(I, ref, atol=1e-12)


def test_projection_gather_and_scatter_are_adjoint():
    """project (a gather) and project_adjoint (np.add.at scatter) are written
    independently: <P V, z> = <V, P^H z> for random fractional shifts."""
    rng = np.random.default_rng(4)
    N, Nf = 12, 4
    V = _rand_c(rng, (N, N, Nf))
    z = _rand_c(rng, (N, N))
    s = rng.uniform(-3.7, 3.7, size=(Nf, 2))
    lhs = np.vdot(z, pj.project(V, s))
    rhs = np.vdot(pj.project_adjoint(z, s, Nf), V)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("N", [8, 12])
def test_centred_dft_is_the_nonuniform_dft_on_a_cartesian_blade(N):
    """theta = 0, L = R = N, one bin at Delta = 0: the blade's samples are the
    Cartesian grid, so numpy's FFT step must reproduce the NDFT oracle."""
    rng = np.random.default_rng(5)
    V = _rand_c(rng, (1, N, N, 1))
    g = make_geometry(N, N, N, [0.0], [0.0])
    y = oracle.forward(V, g)[0]                 # [l, j] = [u2, u1]
    Z = pj.dft(V[0, :, :, 0])
    assert np.allclose(Z, y, atol=1e-12 * np.abs(y).max())
    assert np.allclose(pj.idft(Z), V[0, :, :, 0], atol=1e-12)
    assert abs(np.linalg.norm(Z) - np.linalg.norm(V)) < 1e-12 * np.linalg.norm(V)


@pytest.mark.parametrize("th", [0.0, np.pi / 2])
@pytest.mark.parametrize("L,R", [(4, 8), (6, 16), (8, 10)])
def test_mask_at_0_and_90_degrees_is_the_blade_lattice(L, R, th):
    """With even L and R at 0 or 90 degrees the blade's samples sit on
    Cartesian cells: the mask is exactly those cells (sample positions taken
    from the non-uniform oracle's geometry, a separate code path)."""
    N = 16
    m = pj.blade_mask(N, th, L, R)
    g = make_geometry(N, L, R, [th], [0.0])
    k1, k2, _ = oracle.sample_coords(g)
    cells = {(int(round(N * b)) + N // 2, int(round(N * a)) + N // 2) for a, b in zip(k1, k2)}
    got = {(int(a), int(b)) for a, b in zip(*np.nonzero(m))}
    assert got == cells
    assert m.sum() == L * R


@pytest.mark.parametrize("L,R", [(5, 7), (3, 9)])
def test_mask_for_odd_blade_sizes_keeps_the_sample_count(L, R):
    for th in (0.0, np.pi / 2):
        assert pj.blade_mask(16, th, L, R).sum() == L * R


def test_mask_area_tracks_the_blade_rectangle():
    for th in np.linspace(0.1, 3.0, 7):
        m = pj.blade_mask(64, th, 12, 48)
        assert abs(int(m.sum()) - 12 * 48) <= 2 * (12 + 48)


@pytest.mark.parametrize("delta", [2.0, -3.0])
def test_integer_shift_agrees_with_the_nonuniform_model(delta):
    """theta = 0, L = R = N, integer Delta and an object away from the edges:
    the zero-filled interpolated shift and the Fourier phase of the
    non-uniform model are the same translation."""
    rng = np.random.default_rng(6)
    N = 16
    V = np.zeros((1, N, N, 2), dtype=complex)
    V[0, 4:12, 4:12, :] = _rand_c(rng, (8, 8, 2))
    g = make_geometry(N, N, N, [0.0], [0.0, delta])
    y_nu = oracle.forward(V, g)[0]
    y_pj = pj.forward(V, g, 0)
    assert np.allclose(y_pj, y_nu, atol=1e-12 * np.abs(y_nu).max())


def test_forward_and_adjoint_are_adjoint():
    rng = np.random.default_rng(7)
    N, Nf, T = 12, 3, 2
    g = make_geometry(N, 6, 10, [0.3, 1.9], [-1.2, 0.4, 2.7], [1, 0], T)
    V = _rand_c(rng, (T, N, N, Nf))
    z = _rand_c(rng, (N, N))
    for b in range(2):
        lhs = np.vdot(z, pj.forward(V, g, b))
        rhs = np.vdot(pj.adjoint(z, g, b), V)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_loss_gradient_matches_finite_differences():
    """All terms on (both data terms with an independent image, TV in x-y,
    along the spectrum and in time, L1) on a two-frame volume."""
    rng = np.random.default_rng(8)
    N, Nf, T = 8, 3, 2
    g = make_geometry(N, 4, 6, [0.4, 2.2], [-1.3, 0.2, 1.6], [0, 1], T)
    V = 0.3 * _rand_c(rng, (T, N, N, Nf))
    ycart = _rand_c(rng, (2, N, N))
    img = _rand_c(rng, (2, N, N))
    p = pj.ProjParams(w_kspace=0.3, w_image=1.1, tv_xy=0.05, tv_f=0.07, tv_t=0.04, l1=0.02, tv_eps=0.1)
    for b in range(2):
        L0, G = pj.loss_and_grad(V, ycart, img, g, b, p)
        for _ in range(3):
            D = _rand_c(rng, V.shape)
            h = 1e-6
            Lp, _ = pj.loss_and_grad(V + h * D, ycart, img, g, b, p)
            Lm, _ = pj.loss_and_grad(V - h * D, ycart, img, g, b, p)
            fd = (Lp - Lm) / (2 * h)
            an = float(np.sum(G.real * D.real + G.imag * D.imag))
            assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (fd, an)


def test_default_image_is_the_masked_inverse_dft():
    """Without an image the image term equals the k-space term on the mask
    (the DFT is unitary), so the two weights simply add."""
    rng = np.random.default_rng(9)
    N = 8
    g = make_geometry(N, 4, 6, [0.7], [0.0, 1.0])
    V = _rand_c(rng, (1, N, N, 2))
    ycart = _rand_c(rng, (1, N, N))
    p1 = pj.ProjParams(w_kspace=0.0, w_image=1.0, tv_xy=0.0)
    p2 = pj.ProjParams(w_kspace=1.0, w_image=0.0, tv_xy=0.0)
    L1, G1 = pj.loss_and_grad(V, ycart, None, g, 0, p1)
    L2, G2 = pj.loss_and_grad(V, ycart, None, g, 0, p2)
    assert abs(L1 - L2) < 1e-12 * L2
    assert np.allclose(G1, G2, atol=1e-12 * np.abs(G2).max())


def test_reconstruction_fits_blade_data_of_a_known_volume():
    """Data made by the forward model from a volume: the loss of each blade
    falls over two passes through the blades."""
    rng = np.random.default_rng(10)
    N, Nf = 16, 2
    g = make_geometry(N, 6, 16, np.pi * np.arange(4) / 4, [0.0, 1.5])
    Vt = np.zeros((1, N, N, Nf), dtype=complex)
    Vt[0, 4:12, 5:11, 0] = 1.0
    Vt[0, 6:9, 6:10, 1] = 0.5
    ycart = np.stack([pj.forward(Vt, g, b) for b in range(4)])
    p = pj.ProjParams(iters=40, lr=0.05, tv_xy=0.0)
    V, tr = pj.reconstruct(ycart, None, g, p)
    assert tr[-4:].sum() < 0.2 * tr[:4].sum()


def test_baseline_of_one_blade_is_its_image():
    rng = np.random.default_rng(11)
    N = 12
    g = make_geometry(N, 4, 8, [0.4, 1.3], [0.0])
    ycart = _rand_c(rng, (2, N, N))
    assert np.allclose(pj.baseline(ycart, g, 1, 2), pj.image_of(ycart, g, 1), atol=1e-12)


def test_baseline_averages_overlapping_blades():
    """Blades whose data agree give that data on the union of their masks;
    where only one blade covers a cell its value is kept, where two do the
    mean of the two."""
    rng = np.random.default_rng(12)
    N = 16
    g = make_geometry(N, 6, 12, [0.0, np.pi / 2], [0.0])
    y = _rand_c(rng, (N, N))
    z = _rand_c(rng, (N, N))
    m0 = pj.blade_mask(N, 0.0, 6, 12)
    m1 = pj.blade_mask(N, np.pi / 2, 6, 12)
    same = pj.dft(pj.baseline(np.stack([y, y]), g))
    assert np.allclose(same, y * (m0 | m1), atol=1e-12)
    mix = pj.dft(pj.baseline(np.stack([y, z]), g))
    ref = np.where(m0 & m1, 0.5 * (y + z), np.where(m0, y, np.where(m1, z, 0)))
    assert np.allclose(mix, ref, atol=1e-12)
