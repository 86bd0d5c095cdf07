"""Pins of oracle.sht (no GPU): scipy harmonics, exact GL round trips, adjointness."""
import numpy as np
import pytest
from scipy.special import sph_harm_y

from oracle import alm, grids, sht
from oracle.legendre import lambda_all, lambda_m


def _real_Y_scipy(grid, lmax):
    th, ph = grid.pixel_angles()
    ell, ms = alm.layout(lmax)
    Y = np.empty((grid.npix, ell.size))
    for i, (l, m) in enumerate(zip(ell, ms)):
        c = ((-1) ** abs(m)) * sph_harm_y(l, abs(m), th, ph)
        if m == 0:
            Y[:, i] = c.real
        elif m > 0:
            Y[:, i] = np.sqrt(2) * c.real
        else:
            Y[:, i] = np.sqrt(2) * c.imag
    return Y


@pytest.mark.parametrize("grid,lmax", [(grids.healpix(4), 11), (grids.gauss_legendre(9), 9),
                                       (grids.healpix(3), 12)])
def test_dense_Y_matches_scipy(grid, lmax):
    np.testing.assert_allclose(sht.dense_Y(grid, lmax), _real_Y_scipy(grid, lmax), atol=1e-12)


def test_low_order_modes_closed_form():
    g = grids.healpix(8)
    th, ph = g.pixel_angles()
    L = 4
    ell, ms = alm.layout(L)
    cases = [((1, 0), np.sqrt(3 / (4 * np.pi)) * np.cos(th)),
             ((1, 1), np.sqrt(3 / (4 * np.pi)) * np.sin(th) * np.cos(ph)),
             ((1, -1), np.sqrt(3 / (4 * np.pi)) * np.sin(th) * np.sin(ph)),
             ((2, 2), np.sqrt(15 / (16 * np.pi)) * np.sin(th) ** 2 * np.cos(2 * ph)),
             ((0, 0), np.full(th.shape, np.sqrt(1 / (4 * np.pi))))]
    for (l, m), ref in cases:
        a = np.zeros(ell.size)
        a[np.flatnonzero((ell == l) & (ms == m))[0]] = 1.0
        np.testing.assert_allclose(sht.synthesis(g, L, a), ref, atol=1e-14)


@pytest.mark.parametrize("grid,lmax", [(grids.healpix(4), 11), (grids.healpix(5), 14),
                                       (grids.gauss_legendre(12), 12),
                                       (grids.gauss_legendre(7, nphi=20), 7)])
def test_ring_factored_equals_dense(grid, lmax):
    rng = np.random.default_rng(1)
    Y = sht.dense_Y(grid, lmax)
    a = rng.standard_normal(Y.shape[1])
    f = rng.standard_normal(Y.shape[0])
    np.testing.assert_allclose(sht.synthesis(grid, lmax, a), Y @ a, atol=1e-12)
    np.testing.assert_allclose(sht.adjoint(grid, lmax, f), Y.T @ f, atol=1e-11)
    w = grid.pixel_weights()
    np.testing.assert_allclose(sht.analysis(grid, lmax, f), Y.T @ (w * f), atol=1e-12)


@pytest.mark.parametrize("lmax", [7, 31, 63])
def test_gl_round_trip_exact(lmax):
    g = grids.gauss_legendre(lmax)
    a = np.random.default_rng(lmax).standard_normal((lmax + 1) ** 2)
    back = sht.analysis(g, lmax, sht.synthesis(g, lmax, a))
    np.testing.assert_allclose(back, a, atol=1e-12 * np.abs(a).max())


def test_gl_singular_values_unity():
    lmax = 10
    g = grids.gauss_legendre(lmax)
    Y = sht.dense_Y(g, lmax)
    s = np.linalg.svd(np.sqrt(g.pixel_weights())[:, None] * Y, compute_uv=False)
    np.testing.assert_allclose(s, 1.0, atol=1e-12)


def test_healpix_round_trip_is_approximate():
    # App. A.1: on HEALPix, Y^T W Y ~ I only to 10-20 % in the singular values
    nside = 4
    lmax = 3 * nside - 1
    g = grids.healpix(nside)
    Y = sht.dense_Y(g, lmax)
    s = np.linalg.svd(np.sqrt(g.pixel_weights())[:, None] * Y, compute_uv=False)
    assert s.max() < 1.35 and s.min() > 0.5 and np.abs(s - 1).max() > 1e-3


@pytest.mark.parametrize("grid,lmax", [(grids.healpix(16), 47), (grids.gauss_legendre(40), 40)])
def test_adjoint_identity(grid, lmax):
    rng = np.random.default_rng(7)
    a = rng.standard_normal((lmax + 1) ** 2)
    f = rng.standard_normal(grid.npix)
    lhs = sht.synthesis(grid, lmax, a) @ f
    rhs = a @ sht.adjoint(grid, lmax, f)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs) * 100 + 1e-10


@pytest.mark.parametrize("kind,n,lmax", [("gl", 31, 31), ("hp", 16, 47), ("hp", 8, 40)])
@pytest.mark.parametrize("weighted", [False, True])
def test_adjoint_of_sampled_orders_equals_full_adjoint(kind, n, lmax, weighted):
    # the per-m form (used for full-size checks on a sample of m) against the full adjoint,
    # itself pinned by the dense Y and the adjoint identity
    g = grids.gauss_legendre(lmax) if kind == "gl" else grids.healpix(n)
    f = np.random.default_rng(lmax + n).standard_normal(g.npix)
    full = sht.adjoint(g, lmax, f, weighted=weighted)
    ms = [0, 1, 2, lmax // 2, lmax - 1, lmax]
    got = sht.adjoint_m(g, lmax, f, ms, weighted=weighted)
    scale = np.abs(full).max()
    for m in ms:
        c, s = sht.packed_m(full, lmax, m)
        np.testing.assert_allclose(got[m][0], c, atol=1e-13 * scale, rtol=0)
        np.testing.assert_allclose(got[m][1], s, atol=1e-13 * scale, rtol=0)


def test_lambda_of_one_order_equals_the_triangle_walk():
    theta = grids.healpix(64).theta
    tab = {l: lam for l, lam in lambda_all(300, theta)}
    for m in (0, 3, 150, 299, 300):
        lm = lambda_m(m, 300, theta)
        ref = np.stack([tab[l][m] for l in range(m, 301)])
        np.testing.assert_allclose(lm, ref, rtol=0, atol=1e-14 * max(np.abs(ref).max(), 1e-300))
