"""Pins of oracle.grids against closed forms (no GPU)."""
import os

import numpy as np
import pytest

from oracle import grids

GOLD = os.path.join(os.path.dirname(__file__), "golden", "healpix_nside1_nside2.txt")


@pytest.mark.parametrize("lmax", [3, 15, 63])
def test_gl_quadrature_is_exact_for_polynomials(lmax):
    g = grids.gauss_legendre(lmax)
    x = np.cos(g.theta)
    gw = g.weight * g.nphi / (2 * np.pi)         # back to the 1-D Gauss weights
    for k in range(0, 2 * lmax + 2):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(gw * x ** k) - exact) < 1e-13
    assert abs(g.pixel_weights().sum() - 4 * np.pi) < 1e-12
    assert np.all(np.diff(g.theta) > 0) and np.all(g.nphi == 2 * lmax + 1)


def test_healpix_small_nside_matches_published_geometry():
    rows = np.loadtxt(GOLD)
    for nside in (1, 2):
        g = grids.healpix(nside)
        sel = rows[rows[:, 0] == nside]
        assert g.nring == len(sel)
        np.testing.assert_allclose(np.cos(g.theta), sel[:, 2], atol=1e-15)
        np.testing.assert_array_equal(g.nphi, sel[:, 3].astype(int))
        np.testing.assert_allclose(g.phi0 / np.pi, sel[:, 4], atol=1e-15)


@pytest.mark.parametrize("nside", [1, 4, 7, 32, 256])
def test_healpix_counts_and_symmetry(nside):
    g = grids.healpix(nside)
    assert g.npix == 12 * nside * nside
    assert g.nring == 4 * nside - 1
    z = np.cos(g.theta)
    np.testing.assert_allclose(z, -z[::-1], atol=1e-14)
    np.testing.assert_array_equal(g.nphi, g.nphi[::-1])
    assert abs(g.pixel_weights().sum() - 4 * np.pi) < 1e-10
    # equatorial belt: equal z spacing 2/(3 Nside)
    belt = z[nside - 1: 3 * nside]
    np.testing.assert_allclose(np.diff(belt), -2.0 / (3 * nside), atol=1e-14)
    # polar caps: 4i pixels on ring i, z = 1 - i^2 / (3 Nside^2)
    i = np.arange(1, nside)
    np.testing.assert_array_equal(g.nphi[: nside - 1], 4 * i)
    np.testing.assert_allclose(z[: nside - 1], 1 - i * i / (3.0 * nside * nside), atol=1e-15)
