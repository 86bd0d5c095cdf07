"""Ring grids on the sphere and their quadrature weights (oracle, test-only).

A grid here is a stack of iso-latitude rings, north to south.  Ring r has
colatitude theta_r, nphi_r equispaced pixels starting at azimuth phi0_r, and
one quadrature weight w_r shared by its pixels.  Pixels are stored ring by
ring, increasing azimuth within a ring.

* Gauss-Legendre: L+1 rings at the Gauss-Legendre nodes in cos(theta), nphi
  >= 2L+1 pixels per ring, phi0 = 0, w = g_r * 2 pi / nphi.  On this grid
  Y^T W Y = I holds exactly for band-limit L (Sec. 2.1; App. A.1 notes the
  singular values of Y^T W^(1/2) are all 1 there).
* HEALPix ring scheme (Gorski et al. 2005 geometry): 4 Nside - 1 rings,
  polar rings with 4 i pixels, equatorial rings with 4 Nside pixels, uniform
  weights 4 pi / Npix.  Y^T W Y = I holds only approximately there (Sec. 3.2,
  App. A.1), which the paper accepts.

Parity: pinned (tests/test_oracle_grids.py) -- quadrature exactness of
polynomials, Nside = 1 pixel centres, ring counts and symmetry.
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class RingGrid:
    kind: str            # "gl" or "healpix"
    n: int               # GL: number of rings; HEALPix: Nside
    theta: np.ndarray    # [nring] colatitude
    phi0: np.ndarray     # [nring] azimuth of the first pixel
    nphi: np.ndarray     # [nring] pixels per ring
    weight: np.ndarray   # [nring] quadrature weight of each pixel in the ring
    offset: np.ndarray   # [nring + 1] first pixel of each ring

    @property
    def nring(self):
        return self.theta.size

    @property
    def npix(self):
        return int(self.offset[-1])

    def pixel_weights(self):
        return np.repeat(self.weight, self.nphi)

    def pixel_angles(self):
        """(theta, phi) of every pixel, ring order."""
        th = np.repeat(self.theta, self.nphi)
        ph = np.concatenate([
            self.phi0[r] + 2.0 * np.pi * np.arange(self.nphi[r]) / self.nphi[r]
            for r in range(self.nring)
        ])
        return th, ph


def gauss_legendre(lmax, nphi=None):
    """GL grid with lmax+1 rings and nphi (default 2 lmax + 1) pixels per ring."""
    nring = lmax + 1
    if nphi is None:
        nphi = 2 * lmax + 1
    if nphi < 2 * lmax + 1:
        raise ValueError("nphi must be >= 2 lmax + 1")
    x, g = np.polynomial.legendre.leggauss(nring)
    order = np.argsort(-x)                 # north (cos theta = +1) first
    x, g = x[order], g[order]
    theta = np.arccos(x)
    nphis = np.full(nring, nphi, dtype=np.int64)
    weight = g * 2.0 * np.pi / nphi
    offset = np.concatenate([[0], np.cumsum(nphis)])
    return RingGrid("gl", nring, theta, np.zeros(nring), nphis, weight, offset)


def healpix(nside):
    """HEALPix ring-scheme geometry for a given Nside (any positive integer)."""
    ns = int(nside)
    nring = 4 * ns - 1
    z = np.empty(nring)
    nphi = np.empty(nring, dtype=np.int64)
    phi0 = np.empty(nring)
    for i in range(1, nring + 1):
        # distance from the nearer pole, in ring units
        ip = i if i <= 2 * ns else 4 * ns - i
        if ip < ns:                        # polar cap ring
            zz = 1.0 - ip * ip / (3.0 * ns * ns)
            nphi[i - 1] = 4 * ip
            phi0[i - 1] = np.pi / (4.0 * ip)
        else:                              # equatorial belt ring
            zz = 4.0 / 3.0 - 2.0 * ip / (3.0 * ns)
            nphi[i - 1] = 4 * ns
            phi0[i - 1] = np.pi / (4.0 * ns) if (ip - ns) % 2 == 0 else 0.0
        z[i - 1] = zz if i <= 2 * ns else -zz
    theta = np.arccos(z)
    npix = 12 * ns * ns
    weight = np.full(nring, 4.0 * np.pi / npix)
    offset = np.concatenate([[0], np.cumsum(nphi)])
    return RingGrid("healpix", ns, theta, phi0, nphi, weight, offset)


def healpix_lmax(nside):
    """Band-limit used with a HEALPix data grid: 3 Nside - 1."""
    return 3 * int(nside) - 1
