"""Spherical harmonic transforms on ring grids (oracle, test-only).

Sec. 2.1 names three operators: synthesis Y (coefficients -> pixels),
analysis Y^T W (pixels -> coefficients, quadrature-weighted) and, in Sec.
3.2, adjoint synthesis Y^T (the plain transpose, which is what P^T contains).

With the real basis of ``oracle.alm`` and pixel (theta_r, phi_j),
phi_j = phi0_r + 2 pi j / nphi_r, synthesis is

    f(theta_r, phi_j) = Fc_0(r) + sqrt(2) sum_{m>=1} [Fc_m(r) cos(m phi_j) + Fs_m(r) sin(m phi_j)]
    Fc_m(r) = sum_l lambda_lm(theta_r) c_lm,   Fs_m(r) = sum_l lambda_lm(theta_r) s_lm.

The azimuthal sums are evaluated per ring by a length-nphi DFT after folding
frequencies m modulo nphi (numpy.fft serves as the DFT primitive).  The
adjoint applies the transposes of the same two factors in reverse order.

``dense_Y`` builds the explicit matrix (pixels x coefficients) for small L,
so that dense A, M_PI and gradients can be formed and checked.

Parity: pinned (tests/test_oracle_sht.py) -- dense Y against scipy's
spherical harmonics, the exact Gauss-Legendre round trip Y^T W Y = I
(Sec. 2.1), unit singular values of W^(1/2) Y on GL (App. A.1), and the
adjoint identity <Y a, f> = <a, Y^T f>.
"""
import numpy as np

from . import alm as _alm
from .legendre import lambda_all, lambda_lm_table, lambda_m

_SQRT2 = np.sqrt(2.0)


def _phase_synth(grid, Fc, Fs, lmax):
    """Azimuthal synthesis: Fc, Fs of shape [lmax+1, nring] -> pixel map."""
    out = np.empty(grid.npix)
    m = np.arange(lmax + 1)
    for r in range(grid.nring):
        n = int(grid.nphi[r])
        g = Fc[:, r] - 1j * Fs[:, r]
        g[1:] *= _SQRT2
        g = g * np.exp(1j * m * grid.phi0[r])
        h = np.zeros(n, dtype=np.complex128)
        np.add.at(h, m % n, g)
        f = np.fft.ifft(h) * n            # sum_k h_k exp(+2 pi i j k / n)
        out[grid.offset[r]: grid.offset[r + 1]] = f.real
    return out


def _phase_adjoint(grid, fmap, lmax):
    """Transpose of _phase_synth: pixel map -> Gc, Gs of shape [lmax+1, nring]."""
    Gc = np.zeros((lmax + 1, grid.nring))
    Gs = np.zeros((lmax + 1, grid.nring))
    m = np.arange(lmax + 1)
    for r in range(grid.nring):
        n = int(grid.nphi[r])
        f = fmap[grid.offset[r]: grid.offset[r + 1]]
        H = np.fft.fft(f)                 # sum_j f_j exp(-2 pi i j k / n)
        G = H[m % n] * np.exp(-1j * m * grid.phi0[r])
        # sum_j f_j cos(m phi_j) = Re G, sum_j f_j sin(m phi_j) = -Im G
        Gc[:, r] = G.real
        Gs[:, r] = -G.imag
        Gc[1:, r] *= _SQRT2
        Gs[1:, r] *= _SQRT2
    Gs[0] = 0.0
    return Gc, Gs


def synthesis(grid, lmax, packed):
    """Y a: packed (lmax+1)^2 coefficients -> map on ``grid``."""
    X = _alm.to_2d(packed, lmax)
    Fc = np.zeros((lmax + 1, grid.nring))
    Fs = np.zeros((lmax + 1, grid.nring))
    for l, lam in lambda_all(lmax, grid.theta):
        ms = np.arange(l + 1)
        Fc[: l + 1] += lam * X[l, lmax + ms][:, None]
        Fs[: l + 1] += lam * X[l, lmax - ms][:, None]
    Fs[0] = 0.0
    return _phase_synth(grid, Fc, Fs, lmax)


def adjoint(grid, lmax, fmap, weighted=False):
    """Y^T f (weighted=False) or Y^T W f (weighted=True): map -> packed coefficients."""
    f = np.asarray(fmap, dtype=np.float64)
    if weighted:
        f = f * grid.pixel_weights()
    Gc, Gs = _phase_adjoint(grid, f, lmax)
    X = np.zeros((lmax + 1, 2 * lmax + 1))
    for l, lam in lambda_all(lmax, grid.theta):
        ms = np.arange(l + 1)
        X[l, lmax + ms] = (lam * Gc[: l + 1]).sum(axis=1)
        X[l, lmax - ms[1:]] = (lam[1:] * Gs[1: l + 1]).sum(axis=1)
    return _alm.from_2d(X, lmax)


def adjoint_m(grid, lmax, fmap, ms, weighted=False):
    """Y^T f (or Y^T W f) restricted to the orders m in ``ms``: {m: (cos part, sin part)},
    each of length lmax - m + 1 (l = m..lmax; the sin part of m = 0 is zero).

    The Legendre stage is independent per m, so this equals the matching entries of
    ``adjoint`` while touching only the requested columns: the full azimuthal transform of
    every ring, then the per-m recurrence over all rings."""
    f = np.asarray(fmap, dtype=np.float64)
    if weighted:
        f = f * grid.pixel_weights()
    ms = [int(m) for m in ms]
    marr = np.asarray(ms)
    Gc = np.zeros((len(ms), grid.nring))
    Gs = np.zeros((len(ms), grid.nring))
    for r in range(grid.nring):
        n = int(grid.nphi[r])
        H = np.fft.fft(f[grid.offset[r]: grid.offset[r + 1]])
        G = H[marr % n] * np.exp(-1j * marr * grid.phi0[r])
        Gc[:, r] = G.real
        Gs[:, r] = -G.imag
    out = {}
    for i, m in enumerate(ms):
        lam = lambda_m(m, lmax, grid.theta)            # [l - m, ring]
        c = lam @ Gc[i]
        s = lam @ Gs[i]
        if m > 0:
            c, s = _SQRT2 * c, _SQRT2 * s
        else:
            s = np.zeros_like(s)
        out[m] = (c, s)
    return out


def packed_m(packed, lmax, m):
    """The (cos part, sin part) of order m of a packed coefficient vector (l = m..lmax)."""
    n = lmax - m + 1
    if m == 0:
        return np.asarray(packed[:n]), np.zeros(n)
    o = (lmax + 1) + (m - 1) * (2 * lmax + 2 - m)
    return np.asarray(packed[o: o + n]), np.asarray(packed[o + n: o + 2 * n])


def analysis(grid, lmax, fmap):
    """Y^T W f."""
    return adjoint(grid, lmax, fmap, weighted=True)


def dense_Y(grid, lmax):
    """Explicit synthesis matrix of shape [npix, (lmax+1)^2] (small lmax only)."""
    lam = lambda_lm_table(lmax, grid.theta)          # [l, m, ring]
    ell, ms = _alm.layout(lmax)
    th, ph = grid.pixel_angles()
    ring_of_pix = np.repeat(np.arange(grid.nring), grid.nphi)
    Y = np.empty((grid.npix, ell.size))
    for i in range(ell.size):
        l, m = ell[i], ms[i]
        base = lam[l, abs(m), ring_of_pix]
        if m == 0:
            Y[:, i] = base
        elif m > 0:
            Y[:, i] = _SQRT2 * base * np.cos(m * ph)
        else:
            Y[:, i] = _SQRT2 * base * np.sin(-m * ph)
    return Y
