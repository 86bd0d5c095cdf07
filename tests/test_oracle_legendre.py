"""Pins of oracle.legendre against independent implementations (no GPU)."""
import math

import mpmath
import numpy as np
import pytest
from scipy.special import sph_harm_y

from oracle import grids, legendre


def _lam_mpmath(l, m, theta):
    """lambda_lm from mpmath's associated Legendre function (Condon-Shortley phase removed)."""
    mpmath.mp.dps = 40
    x = mpmath.cos(mpmath.mpf(theta))
    norm = mpmath.sqrt((2 * l + 1) / (4 * mpmath.pi) * mpmath.factorial(l - m) / mpmath.factorial(l + m))
    return float((-1) ** m * norm * mpmath.legenp(l, m, x))


def test_lambda_matches_scipy_small_l():
    theta = np.array([0.05, 0.4, 1.0, 1.5707963, 2.2, 3.05])
    L = 40
    tab = legendre.lambda_lm_table(L, theta)
    for l in range(L + 1):
        for m in range(l + 1):
            ref = ((-1) ** m) * sph_harm_y(l, m, theta, 0.0).real
            np.testing.assert_allclose(tab[l, m], ref, rtol=1e-11, atol=1e-13)


def test_lambda_orthonormal_under_gl_quadrature():
    L = 48
    g = grids.gauss_legendre(L)
    gw = g.weight * g.nphi                      # 2 pi * Gauss weight
    tab = legendre.lambda_lm_table(L, g.theta)
    for m in (0, 1, 7, 30, 48):
        lam = tab[m:, m, :]                     # [l, ring]
        G = (lam * gw) @ lam.T
        np.testing.assert_allclose(G, np.eye(L + 1 - m), atol=1e-12)


@pytest.mark.parametrize("l,m,theta", [
    (300, 200, 0.8),        # ordinary range
    (1200, 1000, 0.95),     # lambda_mm ~ 1e-50
    (3000, 2000, 0.775),    # lambda_mm underflows FP64 (~1e-310); lambda_lm is O(1)
    (3071, 2900, 1.3),
])
def test_lambda_scaled_recurrence_high_l(l, m, theta):
    ref = _lam_mpmath(l, m, theta)
    got = None
    for ll, lam in legendre.lambda_all(l, np.array([theta]), mmax=m):
        if ll == l:
            got = lam[m, 0]
    assert got is not None
    assert abs(got - ref) <= 1e-10 * max(abs(ref), 1e-30) + 1e-300, (got, ref)


def _lam_mp_recurrence(l, m, theta):
    """Same seeds/recurrence in mpmath floats, whose exponent range is unbounded."""
    mpmath.mp.dps = 30
    x, s = mpmath.cos(mpmath.mpf(theta)), mpmath.sin(mpmath.mpf(theta))
    v = mpmath.sqrt(1 / (4 * mpmath.pi))
    for j in range(1, m + 1):
        v *= mpmath.sqrt(mpmath.mpf(2 * j + 1) / (2 * j)) * s
    p2, p1 = mpmath.mpf(0), v
    if l == m:
        return p1
    p2, p1 = p1, mpmath.sqrt(2 * m + 3) * x * v
    for ll in range(m + 2, l + 1):
        a = mpmath.sqrt(mpmath.mpf(4 * ll * ll - 1) / (ll * ll - m * m))
        a1 = mpmath.sqrt(mpmath.mpf(4 * (ll - 1) ** 2 - 1) / ((ll - 1) ** 2 - m * m))
        p2, p1 = p1, a * (x * p1 - p2 / a1)
    return p1


def test_negligible_values_are_reported_as_zero():
    # deep in the evanescent region the true value is far below 1e-30
    ref = _lam_mp_recurrence(1000, 900, 0.2)
    assert abs(ref) < mpmath.mpf(10) ** -100
    for ll, lam in legendre.lambda_all(1000, np.array([0.2]), mmax=900):
        pass
    assert lam[900, 0] == 0.0
