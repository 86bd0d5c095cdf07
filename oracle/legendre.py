"""Normalised associated Legendre functions lambda_lm(theta) (oracle, test-only).

lambda_lm is the orthonormal associated Legendre function without the
Condon-Shortley phase, so that the complex harmonic is
Y_lm(theta, phi) = lambda_lm(theta) exp(i m phi) with unit norm on the
sphere (the SHT of Sec. 2.1 is built from these).

Seeds and recurrence (standard, e.g. Press et al., Numerical Recipes 6.7):

    lambda_mm     = sqrt(1/(4 pi)) * prod_{j=1..m} sqrt((2j+1)/(2j)) * sin(theta)
    lambda_{m+1,m} = sqrt(2m+3) cos(theta) lambda_mm
    lambda_lm     = a_lm (cos(theta) lambda_{l-1,m} - lambda_{l-2,m} / a_{l-1,m}),
    a_lm          = sqrt((4 l^2 - 1) / (l^2 - m^2)).

At high m and near the poles lambda_mm falls far below the FP64 range while
lambda_lm at larger l can still be of order one, so values are carried as
v * 2^(-600 k) with an integer k >= 0 per (m, ring); v is divided by 2^600
when it grows past 2^500 while k > 0, and a value is reported only once k == 0.
A value still carrying k > 0 is below 2^-100 (~1e-30) and is reported as 0.

Parity: pinned (tests/test_oracle_legendre.py) against
scipy.special.sph_harm_y (an independent implementation) and against the
orthonormality of lambda_lm under Gauss-Legendre quadrature.
"""
import numpy as np

_SHIFT = 600
_BIG = 2.0 ** _SHIFT
_GROW = 2.0 ** 500      # rescale threshold while k > 0, so that k > 0 means |value| < 2^-100


def seeds(mmax, theta):
    """lambda_mm for m = 0..mmax as (v, k) arrays of shape [mmax+1, nring]."""
    s = np.sin(np.asarray(theta, dtype=np.float64))
    nr = s.size
    v = np.empty((mmax + 1, nr))
    k = np.zeros((mmax + 1, nr), dtype=np.int64)
    cur = np.full(nr, np.sqrt(1.0 / (4.0 * np.pi)))
    ck = np.zeros(nr, dtype=np.int64)
    v[0] = cur
    for m in range(1, mmax + 1):
        cur = cur * (np.sqrt((2.0 * m + 1.0) / (2.0 * m)) * s)
        small = (cur != 0.0) & (np.abs(cur) < 1.0 / _BIG)
        cur = np.where(small, cur * _BIG, cur)
        ck = ck + small
        v[m] = cur
        k[m] = ck
    return v, k


def lambda_all(lmax, theta, mmax=None):
    """Generator over l = 0..lmax yielding (l, lam) with lam[m, ring] for m <= min(l, mmax).

    This walks the recurrence in l for all (m, ring) at once, which is the
    order the paper's SHT cost model counts (one pass over the (l, m)
    triangle per ring).
    """
    theta = np.asarray(theta, dtype=np.float64)
    if mmax is None:
        mmax = lmax
    x = np.cos(theta)
    sv, sk = seeds(mmax, theta)
    nm = mmax + 1
    p1 = np.zeros((nm, theta.size))      # lambda_{l-1,m} (scaled)
    p2 = np.zeros((nm, theta.size))      # lambda_{l-2,m} (scaled)
    kk = np.zeros((nm, theta.size), dtype=np.int64)
    ms = np.arange(nm, dtype=np.float64)
    for l in range(lmax + 1):
        cur = np.zeros((nm, theta.size))
        top = min(l, mmax)
        # m = l: seed
        if l <= mmax:
            cur[l] = sv[l]
            kk[l] = sk[l]
        # m = l - 1: second seed
        if 1 <= l <= mmax + 1:
            m = l - 1
            cur[m] = np.sqrt(2.0 * m + 3.0) * x * p1[m]
        # m <= l - 2: three-term recurrence
        if l >= 2:
            mm = min(l - 2, mmax)
            msel = ms[: mm + 1]
            a_l = np.sqrt((4.0 * l * l - 1.0) / (l * l - msel * msel))[:, None]
            a_lm1 = np.sqrt((4.0 * (l - 1) ** 2 - 1.0) / ((l - 1) ** 2 - msel * msel))[:, None]
            cur[: mm + 1] = a_l * (x * p1[: mm + 1] - p2[: mm + 1] / a_lm1)
        # rescale values that have grown back into range
        grow = (kk[: top + 1] > 0) & (np.abs(cur[: top + 1]) > _GROW)
        if grow.any():
            c = cur[: top + 1]
            q1 = p1[: top + 1]
            c[grow] /= _BIG
            q1[grow] /= _BIG
            kk[: top + 1][grow] -= 1
        p2[: top + 1] = p1[: top + 1]
        p1[: top + 1] = cur[: top + 1]
        lam = np.where(kk[: top + 1] == 0, cur[: top + 1], 0.0)
        yield l, lam


def lambda_lm_table(lmax, theta):
    """Dense table lam[l, m, ring] (zero for m > l). For small lmax only."""
    theta = np.asarray(theta, dtype=np.float64)
    out = np.zeros((lmax + 1, lmax + 1, theta.size))
    for l, lam in lambda_all(lmax, theta):
        out[l, : l + 1] = lam
    return out


def lambda_m(m, lmax, theta):
    """lambda_lm(theta) for one m and l = m..lmax, shape [lmax - m + 1, nring].

    The same seeds, recurrence and exponent handling as lambda_all, walked along l for a
    single m (used to check transforms at full size on a sample of m)."""
    theta = np.asarray(theta, dtype=np.float64)
    x = np.cos(theta)
    sv, sk = seeds(m, theta)
    out = np.zeros((lmax - m + 1, theta.size))
    if lmax < m:
        return out
    cur, k = sv[m].copy(), sk[m].copy()
    out[0] = np.where(k == 0, cur, 0.0)
    prev = np.zeros_like(cur)
    for l in range(m + 1, lmax + 1):
        if l == m + 1:
            nxt = np.sqrt(2.0 * m + 3.0) * x * cur
        else:
            a_l = np.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
            a_lm1 = np.sqrt((4.0 * (l - 1) ** 2 - 1.0) / ((l - 1) ** 2 - m * m))
            nxt = a_l * (x * cur - prev / a_lm1)
        grow = (k > 0) & (np.abs(nxt) > _GROW)
        if grow.any():
            nxt = np.where(grow, nxt / _BIG, nxt)
            cur = np.where(grow, cur / _BIG, cur)
            k = k - grow
        prev, cur = cur, nxt
        out[l - m] = np.where(k == 0, cur, 0.0)
    return out
