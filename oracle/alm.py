"""Real harmonic coefficient layout (oracle, test-only).

A component s_k with band-limit L has (L+1)^2 real coefficients (Sec. 3.3
counts (L_k+1)^2 columns of U per component).  They are the coefficients of
the real orthonormal basis

    Y_l0           = lambda_l0(theta)
    Y_lm^c (m > 0) = sqrt(2) lambda_lm(theta) cos(m phi)
    Y_lm^s (m > 0) = sqrt(2) lambda_lm(theta) sin(m phi)

stored m-major: m = 0 with l = 0..L; then for each m = 1..L the cos block
l = m..L followed by the sin block l = m..L.

Inside the oracle a coefficient vector is handled as a 2-D array
X[l, L + m] (cos part, m >= 0) and X[l, L - m] (sin part, m > 0), zero for
|m| > l, so that per-l operators (beams, priors, the U blocks) are plain
broadcasts.
"""
import numpy as np


def nalm(lmax):
    return (lmax + 1) ** 2


def layout(lmax):
    """(ell, msigned) of every packed index; msigned < 0 marks the sin part."""
    ells = [np.arange(lmax + 1)]
    ms = [np.zeros(lmax + 1, dtype=np.int64)]
    for m in range(1, lmax + 1):
        l = np.arange(m, lmax + 1)
        ells += [l, l]
        ms += [np.full(l.size, m), np.full(l.size, -m)]
    return np.concatenate(ells), np.concatenate(ms)


def to_2d(packed, lmax, lwork=None):
    """Packed (lmax+1)^2 vector -> X of shape [lwork+1, 2 lwork+1] (drops l > lwork)."""
    if lwork is None:
        lwork = lmax
    ell, ms = layout(lmax)
    keep = ell <= lwork
    X = np.zeros((lwork + 1, 2 * lwork + 1))
    X[ell[keep], lwork + ms[keep]] = np.asarray(packed)[keep]
    return X


def from_2d(X, lmax):
    """X of shape [lwork+1, 2 lwork+1] -> packed (lmax+1)^2 vector (zero for l > lwork)."""
    lwork = X.shape[0] - 1
    ell, ms = layout(lmax)
    out = np.zeros(ell.size)
    keep = ell <= lwork
    out[keep] = X[ell[keep], lwork + ms[keep]]
    return out


def ell_of_index(lmax):
    return layout(lmax)[0]
