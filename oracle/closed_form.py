"""Closed-form diagonal Wiener filter (oracle, test-only).

When every band grid is Gauss-Legendre with at least L_nu+1 rings and
2 L_nu + 1 pixels per ring, the mixing is a scalar q_{nu,k} and the inverse
noise is flat per unit area, tau_nu = w / sigma_nu^2, then
Y^T diag(tau) Y = sigma_nu^-2 Y^T W Y = sigma_nu^-2 I exactly (Sec. 2.1), so
A is block diagonal over (l, m) with m-independent blocks

    A_l = diag(C_{k,l}^-1) + sum_{nu : l <= L_nu} b_{nu,l}^2 q_nu q_nu^T / sigma_nu^2

restricted to the components with l <= L_k.  This is the flat case of
Sec. 3.3 (T = I), where M_PI equals A^-1.  It involves no SHT, so it pins
the assembly of A, the solve and M_PI independently of the transforms.
"""
import numpy as np

from . import alm as _alm


def A_blocks(lmax_comp, lmax_band, beam, cl, q, sigma):
    ncomp, nobs = len(lmax_comp), len(lmax_band)
    Lmax = max(lmax_comp)
    A = np.zeros((Lmax + 1, ncomp, ncomp))
    for l in range(Lmax + 1):
        for k in range(ncomp):
            if l > lmax_comp[k]:
                A[l, k, k] = 1.0          # placeholder on absent coefficients
                continue
            c = cl[k]
            if c is not None and np.isfinite(c[l]):
                A[l, k, k] += 1.0 / c[l]
        for nu in range(nobs):
            if l > lmax_band[nu]:
                continue
            act = np.array([l <= lmax_comp[k] for k in range(ncomp)])
            qv = np.where(act, q[nu], 0.0)
            A[l] += beam[nu][l] ** 2 * np.outer(qv, qv) / sigma[nu] ** 2
    return A


def _apply_blocks(B, lmax_comp, x):
    ncomp = len(lmax_comp)
    Lw = B.shape[0] - 1
    offs = np.concatenate([[0], np.cumsum([_alm.nalm(L) for L in lmax_comp])])
    X = np.stack([_alm.to_2d(x[offs[k]:offs[k + 1]], lmax_comp[k], Lw) for k in range(ncomp)], -1)
    Y = np.einsum("lkj,lmj->lmk", B, X)
    return np.concatenate([_alm.from_2d(Y[..., k], lmax_comp[k]) for k in range(ncomp)])


def apply_A(lmax_comp, lmax_band, beam, cl, q, sigma, x):
    return _apply_blocks(A_blocks(lmax_comp, lmax_band, beam, cl, q, sigma), lmax_comp, x)


def solve(lmax_comp, lmax_band, beam, cl, q, sigma, b):
    A = A_blocks(lmax_comp, lmax_band, beam, cl, q, sigma)
    return _apply_blocks(np.linalg.inv(A), lmax_comp, b)
