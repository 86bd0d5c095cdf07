"""Block-diagonal preconditioner M_diag (oracle, test-only).

The paper compares M_PI with the block-diagonal preconditioner of earlier Gibbs-sampling
work (Sec. 5): M_diag = (U^T diag(T) U)^-1.  In the notation of oracle.precond, T holds
the bands' Y^T N^-1 Y (scaled by alpha^-2) and U the alpha b q blocks and S^-1/2, so for
every real coefficient (l, m, cos / sin) M_diag^-1 is the Ncomp x Ncomp block

    B_{kk'} = delta_{kk'} C_{k,l}^-1 + sum_nu b_{nu,l}^2 q_{nu,k} q_{nu,k'} D_nu(l, m, c/s),

D_nu = diag(Y_nu^T N_nu^-1 Y_nu) (q: the preconditioner's scalar mixing, Eq. optimal-q for
variable maps), restricted to the components with l <= L_k and the bands with l <= L_nu.

The diagonal is O(L) per element from ring sums (the paper's remark): with
Y_lm^c = sqrt(2) lambda_lm cos(m phi), 2 cos^2(m phi) = 1 + cos(2 m phi), so

    D(l, 0)     = sum_r lambda_l0(theta_r)^2 S_r
    D(l, m, c)  = sum_r lambda_lm(theta_r)^2 (S_r + C_r(2m))
    D(l, m, s)  = sum_r lambda_lm(theta_r)^2 (S_r - C_r(2m))

with S_r = sum_j tau_rj and C_r(k) = sum_j tau_rj cos(k phi_rj), the real part of a ring DFT.

Parity: pinned (tests/test_oracle_diagprec.py) -- the ring-sum diagonal against the plain
definition sum_i tau_i Y(n_i)^2 from the dense Y, the block inverse against the
coefficient-wise diagonal blocks of the dense A for scalar mixing, and the paper's comparison
(M_PI needs fewer PCG iterations than M_diag on the multi-resolution model).
"""
import numpy as np

from . import alm as _alm
from . import legendre as _leg
from . import precond as _precond
from . import sht as _sht


def diag_YtNY_dense(grid, lmax, tau):
    """diag(Y^T N^-1 Y) from the explicit Y (small sizes)."""
    Y = _sht.dense_Y(grid, lmax)
    return np.einsum("ij,ij,i->j", Y, Y, np.asarray(tau, dtype=np.float64))


def diag_YtNY(grid, lmax, tau):
    """diag(Y^T N^-1 Y) from ring sums, packed layout at band-limit lmax."""
    tau = np.asarray(tau, dtype=np.float64)
    S = np.zeros(grid.nring)
    C = np.zeros((lmax + 1, grid.nring))            # C_r(2m), m = 0..lmax
    m = np.arange(lmax + 1)
    for r in range(grid.nring):
        n = int(grid.nphi[r])
        t = tau[grid.offset[r]:grid.offset[r + 1]]
        H = np.fft.fft(t)                           # sum_j t_j exp(-2 pi i j k / n)
        S[r] = t.sum()
        k = 2 * m
        C[:, r] = (H[k % n] * np.exp(-1j * k * grid.phi0[r])).real
    Dc = np.zeros((lmax + 1, lmax + 1))             # [l, m]
    Ds = np.zeros((lmax + 1, lmax + 1))
    for l, lam in _leg.lambda_all(lmax, grid.theta):
        l2 = lam[:l + 1] ** 2                       # [m, ring], m <= l
        mm = np.arange(l + 1)
        Dc[l, :l + 1] = (l2 * (S[None, :] + C[mm])).sum(axis=1)
        Ds[l, :l + 1] = (l2 * (S[None, :] - C[mm])).sum(axis=1)
        Dc[l, 0] = (l2[0] * S).sum()                # m = 0: Y_l0^2 = lambda_l0^2
    ell, ms = _alm.layout(lmax)
    return np.where(ms >= 0, Dc[ell, np.abs(ms)], Ds[ell, np.abs(ms)])


def diag_blocks(model):
    """Inverse blocks [n, ncomp, ncomp] of M_diag^-1 over the packed layout of Lmax = max L_k
    (rows / columns of absent components are zero)."""
    Lmax = max(model.lmax_comp)
    ell, ms = _alm.layout(Lmax)
    n = ell.size
    nc = model.ncomp
    q = _precond.preconditioner_q(model)
    Bm = np.zeros((n, nc, nc))
    for nu in range(model.nobs):
        Ln = model.lmax_band[nu]
        D = diag_YtNY(model.grids[nu], Ln, model.tau[nu])
        Dw = _alm.from_2d(_alm.to_2d(D, Ln, Lmax), Lmax)   # zero for l > L_nu
        b = np.zeros(Lmax + 1)
        b[:min(Ln, Lmax) + 1] = model.beam[nu][:min(Ln, Lmax) + 1]
        w = b[ell] ** 2 * Dw
        Bm += w[:, None, None] * np.outer(q[nu], q[nu])[None, :, :]
    present = np.stack([ell <= Lk for Lk in model.lmax_comp], axis=1)   # [n, nc]
    for k, Lk in enumerate(model.lmax_comp):
        c = model.cl[k]
        if c is None:
            continue
        cl = np.asarray(c, dtype=np.float64)
        ci = np.zeros(Lmax + 1)
        with np.errstate(divide="ignore"):
            ci[:Lk + 1] = np.where(np.isfinite(cl[:Lk + 1]), 1.0 / cl[:Lk + 1], 0.0)
        Bm[:, k, k] += ci[ell]
    Binv = np.zeros_like(Bm)
    for i in range(n):
        idx = np.where(present[i])[0]
        if idx.size:
            Binv[i][np.ix_(idx, idx)] = np.linalg.inv(Bm[i][np.ix_(idx, idx)])
    return Binv


def apply_M_diag(model, r, Binv=None):
    """z = M_diag r."""
    if Binv is None:
        Binv = diag_blocks(model)
    Lmax = max(model.lmax_comp)
    parts = model.split(r)
    X = np.stack([_alm.from_2d(_alm.to_2d(p, Lk, Lmax), Lmax)
                  for p, Lk in zip(parts, model.lmax_comp)], axis=1)   # [n, nc]
    Z = np.einsum("ikj,ij->ik", Binv, X)
    return model.stack([_alm.from_2d(_alm.to_2d(Z[:, k], Lmax, Lk), Lk)
                        for k, Lk in enumerate(model.lmax_comp)])
