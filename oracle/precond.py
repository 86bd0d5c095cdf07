"""The pseudo-inverse preconditioner M_PI (oracle, test-only).

Sec. 3.3 factors A = U^T T U (Eq. A-for-pseudoinv) with

    T = diag(N~_nu^-1, I),    N~_nu^-1 = alpha_nu^-2 Y_nu^T N_nu^-1 Y_nu,
    U = [alpha B Q~ ; S^-1/2],

and, with Q~_{nu,k} ~ q_{nu,k} I, U is block diagonal over (l, m) with blocks
that do not depend on m:

    U[(l,m,nu),(l,m,k)]      = alpha_nu b_{nu,l} q_{nu,k}   (Eq. U-data)
    U[(l,m,Nobs+k),(l,m,k)]  = C_{k,l}^-1/2                 (Eq. U-prior)

Rows of band nu exist for l <= L_nu, rows and columns of component k for
l <= L_k; the oracle zero-pads them (Sec. 3.3 states zero-padding gives the
same numbers).  U^+ is the SVD pseudo-inverse per l (Sec. 3.1), cut off at
1e-12 times the largest singular value.  Then

    M_PI = U^+ T^+ (U^+)^T,   T^+_nu = alpha_nu^2 Y_nu^T W_nu N_nu W_nu Y_nu

(Eq. fullmodel-preconditioner), with N_nu = diag(1/tau_nu).

alpha_nu = sqrt(sum (tau/w)^2 / sum (tau/w))   (Eq. optimal-alpha, App. A.1)
q_{nu,k} = sum q^2 / sum q                     (Eq. optimal-q, App. A.2)

Parity: pinned (tests/test_oracle_precond.py) -- U^+ U = I (Sec. 3.1), the
flat-noise case M_PI = A^-1 (Sec. 3.3) against ``oracle.closed_form``,
alpha and q against brute-force minimisation of the norms in App. A.
"""
import numpy as np

from . import alm as _alm
from . import sht as _sht

PINV_RCOND = 1e-12


def optimal_alpha(tau, w):
    """Eq. optimal-alpha: least-squares scalar with alpha^-2 tau/w ~ 1."""
    r = np.asarray(tau, dtype=np.float64) / np.asarray(w, dtype=np.float64)
    return float(np.sqrt(np.sum(r * r) / np.sum(r)))


def optimal_q(qmap):
    """Eq. optimal-q: least-squares scalar approximation of a mixing map."""
    q = np.asarray(qmap, dtype=np.float64)
    return float(np.sum(q * q) / np.sum(q))


def preconditioner_q(model):
    """Scalar mixing used in U: given q, or Eq. optimal-q of each variable map."""
    q = np.array(model.q, dtype=np.float64, copy=True)
    if model.mix_map is not None:
        for nu in range(model.nobs):
            for k in range(model.ncomp):
                if model.mix_map[nu][k] is not None:
                    q[nu, k] = optimal_q(model.mix_map[nu][k])
    return q


def alphas(model):
    return np.array([optimal_alpha(model.tau[nu], model.grids[nu].pixel_weights())
                     for nu in range(model.nobs)])


def U_blocks(model):
    """U_l for l = 0..Lmax as an array [Lmax+1, Nobs+Ncomp, Ncomp] (zero-padded)."""
    nobs, ncomp = model.nobs, model.ncomp
    Lmax = max(model.lmax_comp)
    al = alphas(model)
    q = preconditioner_q(model)
    U = np.zeros((Lmax + 1, nobs + ncomp, ncomp))
    for l in range(Lmax + 1):
        for k in range(ncomp):
            if l > model.lmax_comp[k]:
                continue
            for nu in range(nobs):
                if l <= model.lmax_band[nu]:
                    U[l, nu, k] = al[nu] * model.beam[nu][l] * q[nu, k]
            c = model.cl[k]
            if c is not None and np.isfinite(c[l]):
                U[l, nobs + k, k] = c[l] ** -0.5
    return U


def pinv_blocks(U):
    """U^+ per l by SVD (Sec. 3.1): [Lmax+1, Ncomp, Nobs+Ncomp]."""
    return np.stack([np.linalg.pinv(U[l], rcond=PINV_RCOND) for l in range(U.shape[0])])


def _stack_to_3d(model, x, Lw):
    """Stacked vector -> array [Lw+1, 2Lw+1, Ncomp]."""
    xs = model.split(x)
    return np.stack([_alm.to_2d(xs[k], model.lmax_comp[k], Lw) for k in range(model.ncomp)], axis=-1)


def _3d_to_stack(model, X):
    return np.concatenate([_alm.from_2d(X[..., k], model.lmax_comp[k]) for k in range(model.ncomp)])


def T_plus_band(model, nu, alpha, t_packed):
    """T^+_nu t = alpha^2 Y^T W N W Y t with N = diag(1/tau) (Sec. 3.3)."""
    g = model.grids[nu]
    Ln = model.lmax_band[nu]
    w = g.pixel_weights()
    f = _sht.synthesis(g, Ln, t_packed)
    f = f * (alpha * alpha * w * w / model.tau[nu])
    return _sht.adjoint(g, Ln, f)


def apply_precond(model, r, Up=None):
    """z = M_PI r = U^+ T^+ (U^+)^T r."""
    if Up is None:
        Up = pinv_blocks(U_blocks(model))
    al = alphas(model)
    Lw = Up.shape[0] - 1
    R = _stack_to_3d(model, np.asarray(r, dtype=np.float64), Lw)     # [l, m, k]
    t = np.einsum("lkj,lmk->lmj", Up, R)                              # (U^+)^T r, [l, m, nobs+ncomp]
    for nu in range(model.nobs):
        Ln = model.lmax_band[nu]
        tp = _alm.from_2d(t[..., nu], Ln)
        tp = T_plus_band(model, nu, al[nu], tp)
        t[..., nu] = _alm.to_2d(tp, Ln, Lw)
    Z = np.einsum("lkj,lmj->lmk", Up, t)                              # U^+ t
    return _3d_to_stack(model, Z)
