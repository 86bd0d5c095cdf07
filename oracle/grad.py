"""Derivatives of the Wiener / CR solution with respect to the model parameters (oracle, test-only).

The paper solves A x = b (Eq. A) for fixed model parameters and has no gradient.
A loss L(x) of the solution depends on a parameter theta through A(theta) and
b(theta); differentiating A x = b gives A dx/dtheta = db/dtheta - (dA/dtheta) x,
so with the adjoint solution lambda of A lambda = dL/dx (A is symmetric)

    dL/dtheta = lambda^T (db/dtheta - (dA/dtheta) x).

The parameters are the scalar mixing entries q_{nu,k} (P_{nu,k} = Y_nu B_nu q_{nu,k},
Eq. P with a spatially constant Q) and a log-scale t_k of each prior spectrum,
C_{k,l} -> exp(t_k) C_{k,l}, taken at t_k = 0.  With the CR right-hand side of
Sec. 2.3 (read with S^-1/2 omega_2), b = P^T (N^-1 d + N^-1/2 omega_1) + S^-1/2 omega_2:

    dA/dq_{nu,k} = dP_nu^T N^-1 P_nu + P_nu^T N^-1 dP_nu,   dP_nu = Y_nu B_nu E_k
    db/dq_{nu,k} = dP_nu^T (N^-1 d_nu + N^-1/2 omega_1,nu)
    dA/dt_k = -S_k^-1 (block k),   db/dt_k = -1/2 S_k^-1/2 omega_2,k

where E_k picks component k (zero-padded or truncated to L_nu).  ``grad_terms_dense``
writes these matrices out; ``grad_terms`` applies them as operators.  A spectral
index beta_k with q_{nu,k} = (nu / nu_0)^beta_k follows by the chain rule.

Spatially variable mixing (Eq. Q): Q~_{nu,k} = Y_nu^T W diag(q) Y_k on the pair's mixing
grid, so the derivative in the map value q(p) at pixel p is the rank-one
dQ~/dq(p) = (Y_nu^T W)[:, p] Y_k[p, :], and with u_nu = B_nu Y_band^T (N^-1 d + N^-1/2 w1
- N^-1 P x), v_nu = B_nu Y_band^T N^-1 P lambda (the same two adjoint passes as above)

    dL/dq_{nu,k}(p) = w_p [ (Y_k lambda_k)(p) (Y_nu u_nu)(p) - (Y_k x_k)(p) (Y_nu v_nu)(p) ]

(``grad_mix_maps``; ``grad_mix_maps_dense`` builds dP per pixel instead).  For a variable
pair the scalar entry dq_{nu,k} is the derivative in a uniform offset added to the map,
the sum of the map over its pixels; on a grid that integrates the products exactly it
equals the scalar-mixing entry of the same q.

Parity: pinned (tests/test_oracle_grad.py) -- central finite differences of the loss
of the dense Cholesky solve (in q, prior scales and mixing-map pixels), operator form =
dense form, and the offset derivative of a constant map = the scalar-mixing derivative.
"""
import numpy as np

from . import alm as _alm
from . import model as _model
from . import sht as _sht


def _select(model, nu, k, xk):
    """E_k: component k's coefficients at band-limit L_nu (padded or truncated)."""
    return _model._retruncate(xk, model.lmax_comp[k], model.lmax_band[nu])


def dense_dP(model, nu, k):
    """dP_nu / dq_{nu,k} = Y_nu B_nu E_k as a dense [npix_nu, nvec] matrix."""
    n = model.nvec()
    o = model.comp_offsets()
    Ln = model.lmax_band[nu]
    M = np.zeros((_alm.nalm(Ln), n))
    Lk = model.lmax_comp[k]
    for j in range(_alm.nalm(Lk)):
        e = np.zeros(_alm.nalm(Lk))
        e[j] = 1.0
        M[:, o[k] + j] = _select(model, nu, k, e)
    M = M * model.beam[nu][_alm.ell_of_index(Ln)][:, None]
    return _sht.dense_Y(model.grids[nu], Ln) @ M


def _data_maps(model, d, omega1):
    """N^-1 d + N^-1/2 omega_1 per band."""
    out = []
    for nu in range(model.nobs):
        v = model.tau[nu] * d[nu]
        if omega1 is not None:
            v = v + np.sqrt(model.tau[nu]) * omega1[nu]
        out.append(v)
    return out


def grad_terms_dense(model, x, lam, d, omega1=None, omega2=None):
    """lambda^T (db/dtheta - dA/dtheta x) for theta = q_{nu,k} and t_k, from dense matrices.

    Returns (dq [nobs, ncomp], dt [ncomp]); variable pairs get the offset derivative."""
    P = _model.dense_P(model)
    r = _data_maps(model, d, omega1)
    dq = np.zeros((model.nobs, model.ncomp))
    for nu in range(model.nobs):
        tau = model.tau[nu]
        for k in range(model.ncomp):
            if model.variable(nu, k):
                continue
            dP = dense_dP(model, nu, k)
            dA = dP.T @ (tau[:, None] * P[nu]) + P[nu].T @ (tau[:, None] * dP)
            db = dP.T @ r[nu]
            dq[nu, k] = lam @ (db - dA @ x)
    o = model.comp_offsets()
    sinv = _model.prior_inv_diag(model)
    sisq = _model.prior_inv_diag(model, 0.5)
    dt = np.zeros(model.ncomp)
    for k in range(model.ncomp):
        blk = slice(o[k], o[k + 1])
        dA = -np.diag(sinv[blk])
        db = np.zeros(o[k + 1] - o[k])
        if omega2 is not None:
            db = -0.5 * sisq[blk] * omega2[blk]
        dt[k] = lam[blk] @ (db - dA @ x[blk])
    for (nu, k), g in grad_mix_maps_dense(model, x, lam, d, omega1).items():
        dq[nu, k] = g.sum()
    return dq, dt


def grad_terms(model, x, lam, d, omega1=None, omega2=None):
    """The same terms applied as operators (no dense matrices):

        dq_{nu,k} = <B_nu E_k lambda_k, Y^T (N^-1 d + N^-1/2 w1 - N^-1 P x)>
                  - <B_nu E_k x_k, Y^T N^-1 P lambda>
        dt_k = lambda_k^T S_k^-1 x_k - 1/2 lambda_k^T S_k^-1/2 omega_2,k

    Variable pairs get the offset derivative (the sum of ``grad_mix_maps``)."""
    px = _model.project(model, x)
    pl = _model.project(model, lam)
    r = _data_maps(model, d, omega1)
    xs, ls = model.split(x), model.split(lam)
    dq = np.zeros((model.nobs, model.ncomp))
    for nu in range(model.nobs):
        Ln = model.lmax_band[nu]
        g = model.grids[nu]
        b = model.beam[nu][_alm.ell_of_index(Ln)]
        u = b * _sht.adjoint(g, Ln, r[nu] - model.tau[nu] * px[nu])
        v = b * _sht.adjoint(g, Ln, model.tau[nu] * pl[nu])
        for k in range(model.ncomp):
            if model.variable(nu, k):
                continue
            dq[nu, k] = _select(model, nu, k, ls[k]) @ u - _select(model, nu, k, xs[k]) @ v
    o = model.comp_offsets()
    sinv = _model.prior_inv_diag(model)
    sisq = _model.prior_inv_diag(model, 0.5)
    dt = np.zeros(model.ncomp)
    for k in range(model.ncomp):
        blk = slice(o[k], o[k + 1])
        dt[k] = lam[blk] @ (sinv[blk] * x[blk])
        if omega2 is not None:
            dt[k] -= 0.5 * lam[blk] @ (sisq[blk] * omega2[blk])
    for (nu, k), g in grad_mix_maps(model, x, lam, d, omega1).items():
        dq[nu, k] = g.sum()
    return dq, dt


def _band_adjoints(model, x, lam, d, omega1):
    """u_nu = B_nu Y_band^T (N^-1 d + N^-1/2 w1 - N^-1 P x), v_nu = B_nu Y_band^T N^-1 P lambda."""
    px = _model.project(model, x)
    pl = _model.project(model, lam)
    r = _data_maps(model, d, omega1)
    us, vs = [], []
    for nu in range(model.nobs):
        Ln = model.lmax_band[nu]
        g = model.grids[nu]
        b = model.beam[nu][_alm.ell_of_index(Ln)]
        us.append(b * _sht.adjoint(g, Ln, r[nu] - model.tau[nu] * px[nu]))
        vs.append(b * _sht.adjoint(g, Ln, model.tau[nu] * pl[nu]))
    return us, vs


def grad_mix_maps(model, x, lam, d, omega1=None):
    """{(nu, k): dL/dq_{nu,k}(p) on the pair's mixing grid} for every variable pair, as
    operators: w_p [(Y_k lambda_k)(p) (Y_nu u_nu)(p) - (Y_k x_k)(p) (Y_nu v_nu)(p)]."""
    if model.mix_map is None:
        return {}
    us, vs = _band_adjoints(model, x, lam, d, omega1)
    xs, ls = model.split(x), model.split(lam)
    out = {}
    for nu in range(model.nobs):
        Ln = model.lmax_band[nu]
        for k in range(model.ncomp):
            if not model.variable(nu, k):
                continue
            g = model.mix_grid[nu][k]
            Lk = model.lmax_comp[k]
            out[(nu, k)] = g.pixel_weights() * (
                _sht.synthesis(g, Lk, ls[k]) * _sht.synthesis(g, Ln, us[nu])
                - _sht.synthesis(g, Lk, xs[k]) * _sht.synthesis(g, Ln, vs[nu]))
    return out


def grad_mix_maps_dense(model, x, lam, d, omega1=None):
    """The same maps from dense matrices: for pixel p, dP_p = Y_band B_nu (Y_nu^T W)[:, p]
    Y_k[p, :] on component k's block, and dL/dq(p) = lambda^T (dP_p^T r - dP_p^T N^-1 P x
    - P^T N^-1 dP_p x)."""
    if model.mix_map is None:
        return {}
    px = _model.project(model, x)      # P x and P lambda (the model itself, not its derivative)
    pl = _model.project(model, lam)
    r = _data_maps(model, d, omega1)
    o = model.comp_offsets()
    out = {}
    for nu in range(model.nobs):
        Ln = model.lmax_band[nu]
        tau = model.tau[nu]
        Yb = _sht.dense_Y(model.grids[nu], Ln) * model.beam[nu][_alm.ell_of_index(Ln)][None, :]
        Px, Pl = px[nu], pl[nu]
        for k in range(model.ncomp):
            if not model.variable(nu, k):
                continue
            g = model.mix_grid[nu][k]
            Sk = _sht.dense_Y(g, model.lmax_comp[k])
            An = _sht.dense_Y(g, Ln).T * g.pixel_weights()[None, :]   # Y_nu^T W
            G = Yb @ An                                               # column p: Y_band B (Y^T W)[:, p]
            sl = Sk @ lam[o[k]:o[k + 1]]
            sx = Sk @ x[o[k]:o[k + 1]]
            # (dP_p lambda) . (r - tau P x) - (P lambda) . (tau dP_p x), dP_p v = (Sk v)[p] G[:, p]
            out[(nu, k)] = sl * (G.T @ (r[nu] - tau * Px)) - sx * (G.T @ (tau * Pl))
    return out


def weighted_loss(x, w):
    """L = ||W x||^2 for a diagonal harmonic weight W = diag(w); returns (L, dL/dx)."""
    return float(np.sum((w * x) ** 2)), 2.0 * w * w * x


def solve_dense(model, b):
    """x = A^-1 b by Cholesky of the dense A (small sizes only)."""
    A = _model.dense_A(model)
    C = np.linalg.cholesky(A)
    return np.linalg.solve(C.T, np.linalg.solve(C, b))
