"""Data model, projection P and the CR system A (oracle, test-only).

Follows Sec. 2.2-2.3 of the paper:

* d = P s + n (Eq. block-data-model), N_nu = Var(n_nu) diagonal in pixels,
  tau_nu = diag(N_nu^-1) given as a pixel map per band.
* P_{nu,k} = Y_nu B_nu Q~_{nu,k} (Eq. P); B_nu = diag(b_{nu,l}).
* Q~_{nu,k} = Y^T W Q Y on a mixing grid (Eq. Q), or the scalar q_{nu,k} I
  when the mixing map is spatially constant.  Its output is truncated at
  L_nu and its input has band-limit L_k (Sec. 2.2 allows the truncation).
* S = diag(C_{k,l}); "no prior" is C^-1 = 0 (Sec. 3.3).
* A = S^-1 + P^T N^-1 P (Eq. A).
* b = P^T N^-1 d + P^T N^-1/2 omega_1 + S^-1/2 omega_2.  The paper prints
  S^-1 omega_2; the oracle reads it as S^-1/2 omega_2, the only choice for
  which the solution is a draw from the posterior (Var(b) = A).

A stacked vector holds the components one after the other, each as
(L_k+1)^2 packed coefficients (``oracle.alm``).

Parity: pinned (tests/test_oracle_model.py) -- symmetry and positive
definiteness of A (Sec. 2.3), the closed-form diagonal Wiener filter of
``oracle.closed_form`` for flat noise per unit area, and dense-vs-operator
agreement.
"""
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import alm as _alm
from . import sht as _sht


@dataclass
class Model:
    lmax_comp: List[int]                 # L_k
    grids: list                          # band grids (oracle.grids.RingGrid)
    lmax_band: List[int]                 # L_nu
    beam: List[np.ndarray]               # b_{nu,l}, l = 0..L_nu
    cl: List[Optional[np.ndarray]]       # C_{k,l}, l = 0..L_k; None = no prior; inf = no prior at l
    tau: List[np.ndarray]                # diag(N_nu^-1) on the band grid
    q: np.ndarray                        # [nobs, ncomp] scalar mixing (used when mix_map is None)
    mix_grid: Optional[list] = None      # [nobs][ncomp] RingGrid or None (variable mixing)
    mix_map: Optional[list] = None       # [nobs][ncomp] q_{nu,k}(n) on mix_grid (incl. mask) or None

    @property
    def ncomp(self):
        return len(self.lmax_comp)

    @property
    def nobs(self):
        return len(self.grids)

    def comp_offsets(self):
        n = [_alm.nalm(L) for L in self.lmax_comp]
        return np.concatenate([[0], np.cumsum(n)]).astype(np.int64)

    def nvec(self):
        return int(self.comp_offsets()[-1])

    def split(self, x):
        o = self.comp_offsets()
        return [np.asarray(x[o[k]:o[k + 1]], dtype=np.float64) for k in range(self.ncomp)]

    def stack(self, parts):
        return np.concatenate(parts)

    def variable(self, nu, k):
        return self.mix_map is not None and self.mix_map[nu][k] is not None


def _retruncate(packed, lin, lout):
    """Copy coefficients from band-limit lin to lout (zero-pad or truncate)."""
    lw = max(lin, lout)
    return _alm.from_2d(_alm.to_2d(packed, lin, lw), lout)


def mix_forward(model, nu, k, xk):
    """Q~_{nu,k} x_k: band-limit L_k -> L_nu (Eq. Q)."""
    Lk, Ln = model.lmax_comp[k], model.lmax_band[nu]
    if not model.variable(nu, k):
        return model.q[nu, k] * _retruncate(xk, Lk, Ln)
    g = model.mix_grid[nu][k]
    f = _sht.synthesis(g, Lk, xk) * model.mix_map[nu][k]
    return _sht.analysis(g, Ln, f)


def mix_adjoint(model, nu, k, u):
    """Q~_{nu,k}^T u: band-limit L_nu -> L_k (the transpose Y_in^T Q W Y_out)."""
    Lk, Ln = model.lmax_comp[k], model.lmax_band[nu]
    if not model.variable(nu, k):
        return model.q[nu, k] * _retruncate(u, Ln, Lk)
    g = model.mix_grid[nu][k]
    f = _sht.synthesis(g, Ln, u) * (model.mix_map[nu][k] * g.pixel_weights())
    return _sht.adjoint(g, Lk, f)


def beam_apply(b, packed, lmax):
    return packed * b[_alm.ell_of_index(lmax)]


def project(model, x):
    """P x: stacked components -> list of band maps."""
    xs = model.split(x)
    out = []
    for nu in range(model.nobs):
        Ln = model.lmax_band[nu]
        a = np.zeros(_alm.nalm(Ln))
        for k in range(model.ncomp):
            a += mix_forward(model, nu, k, xs[k])
        a = beam_apply(model.beam[nu], a, Ln)
        out.append(_sht.synthesis(model.grids[nu], Ln, a))
    return out


def project_adjoint(model, maps):
    """P^T applied to a list of band maps -> stacked components."""
    ys = [np.zeros(_alm.nalm(L)) for L in model.lmax_comp]
    for nu in range(model.nobs):
        Ln = model.lmax_band[nu]
        u = _sht.adjoint(model.grids[nu], Ln, maps[nu])
        u = beam_apply(model.beam[nu], u, Ln)
        for k in range(model.ncomp):
            ys[k] += mix_adjoint(model, nu, k, u)
    return model.stack(ys)


def prior_inv_diag(model, power=1.0):
    """Diagonal of S^-power as a stacked vector (0 where there is no prior)."""
    parts = []
    for k, L in enumerate(model.lmax_comp):
        ell = _alm.ell_of_index(L)
        c = model.cl[k]
        if c is None:
            parts.append(np.zeros(ell.size))
            continue
        c = np.asarray(c, dtype=np.float64)[ell]
        with np.errstate(divide="ignore"):
            v = np.where(np.isfinite(c), c ** (-power), 0.0)
        parts.append(v)
    return np.concatenate(parts)


def apply_A(model, x):
    """A x = S^-1 x + P^T N^-1 P x (Eq. A)."""
    x = np.asarray(x, dtype=np.float64)
    maps = project(model, x)
    maps = [m * t for m, t in zip(maps, model.tau)]
    return prior_inv_diag(model) * x + project_adjoint(model, maps)


def rhs(model, d, omega1=None, omega2=None):
    """b = P^T N^-1 d + P^T N^-1/2 omega_1 + S^-1/2 omega_2 (Sec. 2.3, read with S^-1/2)."""
    maps = [dn * t for dn, t in zip(d, model.tau)]
    if omega1 is not None:
        maps = [m + np.sqrt(t) * w for m, t, w in zip(maps, model.tau, omega1)]
    b = project_adjoint(model, maps)
    if omega2 is not None:
        b = b + prior_inv_diag(model, 0.5) * omega2
    return b


def dense_P(model):
    """Dense P as a list of per-band matrices [npix_nu, nvec] (small sizes only)."""
    n = model.nvec()
    eye = np.eye(n)
    cols = [project(model, eye[:, j]) for j in range(n)]
    return [np.stack([c[nu] for c in cols], axis=1) for nu in range(model.nobs)]


def dense_A(model):
    """Dense A = S^-1 + sum_nu P_nu^T diag(tau_nu) P_nu, built from explicit Y (small sizes only)."""
    n = model.nvec()
    o = model.comp_offsets()
    A = np.diag(prior_inv_diag(model))
    for nu in range(model.nobs):
        Ln = model.lmax_band[nu]
        Y = _sht.dense_Y(model.grids[nu], Ln)
        # M_nu = B_nu [Q~_{nu,1} ... Q~_{nu,K}] as a dense (L_nu+1)^2 x n matrix
        M = np.zeros((_alm.nalm(Ln), n))
        for k in range(model.ncomp):
            Lk = model.lmax_comp[k]
            for j in range(_alm.nalm(Lk)):
                e = np.zeros(_alm.nalm(Lk))
                e[j] = 1.0
                M[:, o[k] + j] = mix_forward(model, nu, k, e)
        M = M * model.beam[nu][_alm.ell_of_index(Ln)][:, None]
        P = Y @ M
        A += P.T @ (model.tau[nu][:, None] * P)
    return A
