"""Mask-restricted preconditioner with a multigrid V-cycle (oracle, test-only).

Sec. 4 of the paper: with the mask carried by the mixing maps, the CR system under the
mask only sees the prior.  With Z = (select pixels in the mask) Y R, R = diag(r_l) a
low-pass filter (Eq. rl: r_l = exp(-beta l^2 (l+1)^2), r^2_{L/2} = 0.05),

    M_mask = Z^T (Z S^-1 Z^T)^-1 Z          (Eq. M_mask)
    M_add  = M_PI + M_mask,

and (Z S^-1 Z^T)^-1 = G^-1, G = Y D Y^T (Eq. W, d_l = r_l^2 / C_l, Y restricted to the
mask pixels), is approximated by one multigrid V-cycle (Sec. 4.4, the basic V-cycle):

* levels: HEALPix grids with Nside halved per level; a coarse pixel belongs to the mask
  when all four of its fine pixels do; band-limit halved per level;
* restriction I_h^H = Y_H R_H Y_h^T W_h (harmonic), R_H the Eq. rl filter at L_H;
  interpolation its transpose;
* coarse operators G_H = Y_H D_H Y_H^T with d_H = r_H^2 d_h;
* smoother M_h = omega diag(G_h)^-1, omega = 0.2, diag(G_h) = sum_l (2l+1)/(4 pi) d_{h,l}
  (constant: G is rotation invariant).  The paper picks omega = 0.2 so that omega M G has
  eigenvalues below 2 on its grids (L = 3 Nside); since lambda_max(G) <= max_l d_l Npix/(4 pi),
  omega is capped at diag(G) / (max_l d_l Npix / (4 pi)) on grids with more pixels per mode;
* bottom level: SVD (here: symmetric eigen-) pseudo-inverse of the dense G, eigenvalues
  below 1e-5 of the largest dropped (the scales the bottom solve is for lie well above;
  the filtered high-l directions below would only amplify rounding).

The coarse-pixel rule needs the parent of a fine pixel: the coarse pixel containing the
fine pixel's centre, found with HEALPix ang2pix (Gorski et al. 2005 geometry: in the
equatorial zone pixel boundaries are the lines t -/+ 3z/4 = const in (t = 2 phi / pi, z),
in the polar caps the lines t' N sqrt(3 (1 - |z|)) = const with t' = t mod 1).

Parity: pinned (tests/test_oracle_maskmg.py) -- ang2pix of every pixel centre returns the
pixel, every coarse pixel has exactly four children, the coarse mask equals a brute-force
rule (a coarse pixel kept iff the four fine pixels nearest its centre, its children, are
all masked), the filter of Eq. rl has the l^2 (l+1)^2 shape with r^2 = 0.05 at L/2 (beta
recovered from a single value), the bottom solve is a
pseudo-inverse of the dense G, the V-cycle operator is symmetric and accelerates CG on G,
M_mask with an exact inner inverse equals the dense Eq. M_mask, and M_add reduces the
PCG iteration count of a masked problem against M_PI (the paper's masked benchmark).  The
optimized V-cycle with J kept exactly reproduces the basic one (its reorganisation is exact);
with J ~ I it is symmetric, removes large-scale error and needs about the basic cycle's
iterations in the masked solve.
The multi-level V-cycle itself is a heuristic approximation with no closed form.
"""
import numpy as np

from . import alm as _alm
from . import grids as _grids
from . import model as _model
from . import precond as _precond
from . import sht as _sht

OMEGA = 0.2


def ang2pix_ring(nside, theta, phi):
    """HEALPix ring-scheme pixel index of points (theta, phi)."""
    N = int(nside)
    z = np.cos(np.asarray(theta, dtype=np.float64))
    t = np.mod(np.asarray(phi, dtype=np.float64), 2 * np.pi) / (0.5 * np.pi)   # [0, 4)
    out = np.empty(z.shape, dtype=np.int64)
    ncap = 2 * N * (N - 1)
    npix = 12 * N * N
    eq = np.abs(z) <= 2.0 / 3.0
    # equatorial zone: lattice of the two families of boundary lines
    a = N * (0.5 + t[eq])
    b = N * 0.75 * z[eq]
    jp = np.floor(a - b).astype(np.int64)
    jm = np.floor(a + b).astype(np.int64)
    ir = N + 1 + jp - jm                      # 1 .. 2N + 1 within the belt
    shifted = ((ir - 1) % 2) == 0             # global ring N - 1 + ir: shifted when (i - N) even
    j = (jp + jm + 1 - N - shifted.astype(np.int64)) // 2
    out[eq] = ncap + (ir - 1) * 4 * N + np.mod(j, 4 * N)
    # polar caps
    pc = ~eq
    zz = np.abs(z[pc])
    tt = t[pc]
    face = np.floor(tt).astype(np.int64)
    tp = tt - face
    tmp = N * np.sqrt(3.0 * (1.0 - zz))
    jp = np.floor(tp * tmp).astype(np.int64)
    jm = np.floor((1.0 - tp) * tmp).astype(np.int64)
    ir = jp + jm + 1                          # ring counted from the nearer pole
    ip = face * ir + np.minimum(jp, ir - 1)
    north = z[pc] > 0
    out[np.where(pc)[0][north]] = 2 * ir[north] * (ir[north] - 1) + ip[north]
    south = ~north
    out[np.where(pc)[0][south]] = npix - 2 * ir[south] * (ir[south] + 1) + ip[south]
    return out


def coarse_parent(nside_fine):
    """Parent (Nside/2, ring scheme) of every pixel of the Nside grid."""
    g = _grids.healpix(nside_fine)
    th, ph = g.pixel_angles()
    return ang2pix_ring(nside_fine // 2, th, ph)


def coarse_mask(nside_fine, mask):
    """A coarse pixel is in the mask when all four of its fine pixels are."""
    par = coarse_parent(nside_fine)
    nc = 12 * (nside_fine // 2) ** 2
    cnt = np.bincount(par, minlength=nc)
    inside = np.bincount(par, weights=mask.astype(np.float64), minlength=nc)
    return (inside == 4) & (cnt == 4)


def rl_filter(L, lfull):
    """Eq. rl: r_l = exp(-beta l^2 (l+1)^2) with r^2 at L/2 equal to 0.05, for l <= lfull."""
    h = 0.5 * L
    beta = -np.log(0.05) / (2.0 * h * h * (h + 1.0) ** 2) if L > 0 else 0.0
    l = np.arange(lfull + 1, dtype=np.float64)
    return np.exp(-beta * l * l * (l + 1.0) ** 2)


def _scale(packed, L, f):
    return packed * f[_alm.ell_of_index(L)]


def _retrunc(packed, lin, lout):
    return _model._retruncate(packed, lin, lout)


class Level:
    def __init__(self, nside, L, mask, d):
        self.nside, self.L = nside, L
        self.grid = _grids.healpix(nside)
        self.mask = mask.astype(bool)
        self.d = d                                           # d_l, l <= L
        self.w = 4.0 * np.pi / (12 * nside * nside)          # HEALPix quadrature weight
        l = np.arange(L + 1)
        dg = float(np.sum((2 * l + 1) / (4 * np.pi) * d))
        # omega M G must stay below 2 (Sec. 4.4); lambda_max(G) <= max d_l Npix / (4 pi), so on
        # grids with more pixels per harmonic mode than the paper's (L = 3 Nside) omega is capped
        bound = float(np.max(d)) * self.grid.npix / (4 * np.pi)
        omega = min(OMEGA, dg / bound) if bound > 0 else OMEGA
        self.smooth = omega / dg
        self.rH = None                                       # restriction filter to the next level
        self.Gp = None                                       # bottom: pseudo-inverse on mask pixels

    def G(self, x):
        """G_h x = P Y D Y^T P^T x (x: full-sky map, zero outside the mask)."""
        xm = np.where(self.mask, x, 0.0)
        a = _sht.adjoint(self.grid, self.L, xm)
        y = _sht.synthesis(self.grid, self.L, _scale(a, self.L, self.d))
        return np.where(self.mask, y, 0.0)


def build_levels(nside0, L0, mask0, cinv, max_bottom=400, rcond=1e-5):
    """The level hierarchy for component prior C^-1 = cinv[l] (l <= L0)."""
    r0 = rl_filter(L0, L0)
    d = r0 * r0 * np.asarray(cinv[:L0 + 1], dtype=np.float64)
    levels = [Level(nside0, L0, mask0, d)]
    while True:
        h = levels[-1]
        if int(h.mask.sum()) <= max_bottom or h.nside < 2 or h.L < 2:
            break
        mH = coarse_mask(h.nside, h.mask)
        if not mH.any():
            break
        LH = h.L // 2
        rH = rl_filter(LH, LH)
        h.rH = rH
        levels.append(Level(h.nside // 2, LH, mH, rH * rH * h.d[:LH + 1]))
    b = levels[-1]
    b.rH = None
    idx = np.where(b.mask)[0]
    Y = _sht.dense_Y(b.grid, b.L)[idx]
    G = (Y * b.d[_alm.ell_of_index(b.L)][None, :]) @ Y.T
    ev, V = np.linalg.eigh(G)
    keep = ev > rcond * ev.max() if ev.size else ev
    inv = np.zeros_like(ev)
    inv[keep] = 1.0 / ev[keep]
    b.Gp = (V * inv[None, :]) @ V.T
    b.idx = idx
    return levels


def restrict(h, H, r):
    """I_h^H r = P_H Y_H R_H Y_h^T W_h r."""
    a = _sht.adjoint(h.grid, h.L, np.where(h.mask, r, 0.0) * h.w)
    a = _scale(_retrunc(a, h.L, H.L), H.L, h.rH)
    return np.where(H.mask, _sht.synthesis(H.grid, H.L, a), 0.0)


def interpolate(h, H, c):
    """(I_h^H)^T c = P_h W_h Y_h R_H Y_H^T P_H^T c."""
    a = _sht.adjoint(H.grid, H.L, np.where(H.mask, c, 0.0))
    a = _retrunc(_scale(a, H.L, h.rH), H.L, h.L)
    return np.where(h.mask, h.w * _sht.synthesis(h.grid, h.L, a), 0.0)


def vcycle(levels, b, k=0):
    """Basic V-cycle approximating G_k^-1 b (Sec. 4.4)."""
    h = levels[k]
    if h.Gp is not None:
        x = np.zeros_like(b)
        x[h.idx] = h.Gp @ b[h.idx]
        return x
    x = h.smooth * np.where(h.mask, b, 0.0)                    # pre-smoothing
    r = b - h.G(x)                                             # residual
    c = vcycle(levels, restrict(h, levels[k + 1], r), k + 1)   # coarse correction
    x = x + interpolate(h, levels[k + 1], c)
    x = x + h.smooth * np.where(h.mask, b - h.G(x), 0.0)       # post-smoothing
    return x


def vcycle_optimized(levels, b, k=0, exact_J=False):
    """Optimized V-cycle (Sec. 4.4, Fig. code:mg): I_h^H = Y_H R_H Y_h^T W_h and
    G_h = P Y_h D_h Y_h^T P inserted, so that restriction and interpolation share their
    transforms with the applications of G_h.  With J = Y_h^T W_h P Y_h (P: the mask) kept
    exactly (exact_J) it is the basic V-cycle reorganised; with J ~ I, as the paper uses,
    a level costs 6 SHTs instead of 8: Y_h^T (L_h), Y_h^T W_h (L_H), Y_H and Y_H^T (L_H on
    the coarse grid), Y_h (L_H) and Y_h (L_h)."""
    h = levels[k]
    if h.Gp is not None:
        x = np.zeros_like(b)
        x[h.idx] = h.Gp @ b[h.idx]
        return x
    H = levels[k + 1]
    bm = np.where(h.mask, b, 0.0)
    x = h.smooth * bm                                                    # pre-smoothing
    u = _sht.adjoint(h.grid, h.L, x)                                     # u = Y_h^T x

    def J(a, La):       # Y_h^T W_h P Y_h a, coefficients a at band-limit La -> L_h
        f = np.where(h.mask, h.w * _sht.synthesis(h.grid, La, a), 0.0)
        return _sht.adjoint(h.grid, h.L, f)

    Du = _scale(u, h.L, h.d)
    JDu = J(Du, h.L) if exact_J else Du
    rt = _sht.adjoint(h.grid, H.L, bm * h.w) - _retrunc(JDu, h.L, H.L)  # Y_h^T W_h b - J D u
    rH = np.where(H.mask, _sht.synthesis(H.grid, H.L, _scale(rt, H.L, h.rH)), 0.0)
    cH = vcycle_optimized(levels, rH, k + 1, exact_J)                    # coarse correction
    ct = _scale(_sht.adjoint(H.grid, H.L, np.where(H.mask, cH, 0.0)), H.L, h.rH)
    x = x + np.where(h.mask, h.w * _sht.synthesis(h.grid, H.L, ct), 0.0)  # x += W_h Y_h c~
    Jc = J(ct, H.L) if exact_J else _retrunc(ct, H.L, h.L)
    y = _sht.synthesis(h.grid, h.L, _scale(u + Jc, h.L, h.d))           # G_h x = Y D Y^T x
    return x + h.smooth * np.where(h.mask, b - y, 0.0)                   # post-smoothing


class MaskPrecond:
    """M_mask for component `comp` of a model, on a HEALPix mask grid (Nside0, mask0 bool).
    cycle: "basic" or "optimized" (J ~ I)."""

    def __init__(self, model, comp, nside0, mask0, max_bottom=400, cycle="basic"):
        if cycle not in ("basic", "optimized"):
            raise ValueError("cycle must be 'basic' or 'optimized'")
        self.cycle = cycle
        cl = model.cl[comp]
        if cl is None:
            raise ValueError("the mask preconditioner needs a prior on the component")
        self.comp = comp
        self.Lk = model.lmax_comp[comp]
        self.L0 = min(3 * nside0 - 1, self.Lk)
        cinv = np.where(np.isfinite(cl), 1.0 / np.asarray(cl, dtype=np.float64), 0.0)
        self.levels = build_levels(nside0, self.L0, np.asarray(mask0, dtype=bool), cinv, max_bottom)
        self.r0 = rl_filter(self.L0, self.L0)

    def apply(self, model, r):
        """z = M_mask r (stacked vectors; only component `comp` is touched)."""
        o = model.comp_offsets()
        k = self.comp
        rk = np.asarray(r[o[k]:o[k + 1]], dtype=np.float64)
        h = self.levels[0]
        a = _scale(_retrunc(rk, self.Lk, self.L0), self.L0, self.r0)
        b = np.where(h.mask, _sht.synthesis(h.grid, self.L0, a), 0.0)          # Z r
        x = vcycle(self.levels, b) if self.cycle == "basic" else vcycle_optimized(self.levels, b)
        u = _sht.adjoint(h.grid, self.L0, np.where(h.mask, x, 0.0))            # Z^T x
        z = np.zeros(model.nvec())
        z[o[k]:o[k + 1]] = _retrunc(_scale(u, self.L0, self.r0), self.L0, self.Lk)
        return z


def apply_M_add(model, masks, r, Up=None):
    """M_add r = M_PI r + sum of the mask preconditioners (Sec. 4.2)."""
    z = _precond.apply_precond(model, r, Up)
    for mp in masks:
        z = z + mp.apply(model, r)
    return z
