"""Helpers that turn skygen workloads into oracle models (test-only)."""
import numpy as np

import skygen
from oracle import grids as ogrids
from oracle.model import Model


def band_grid(b):
    if b.grid == "gl":
        return ogrids.gauss_legendre(b.n, b.nphi)
    return ogrids.healpix(b.n)


def grid_coords(g):
    th, ph = g.pixel_angles()
    return np.cos(th), ph


def oracle_model(work, flat=False, mix_maps=None, mix_grids=None):
    """Oracle Model + drawn inputs for a skygen workload.

    flat=True replaces tau by w / sigma^2 (inverse noise flat per unit area, T = I)."""
    gs = [band_grid(b) for b in work.bands]
    coords = [grid_coords(g) for g in gs]
    weights = [g.pixel_weights() for g in gs]
    inp = skygen.make_inputs(work, coords, weights)
    taus = inp["tau"]
    if flat:
        taus = [w / b.sigma ** 2 for w, b in zip(weights, work.bands)]
        inp["tau"] = taus
        inp["cl"] = skygen.prior_amplitudes(work, taus, weights)
    m = Model(lmax_comp=[c.lmax for c in work.comps], grids=gs,
              lmax_band=[b.lmax for b in work.bands], beam=inp["beams"], cl=inp["cl"],
              tau=taus, q=inp["q"], mix_grid=mix_grids, mix_map=mix_maps)
    return m, inp


def tiny_workload(L=15):
    w = skygen.tiny_plain()
    for b in w.bands:
        b.n = b.lmax = L
    for c in w.comps:
        c.lmax = L
    w.name = f"tiny_gl{L}"
    return w


def multires_small(scale=64):
    return skygen.multires_fullsky(scale=scale)


def split_model(m, fractions=(0.5, 0.5)):
    """Each band of an oracle Model split into detector subsets: the same grid, beam and
    mixing, inverse noise c_h tau (sum of c_h = 1 for a split of one channel's hits).
    Returns (model, groups) with groups[nu] the indices of band nu's subsets."""
    from dataclasses import replace
    nb = len(fractions)
    idx = [nu for nu in range(m.nobs) for _ in range(nb)]
    sm = replace(m, grids=[m.grids[nu] for nu in idx], lmax_band=[m.lmax_band[nu] for nu in idx],
                 beam=[m.beam[nu] for nu in idx],
                 tau=[c * m.tau[nu] for nu in range(m.nobs) for c in fractions],
                 q=np.repeat(np.asarray(m.q), nb, axis=0),
                 mix_grid=None if m.mix_grid is None else [m.mix_grid[nu] for nu in idx],
                 mix_map=None if m.mix_map is None else [m.mix_map[nu] for nu in idx])
    groups = [list(range(nu * nb, (nu + 1) * nb)) for nu in range(m.nobs)]
    return sm, groups
