"""Helpers for GPU parity tests: the same seeded inputs handed to the library."""
import numpy as np

import paper_1710_00621_gb300 as cw


def torch_dev():
    import torch
    return torch.device("cuda:0")


def to_dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=torch_dev())


def to_host(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


class GridCache:
    """One library grid per distinct (kind, n, lmax): bands that share it form one group."""

    def __init__(self):
        self.grids = {}

    def get(self, band):
        key = (band.grid, band.n, band.lmax)
        if key not in self.grids:
            kind = cw.CMBWS_GRID_GL if band.grid == "gl" else cw.CMBWS_GRID_HEALPIX
            n = band.n + 1 if band.grid == "gl" else band.n
            self.grids[key] = cw.cmbws_plan_grid(kind, n, band.lmax)
        return self.grids[key]


def gpu_model(work, inp, prec=cw.CMBWS_FP64, cache=None, mix=None):
    """mix: optional (mix_grid_lmax[nu][k] or None, mix_map[nu][k] numpy or None) for variable
    mixing on Gauss-Legendre grids."""
    cache = cache or GridCache()
    grids = [cache.get(b) for b in work.bands]
    ninv = [to_dev(t) for t in inp["tau"]]
    mg = mm = None
    if mix is not None:
        lm, maps = mix
        gl = {}
        mg = [[None] * len(work.comps) for _ in work.bands]
        mm = [[None] * len(work.comps) for _ in work.bands]
        for nu in range(len(work.bands)):
            for k in range(len(work.comps)):
                if maps[nu][k] is None:
                    continue
                if lm[nu][k] not in gl:
                    gl[lm[nu][k]] = cw.cmbws_plan_grid(cw.CMBWS_GRID_GL, lm[nu][k] + 1, lm[nu][k])
                mg[nu][k] = gl[lm[nu][k]]
                mm[nu][k] = to_dev(maps[nu][k])
    m = cw.cmbws_model_create([c.lmax for c in work.comps], grids, inp["beams"], inp["cl"], ninv,
                              inp["q"], prec, mix_grids=mg, mix_maps=mm)
    return m, grids


def rel_err(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))
