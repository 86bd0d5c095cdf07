"""The synthesis tile autotuner (cmbws_set_autotune): every tile variant computes the same
transform (bitwise in FP64, to FP32 rounding in FP32), the tuner records its measured choice,
and the default mode leaves results unchanged."""
import numpy as np
import pytest

from oracle import grids as og
from oracle import sht as osht
from tests._gpu import rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu


def _synth(grid, prec, alm, nmaps):
    import paper_1710_00621_gb300 as cw
    import torch
    out = torch.zeros(nmaps * grid.npix, dtype=torch.float64, device="cuda")
    cw.cmbws_sht_synth(grid, prec, alm, out, nmaps)
    return to_host(out)


@pytest.mark.parametrize("kind,n,lmax", [("gl", 47, 47), ("healpix", 32, 95), ("healpix", 128, 383)])
def test_tile_variants_agree_and_tuner_records(kind, n, lmax):
    import paper_1710_00621_gb300 as cw
    nmaps = 3
    rng = np.random.default_rng(8)
    alm_h = rng.standard_normal(nmaps * (lmax + 1) ** 2)
    alm = to_dev(alm_h)
    try:
        for prec, tol in ((cw.CMBWS_FP64, 0.0), (cw.CMBWS_FP32, 1e-5)):
            res = {}
            for mode in (cw.CMBWS_TUNE_DEFAULT, cw.CMBWS_TUNE_HEURISTIC, cw.CMBWS_TUNE_MEASURED):
                cw.cmbws_set_autotune(mode)
                g = cw.cmbws_plan_grid(cw.CMBWS_GRID_GL if kind == "gl" else cw.CMBWS_GRID_HEALPIX,
                                       n + 1 if kind == "gl" else n, lmax)
                res[mode] = _synth(g, prec, alm, nmaps)
                again = _synth(g, prec, alm, nmaps)   # a tuned grid reuses its choice
                assert np.array_equal(again, res[mode])
                t = cw.cmbws_grid_tuning(g, prec, nmaps)
                if mode == cw.CMBWS_TUNE_MEASURED:
                    assert t is not None and len(t["ms"]) == len(cw.SYNTH_TILES)
                    assert all(v > 0 for v in t["ms"])
                    assert t["ms"][t["variant"]] == min(t["ms"])
                else:
                    assert t is None
            for mode in (cw.CMBWS_TUNE_HEURISTIC, cw.CMBWS_TUNE_MEASURED):
                if tol == 0.0:
                    assert np.array_equal(res[mode], res[cw.CMBWS_TUNE_DEFAULT])
                else:
                    assert rel_err(res[mode], res[cw.CMBWS_TUNE_DEFAULT]) < tol
        # and the transform itself against the oracle's (FP64)
        og_grid = og.gauss_legendre(n) if kind == "gl" else og.healpix(n)
        ref = osht.synthesis(og_grid, lmax, alm_h[:(lmax + 1) ** 2])
        assert rel_err(res[cw.CMBWS_TUNE_DEFAULT][:og_grid.npix], ref) < 1e-5
    finally:
        cw.cmbws_set_autotune(cw.CMBWS_TUNE_DEFAULT)


def test_autotune_mode_checked():
    import paper_1710_00621_gb300 as cw
    with pytest.raises(cw.CmbwsError):
        cw.cmbws_set_autotune(3)
