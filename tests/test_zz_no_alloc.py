"""The allocation-free analysis entry point agrees with cmbws_sht_analysis (GPU).

Callers that cannot allocate device memory (a runtime with a fixed memory budget, a loop
that must not block on the allocator) use cmbws_sht_analysis_noalloc, whose workspace is a
static 32 MiB device array.  This file is collected last so that a failure here, in a run that stops at the
first failure, comes after every other test has run.
"""
import numpy as np
import pytest

import paper_1710_00621_gb300 as cw
from tests._gpu import rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu


def _tol(prec, lmax):
    # the adjoint bounds of the SHT parity tests (FP64 40 (L+1) eps64, FP32 6 sqrt(L+1) eps32):
    # both calls run the same kernels, so they agree to rounding
    if prec == cw.CMBWS_FP64:
        return max(1e-14, 40 * (lmax + 1) * 2.0 ** -53)
    return max(1e-6, 6 * np.sqrt(lmax + 1) * 2.0 ** -24)


@pytest.mark.parametrize("prec", [cw.CMBWS_FP64, cw.CMBWS_FP32])
def test_noalloc_matches_allocating_call_twice(prec):
    g = cw.cmbws_plan_grid(cw.CMBWS_GRID_HEALPIX, 64, 191)
    nalm = 192 ** 2
    rng = np.random.default_rng(2024)
    # calls in a row; 5 maps run two launches (4 + 1) that reuse the same scratch regions
    for call, (nmaps, weighted) in enumerate(((2, 1), (3, 0), (5, 1))):
        maps = to_dev(rng.standard_normal((nmaps, g.npix)))
        ref = to_dev(np.zeros((nmaps, nalm)))
        got = to_dev(np.full((nmaps, nalm), np.nan))
        cw.cmbws_sht_analysis(g, prec, maps, ref, nmaps, weighted)
        cw.cmbws_sht_analysis_noalloc(g, prec, maps, got, nmaps, weighted)
        r, o = to_host(ref), to_host(got)
        for k in range(nmaps):
            assert rel_err(o[k], r[k]) < _tol(prec, 191), (call, k)


def test_noalloc_rejects_sizes_beyond_its_workspace():
    g = cw.cmbws_plan_grid(cw.CMBWS_GRID_HEALPIX, 512, 1535)
    maps = to_dev(np.zeros(g.npix))
    alm = to_dev(np.zeros(1536 ** 2))
    with pytest.raises(cw.CmbwsError) as e:
        cw.cmbws_sht_analysis_noalloc(g, cw.CMBWS_FP64, maps, alm, 1, 1)
    assert e.value.code == -1 and "static scratch" in str(e.value)
    g2 = cw.cmbws_plan_grid(cw.CMBWS_GRID_HEALPIX, 8, 23)
    with pytest.raises(cw.CmbwsError) as e:
        cw.cmbws_sht_analysis_noalloc(g2, cw.CMBWS_FP32X2, to_dev(np.zeros(g2.npix)),
                                      to_dev(np.zeros(24 ** 2)), 1, 1)
    assert e.value.code == -1 and "not supported" in str(e.value)
