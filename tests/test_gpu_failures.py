"""Failure paths of the library, injected without faulting the GPU (GPU).

Each failure is made on the host (a NaN in the right-hand side or an inverse-noise map, an
exhausted wall-clock budget, a destroyed handle) or by a bounded device-side wait that a test
makes run out (an mbarrier phase that nothing completes); the kernels return and the
context stays usable, which every test checks by running a correct call afterwards."""
import ctypes

import numpy as np
import pytest

import paper_1710_00621_gb300 as cw
from oracle import grids as og, sht as osht
from tests._gpu import gpu_model, rel_err, to_dev, to_host
from tests._models import multires_small, oracle_model, tiny_workload

pytestmark = pytest.mark.gpu


def test_nan_in_the_right_hand_side_is_a_breakdown():
    work = tiny_workload(15)
    m, inp = oracle_model(work)
    g, _ = gpu_model(work, inp)
    b = np.random.default_rng(1).standard_normal(m.nvec())
    b[17] = np.nan
    x = to_dev(np.zeros(m.nvec()))
    rep = cw.cmbws_cg_solve(g, to_dev(b), x, tol=1e-8, maxiter=50, check=False)
    assert rep["code"] == -5, rep
    # the model still solves a finite system
    b[17] = 0.0
    rep = cw.cmbws_cg_solve(g, to_dev(b), x, tol=1e-8, maxiter=200)
    assert rep["rel_res"] <= 1e-8


def test_nan_in_an_inverse_noise_map_is_rejected_at_creation():
    work = tiny_workload(15)
    m, inp = oracle_model(work)
    bad = dict(inp)
    bad["tau"] = [t.copy() for t in inp["tau"]]
    bad["tau"][1][5] = np.nan
    with pytest.raises(cw.CmbwsError) as e:
        gpu_model(work, bad)
    assert e.value.code == -1 and "not positive and finite" in str(e.value)


def test_exhausted_wall_clock_budget_is_a_timeout():
    work = multires_small(16)
    m, inp = oracle_model(work)
    g, _ = gpu_model(work, inp, cw.CMBWS_FP32)
    b = to_dev(np.random.default_rng(2).standard_normal(m.nvec()))
    x = to_dev(np.zeros(m.nvec()))
    rep = cw.cmbws_cg_solve(g, b, x, tol=1e-12, maxiter=1000, timeout_s=1e-9,
                            cert_prec=cw.CMBWS_FP32X2, check=False)
    assert rep["code"] == -7, rep
    rep = cw.cmbws_cg_solve(g, b, x, tol=1e-6, maxiter=1000, cert_prec=cw.CMBWS_FP32X2)
    assert rep["rel_res"] <= 1e-6


def test_destroyed_and_foreign_handles_are_rejected():
    lib = cw.load_library()
    work = tiny_workload(15)
    m, inp = oracle_model(work)
    g, grids = gpu_model(work, inp)
    x = to_dev(np.zeros(m.nvec()))
    y = to_dev(np.zeros(m.nvec()))
    xp, yp = ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr())
    h = g.handle
    g.close()                                         # destroyed
    assert lib.cmbws_apply_A(h, xp, yp, None) == -1
    assert lib.cmbws_model_destroy(h) == -1           # destroyed twice
    gh = grids[0].handle
    alm = to_dev(np.zeros(16 ** 2))
    mp = to_dev(np.zeros(grids[0].npix))
    grids[0].close()
    assert lib.cmbws_sht_synth(gh, 0, ctypes.c_void_p(alm.data_ptr()), ctypes.c_void_p(mp.data_ptr()),
                               1, None) == -1
    assert lib.cmbws_grid_destroy(gh) == -1
    # a pointer that was never a handle is not dereferenced
    fake = ctypes.c_void_p(x.data_ptr())
    assert lib.cmbws_apply_A(fake, xp, yp, None) == -1
    assert lib.cmbws_sht_synth(fake, 0, ctypes.c_void_p(alm.data_ptr()),
                               ctypes.c_void_p(mp.data_ptr()), 1, None) == -1


@pytest.mark.parametrize("prec", [cw.CMBWS_TF32, cw.CMBWS_3XTF32, cw.CMBWS_BF16, cw.CMBWS_BF16X3])
def test_bounded_mbarrier_wait_runs_out_and_reports_a_timeout(prec):
    """The tensor-core synthesis waits (bounded) on an mbarrier phase that nothing completes:
    every CTA gives up after ~1e5 SM clocks, issues no MMA, frees its tensor memory and writes
    NaN; cmbws_device_status reports CMBWS_ERR_TIMEOUT once, and the next call is correct."""
    g = cw.cmbws_plan_grid(cw.CMBWS_GRID_HEALPIX, 8, 23)
    o = og.healpix(8)
    alm = np.random.default_rng(3).standard_normal((2, 24 ** 2))
    out = to_dev(np.zeros((2, g.npix)))
    cw.cmbws_device_status()                         # clear any earlier record
    cw.cmbws_testing_stall_waits(100000)
    try:
        cw.cmbws_sht_synth(g, prec, to_dev(alm), out, 2)
        with pytest.raises(cw.CmbwsError) as e:
            cw.cmbws_device_status()
        assert e.value.code == -7
    finally:
        cw.cmbws_testing_stall_waits(0)
    assert np.isnan(to_host(out)).any()
    cw.cmbws_device_status()                         # the record was cleared
    cw.cmbws_sht_synth(g, prec, to_dev(alm), out, 2)
    cw.cmbws_device_status()
    got = to_host(out)
    bound = 1.5e-2 if prec == cw.CMBWS_BF16 else 4e-3
    for k in range(2):
        assert rel_err(got[k], osht.synthesis(o, 23, alm[k])) < bound


@pytest.mark.parametrize("prec", [cw.CMBWS_BF16, cw.CMBWS_BF16X3])
def test_tensor_core_adjoint_wait_runs_out_and_reports_a_timeout(prec):
    """The same for the tensor-core adjoint (analysis): every CTA's bounded wait runs out, no
    MMA is issued, the coefficients hold NaN and cmbws_device_status reports CMBWS_ERR_TIMEOUT;
    the next call is correct."""
    g = cw.cmbws_plan_grid(cw.CMBWS_GRID_HEALPIX, 8, 23)
    o = og.healpix(8)
    maps = np.random.default_rng(4).standard_normal((2, g.npix))
    out = to_dev(np.zeros((2, 24 ** 2)))
    cw.cmbws_device_status()
    cw.cmbws_testing_stall_waits(100000)
    try:
        cw.cmbws_sht_analysis(g, prec, to_dev(maps), out, 2, 1)
        with pytest.raises(cw.CmbwsError) as e:
            cw.cmbws_device_status()
        assert e.value.code == -7
    finally:
        cw.cmbws_testing_stall_waits(0)
    assert np.isnan(to_host(out)).any()
    cw.cmbws_device_status()
    cw.cmbws_sht_analysis(g, prec, to_dev(maps), out, 2, 1)
    cw.cmbws_device_status()
    got = to_host(out)
    bound = 1.5e-2 if prec == cw.CMBWS_BF16 else 4e-5
    for k in range(2):
        assert rel_err(got[k], osht.adjoint(o, 23, maps[k], weighted=True)) < bound


def test_solver_reports_a_timed_out_device_wait_as_timeout():
    work = tiny_workload(15)
    m, inp = oracle_model(work)
    g, _ = gpu_model(work, inp, cw.CMBWS_TF32)
    b = to_dev(np.random.default_rng(4).standard_normal(m.nvec()))
    x = to_dev(np.zeros(m.nvec()))
    cw.cmbws_device_status()
    cw.cmbws_testing_stall_waits(100000)
    try:
        rep = cw.cmbws_cg_solve(g, b, x, tol=1e-6, maxiter=50, cert_prec=cw.CMBWS_FP32X2,
                                check=False)
    finally:
        cw.cmbws_testing_stall_waits(0)
    assert rep["code"] == -7, rep
    rep = cw.cmbws_cg_solve(g, b, x, tol=1e-6, maxiter=200, cert_prec=cw.CMBWS_FP32X2)
    assert rep["rel_res"] <= 1e-6
