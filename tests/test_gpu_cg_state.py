"""Residual and error history of a solve, and checkpoint / resume of PCG (GPU)."""
import numpy as np
import pytest

import paper_1710_00621_gb300 as cw
from oracle import model as om
from tests._gpu import gpu_model, to_dev, to_host
from tests._models import multires_small, oracle_model, tiny_workload

pytestmark = pytest.mark.gpu


def test_history_tracks_the_residual_and_the_error_to_x_true():
    # Sec. 2.3 / Sec. 5: b = A x_true and the error ||x_i - x_true|| per iteration
    work = tiny_workload(31)
    m, inp = oracle_model(work)
    g, _ = gpu_model(work, inp)
    b = om.apply_A(m, inp["x_true"])
    cw.cmbws_cg_track_error(g, to_dev(inp["x_true"]))
    x = to_dev(np.zeros(m.nvec()))
    rep = cw.cmbws_cg_solve(g, to_dev(b), x, tol=1e-10, maxiter=500)
    res, err = cw.cmbws_cg_history(g)
    assert res.size == err.size == rep["iters"]
    # the recorded residuals are the solver's own: the last is below the stopping point
    assert res[-1] <= 1e-10 and res[0] < 1.0
    # the error record agrees with the final solution's distance to x_true
    final = np.linalg.norm(to_host(x) - inp["x_true"]) / np.linalg.norm(inp["x_true"])
    assert abs(err[-1] - final) <= 1e-9 * max(final, 1e-12) + 1e-14
    assert err[-1] < 1e-6 and err[0] > err[-1]
    cw.cmbws_cg_track_error(g, None)
    x.zero_()
    cw.cmbws_cg_solve(g, to_dev(b), x, tol=1e-6, maxiter=500)
    res2, err2 = cw.cmbws_cg_history(g)
    assert np.all(err2 == -1.0) and res2.size > 0


@pytest.mark.parametrize("prec", [cw.CMBWS_FP64, cw.CMBWS_FP32X2])
def test_interrupted_and_resumed_solve_is_bitwise_the_uninterrupted_one(prec):
    work = multires_small(64)
    m, inp = oracle_model(work)
    d = [mp + n for mp, n in zip(om.project(m, inp["x_true"]), inp["noise"])]
    b = to_dev(om.rhs(m, d))
    g, _ = gpu_model(work, inp, prec)
    x_ref = to_dev(np.zeros(m.nvec()))
    ref = cw.cmbws_cg_solve(g, b, x_ref, tol=1e-10, maxiter=200, cert_prec=prec)
    assert ref["code"] == 0 and ref["iters"] > 6
    cw.cmbws_cg_checkpointing(g, True)
    x1 = to_dev(np.zeros(m.nvec()))
    part = cw.cmbws_cg_solve(g, b, x1, tol=1e-10, maxiter=5, cert_prec=prec, check=False)
    assert part["code"] == -6 and part["iters"] == 5
    n = m.nvec()
    dd, rr, pp = (to_dev(np.zeros(n)) for _ in range(3))
    sc = cw.cmbws_cg_state_export(g, dd, rr, pp)
    assert sc[0] == 5
    # resume on a second model built from the same description (as after a restart)
    g2, _ = gpu_model(work, inp, prec)
    x2 = to_dev(np.zeros(m.nvec()))                  # the interrupted solve's initial guess
    rep = cw.cmbws_cg_resume(g2, b, x2, dd, rr, pp, sc, tol=1e-10, maxiter=200, cert_prec=prec)
    assert rep["code"] == 0 and rep["iters"] == ref["iters"]
    np.testing.assert_array_equal(to_host(x2), to_host(x_ref))
    assert rep["rel_res"] == ref["rel_res"]


def test_checkpoint_errors():
    work = tiny_workload(15)
    m, inp = oracle_model(work)
    g32, _ = gpu_model(work, inp, cw.CMBWS_FP32)
    with pytest.raises(cw.CmbwsError) as e:
        cw.cmbws_cg_checkpointing(g32, True)
    assert e.value.code == -1
    g, _ = gpu_model(work, inp)
    cw.cmbws_cg_checkpointing(g, True)
    b = to_dev(om.apply_A(m, inp["x_true"]))
    x = to_dev(np.zeros(m.nvec()))
    cw.cmbws_cg_solve(g, b, x, tol=1e-8, maxiter=500)           # converges: no checkpoint
    v = to_dev(np.zeros(m.nvec()))
    with pytest.raises(cw.CmbwsError) as e:
        cw.cmbws_cg_state_export(g, v, v, v)
    assert e.value.code == -1 and "no checkpoint" in str(e.value)
