"""CUDA-graph replay of the solvers' operator applies (cmbws_model_set_graphs): the same
launches as the eager applies, so the solutions are bitwise equal."""
import numpy as np
import pytest

from oracle import model as omodel
from tests._gpu import gpu_model, rel_err, to_dev, to_host
from tests._models import multires_small, oracle_model, tiny_workload
from tests.test_oracle_maskmg import _masked_model
from tests.test_gpu_maskmg import _gpu_masked

pytestmark = pytest.mark.gpu


def _solve(gm, b, **kw):
    import paper_1710_00621_gb300 as cw
    import torch
    x = torch.zeros_like(b)
    rep = cw.cmbws_cg_solve(gm, b, x, **kw)
    return to_host(x), rep


def _same(gm, b, **kw):
    """Eager, then graphs on twice (capture, then replay): identical solutions and reports."""
    import paper_1710_00621_gb300 as cw
    cw.cmbws_model_set_graphs(gm, False)
    x0, r0 = _solve(gm, b, **kw)
    cw.cmbws_model_set_graphs(gm, True)
    for _ in range(2):
        x1, r1 = _solve(gm, b, **kw)
        assert np.array_equal(x0, x1)
        for key in ("iters", "outer", "n_sht", "status"):
            assert r0[key] == r1[key], (key, r0[key], r1[key])
        assert r0["rel_res"] == r1["rel_res"]
    cw.cmbws_model_set_graphs(gm, False)
    return x0, r0


def test_graphs_tiny_fp64():
    import paper_1710_00621_gb300 as cw
    w = tiny_workload(15)
    m, inp = oracle_model(w)
    gm, _ = gpu_model(w, inp, cw.CMBWS_FP64)
    b = to_dev(omodel.apply_A(m, inp["x_true"]))
    x, rep = _same(gm, b, tol=1e-10, maxiter=500, precond=1)
    assert rep["rel_res"] <= 1e-10 and rel_err(x, inp["x_true"]) < 1e-7


def test_graphs_multires_fp32_refined_and_M_diag():
    import paper_1710_00621_gb300 as cw
    w = multires_small(32)
    m, inp = oracle_model(w)
    gm, _ = gpu_model(w, inp, cw.CMBWS_FP32)
    b = to_dev(omodel.apply_A(m, inp["x_true"]))
    for pc in (1, 3):
        x, rep = _same(gm, b, tol=1e-7, maxiter=2000, precond=pc, cert_prec=cw.CMBWS_FP32X2)
        assert rep["status"] == 0 and rep["outer"] >= 2


def test_graphs_masked_M_add_and_cycle_change():
    import paper_1710_00621_gb300 as cw
    m, inp, mask = _masked_model()
    gm, keep = _gpu_masked(m, inp, mask, cw.CMBWS_FP32)
    b = to_dev(omodel.apply_A(m, inp["x_true"]))
    kw = dict(tol=1e-6, maxiter=3000, precond=2, cert_prec=cw.CMBWS_FP32X2)
    x_basic, _ = _same(gm, b, **kw)
    # a preconditioner change drops the captured graphs: the replayed solve follows it
    cw.cmbws_model_set_graphs(gm, True)
    _solve(gm, b, **kw)
    cw.cmbws_model_set_vcycle(gm, cw.CMBWS_VCYCLE_OPTIMIZED)
    x_opt_graph, _ = _solve(gm, b, **kw)
    cw.cmbws_model_set_graphs(gm, False)
    x_opt_eager, _ = _solve(gm, b, **kw)
    assert np.array_equal(x_opt_graph, x_opt_eager)
    assert not np.array_equal(x_opt_eager, x_basic)


def test_graphs_with_profiling_fall_back_to_eager():
    import paper_1710_00621_gb300 as cw
    w = tiny_workload(15)
    m, inp = oracle_model(w)
    gm, _ = gpu_model(w, inp, cw.CMBWS_FP64)
    b = to_dev(omodel.apply_A(m, inp["x_true"]))
    cw.cmbws_model_set_graphs(gm, True)
    cw.cmbws_profile_read(reset=True)
    cw.cmbws_profile_enable(True)
    try:
        x1, r1 = _solve(gm, b, tol=1e-10, maxiter=500, precond=1)
    finally:
        cw.cmbws_profile_enable(False)
    prof = cw.cmbws_profile_read(reset=True)
    launches = sum(v[1] for v in prof.values())
    assert launches > 10 * r1["iters"]      # every apply's launches were timed one by one
    cw.cmbws_model_set_graphs(gm, False)
    x0, r0 = _solve(gm, b, tol=1e-10, maxiter=500, precond=1)
    assert np.array_equal(x0, x1)
