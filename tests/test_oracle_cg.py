"""Pins of oracle.cg (no GPU): dense Cholesky solve and the closed-form Wiener filter."""
import numpy as np

from oracle import closed_form, model as om, precond
from oracle.cg import pcg
from tests._models import multires_small, oracle_model, tiny_workload


def test_pcg_matches_cholesky():
    m, inp = oracle_model(multires_small(64))
    A = om.dense_A(m)
    b = A @ inp["x_true"]
    x, info = pcg(lambda v: om.apply_A(m, v), b, lambda v: precond.apply_precond(m, v),
                  tol=1e-12, maxiter=500, x_true=inp["x_true"])
    ref = np.linalg.solve(A, b)
    np.testing.assert_allclose(x, ref, atol=1e-9 * np.abs(ref).max())
    # the PI preconditioner beats plain CG on this problem
    _, info0 = pcg(lambda v: om.apply_A(m, v), b, None, tol=1e-8, maxiter=2000)
    _, info1 = pcg(lambda v: om.apply_A(m, v), b, lambda v: precond.apply_precond(m, v), tol=1e-8)
    assert info1["iters"] < info0["iters"]


def test_wiener_solution_closed_form():
    work = tiny_workload(15)
    m, inp = oracle_model(work, flat=True)
    d = [mp + n for mp, n in zip(om.project(m, inp["x_true"]), inp["noise"])]
    b = om.rhs(m, d)
    sig = [bd.sigma for bd in work.bands]
    ref = closed_form.solve(m.lmax_comp, m.lmax_band, m.beam, m.cl, m.q, sig, b)
    x, _ = pcg(lambda v: om.apply_A(m, v), b, None, tol=1e-13, maxiter=3000)
    np.testing.assert_allclose(x, ref, atol=1e-8 * np.abs(ref).max())
