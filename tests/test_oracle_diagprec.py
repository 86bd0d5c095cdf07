"""Pins of the block-diagonal comparison preconditioner of the oracle (oracle/diagprec.py)."""
import numpy as np
import pytest

import skygen
from oracle import cg as ocg
from oracle import diagprec as od
from oracle import grids as og
from oracle import model as omodel
from oracle import precond as oprec
from tests._models import oracle_model, tiny_workload


@pytest.mark.parametrize("grid,L", [("gl", 15), ("healpix", 23), ("healpix", 10)])
def test_ring_sum_diagonal_equals_the_definition(grid, L):
    g = og.gauss_legendre(L) if grid == "gl" else og.healpix(8)
    tau = np.random.default_rng(L).uniform(0.5, 2.0, g.npix)
    np.testing.assert_allclose(od.diag_YtNY(g, L, tau), od.diag_YtNY_dense(g, L, tau),
                               rtol=1e-11, atol=1e-12 * tau.sum())


def test_blocks_are_the_coefficientwise_blocks_of_A():
    w = tiny_workload(7)
    m, inp = oracle_model(w)
    A = omodel.dense_A(m)
    Binv = od.diag_blocks(m)
    o = m.comp_offsets()
    n = o[1] - o[0]
    for j in range(n):
        idx = [o[k] + j for k in range(m.ncomp)]
        np.testing.assert_allclose(Binv[j], np.linalg.inv(A[np.ix_(idx, idx)]), rtol=1e-10)
    r = np.random.default_rng(0).standard_normal(m.nvec())
    z = od.apply_M_diag(m, r, Binv)
    for j in range(n):
        idx = [o[k] + j for k in range(m.ncomp)]
        np.testing.assert_allclose(z[idx], Binv[j] @ r[idx], rtol=1e-12)


def test_pseudo_inverse_preconditioner_beats_the_diagonal_one():
    """The paper's comparison: on the multi-resolution model M_PI needs fewer iterations."""
    w = skygen.multires_fullsky(scale=32)
    m, inp = oracle_model(w)
    b = omodel.apply_A(m, inp["x_true"])
    Up = oprec.pinv_blocks(oprec.U_blocks(m))
    Binv = od.diag_blocks(m)
    _, r_pi = ocg.pcg(lambda v: omodel.apply_A(m, v), b,
                      apply_M=lambda v: oprec.apply_precond(m, v, Up), tol=1e-6, maxiter=2000)
    _, r_dg = ocg.pcg(lambda v: omodel.apply_A(m, v), b,
                      apply_M=lambda v: od.apply_M_diag(m, v, Binv), tol=1e-6, maxiter=2000)
    assert r_pi["iters"] < r_dg["iters"], (r_pi["iters"], r_dg["iters"])
