"""Pins of the oracle's solution gradient (oracle/grad.py).

The gradient of L(x(theta)), A(theta) x = b(theta), is checked against central finite
differences of the loss of the dense Cholesky solve, which uses no derivative formula;
the operator form is checked against the dense one.
"""
import numpy as np
import pytest

import skygen
from oracle import grad as ograd
from oracle import model as omodel
from tests._models import oracle_model


def _tiny(L=5, contrast=3.0):
    w = skygen.differentiable(lmax=L)
    for b in w.bands:
        b.contrast = contrast
    return w


def _setup(L=5, cr=False):
    w = _tiny(L)
    m, inp = oracle_model(w)
    d = omodel.project(m, inp["x_true"])
    d = [dn + nn for dn, nn in zip(d, inp["noise"])]
    rng = np.random.default_rng(5)
    o1 = [rng.standard_normal(t.size) for t in m.tau] if cr else None
    o2 = rng.standard_normal(m.nvec()) if cr else None
    wgt = skygen.harmonic_weight(m.lmax_comp)
    return w, m, d, o1, o2, wgt


def _loss(m, d, o1, o2, wgt):
    b = omodel.rhs(m, d, o1, o2)
    x = ograd.solve_dense(m, b)
    return ograd.weighted_loss(x, wgt)[0]


def _with_q(m, q):
    m2 = omodel.Model(**{**m.__dict__})
    m2.q = q
    return m2


def _with_cl_scale(m, k, s):
    m2 = omodel.Model(**{**m.__dict__})
    m2.cl = [c if (j != k or c is None) else c * s for j, c in enumerate(m.cl)]
    return m2


@pytest.mark.parametrize("cr", [False, True])
def test_gradient_matches_central_differences(cr):
    w, m, d, o1, o2, wgt = _setup(cr=cr)
    b = omodel.rhs(m, d, o1, o2)
    x = ograd.solve_dense(m, b)
    L0, g = ograd.weighted_loss(x, wgt)
    lam = ograd.solve_dense(m, g)
    dq, dt = ograd.grad_terms_dense(m, x, lam, d, o1, o2)
    h = 1e-5
    for nu in range(m.nobs):
        for k in range(m.ncomp):
            qp, qm = m.q.copy(), m.q.copy()
            step = h * max(1.0, abs(m.q[nu, k]))
            qp[nu, k] += step
            qm[nu, k] -= step
            fd = (_loss(_with_q(m, qp), d, o1, o2, wgt) - _loss(_with_q(m, qm), d, o1, o2, wgt)) / (2 * step)
            assert abs(fd - dq[nu, k]) <= 1e-6 * max(abs(fd), 1e-3 * L0), (nu, k, fd, dq[nu, k])
    for k in range(m.ncomp):
        fd = (_loss(_with_cl_scale(m, k, np.exp(h)), d, o1, o2, wgt)
              - _loss(_with_cl_scale(m, k, np.exp(-h)), d, o1, o2, wgt)) / (2 * h)
        assert abs(fd - dt[k]) <= 1e-6 * max(abs(fd), 1e-3 * L0), (k, fd, dt[k])


@pytest.mark.parametrize("cr", [False, True])
def test_operator_form_equals_dense(cr):
    w, m, d, o1, o2, wgt = _setup(L=7, cr=cr)
    rng = np.random.default_rng(11)
    x = rng.standard_normal(m.nvec())
    lam = rng.standard_normal(m.nvec())
    dq0, dt0 = ograd.grad_terms_dense(m, x, lam, d, o1, o2)
    dq1, dt1 = ograd.grad_terms(m, x, lam, d, o1, o2)
    np.testing.assert_allclose(dq1, dq0, rtol=1e-10, atol=1e-10 * np.abs(dq0).max())
    np.testing.assert_allclose(dt1, dt0, rtol=1e-10, atol=1e-10 * np.abs(dt0).max())


def test_spectral_index_chain_rule():
    """dL/dbeta_k = sum_nu dL/dq_{nu,k} q_{nu,k} ln(nu / nu_0,k) against differences in beta."""
    w, m, d, o1, o2, wgt = _setup()
    b = omodel.rhs(m, d)
    x = ograd.solve_dense(m, b)
    _, g = ograd.weighted_loss(x, wgt)
    lam = ograd.solve_dense(m, g)
    dq, _ = ograd.grad_terms(m, x, lam, d)
    freqs = np.array([bd.freq for bd in w.bands])
    h = 1e-5
    for k, c in enumerate(w.comps):
        if c.beta is None:
            continue
        an = np.sum(dq[:, k] * m.q[:, k] * np.log(freqs / c.nu0))
        qs = []
        for s in (+1, -1):
            q = m.q.copy()
            q[:, k] = (freqs / c.nu0) ** (c.beta + s * h)
            qs.append(_loss(_with_q(m, q), d, None, None, wgt))
        fd = (qs[0] - qs[1]) / (2 * h)
        assert abs(fd - an) <= 1e-6 * abs(fd), (k, fd, an)
