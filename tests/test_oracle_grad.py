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


# ---- spatially variable mixing (Eq. Q): derivatives in the mixing-map pixels ----

def _setup_var(L=5, Lmix=6, cr=False, const=False):
    """The differentiable workload with the dust pairs of every band on variable mixing maps
    (a smooth pattern around the scalar value, or the scalar value itself if const) on a
    Gauss-Legendre mixing grid."""
    from oracle import grids as og
    w, m0, d, o1, o2, wgt = _setup(L, cr)
    g = og.gauss_legendre(Lmix)
    th, ph = g.pixel_angles()
    k = 2
    maps = [[None] * m0.ncomp for _ in range(m0.nobs)]
    grids = [[None] * m0.ncomp for _ in range(m0.nobs)]
    for nu in range(m0.nobs):
        pat = 0.0 if const else 0.4 * np.cos(th) + 0.2 * np.sin(th) * np.cos(ph + nu)
        maps[nu][k] = m0.q[nu, k] * (1.0 + pat)
        grids[nu][k] = g
    m = omodel.Model(**{**m0.__dict__, "mix_map": maps, "mix_grid": grids})
    return w, m, d, o1, o2, wgt


def _with_map(m, nu, k, p, dv):
    maps = [[None if q is None else q.copy() for q in row] for row in m.mix_map]
    maps[nu][k][p] += dv
    return omodel.Model(**{**m.__dict__, "mix_map": maps})


@pytest.mark.parametrize("cr", [False, True])
def test_mixing_map_gradient_matches_central_differences(cr):
    """dL/dq(p) of the dense Cholesky solve's loss against central differences in single
    pixels of the mixing maps (pole, equator, in between; two bands), and the offset entry of
    dq against a uniform shift of the whole map."""
    w, m, d, o1, o2, wgt = _setup_var(cr=cr)
    b = omodel.rhs(m, d, o1, o2)
    x = ograd.solve_dense(m, b)
    L0, g = ograd.weighted_loss(x, wgt)
    lam = ograd.solve_dense(m, g)
    maps = ograd.grad_mix_maps_dense(m, x, lam, d, o1)
    dq, _ = ograd.grad_terms_dense(m, x, lam, d, o1, o2)
    assert set(maps) == {(nu, 2) for nu in range(m.nobs)}
    npix = m.mix_map[0][2].size
    h = 1e-6
    for nu in (0, 3):
        gmap = maps[(nu, 2)]
        for p in (0, npix // 2, npix // 3 + 5, npix - 1):
            fd = (_loss(_with_map(m, nu, 2, p, h), d, o1, o2, wgt)
                  - _loss(_with_map(m, nu, 2, p, -h), d, o1, o2, wgt)) / (2 * h)
            scale = max(abs(fd), 1e-4 * np.abs(gmap).max())
            assert abs(fd - gmap[p]) <= 1e-5 * scale, (nu, p, fd, gmap[p])
        mp = omodel.Model(**{**m.__dict__, "mix_map": [[None if q is None else (q + h if j == nu else q)
                                                          for q in row] for j, row in enumerate(m.mix_map)]})
        mm = omodel.Model(**{**m.__dict__, "mix_map": [[None if q is None else (q - h if j == nu else q)
                                                          for q in row] for j, row in enumerate(m.mix_map)]})
        fd = (_loss(mp, d, o1, o2, wgt) - _loss(mm, d, o1, o2, wgt)) / (2 * h)
        assert abs(fd - dq[nu, 2]) <= 1e-5 * max(abs(fd), 1e-3 * L0), (nu, fd, dq[nu, 2])


@pytest.mark.parametrize("cr", [False, True])
def test_mixing_map_operator_form_equals_dense(cr):
    w, m, d, o1, o2, wgt = _setup_var(L=6, Lmix=8, cr=cr)
    rng = np.random.default_rng(12)
    x = rng.standard_normal(m.nvec())
    lam = rng.standard_normal(m.nvec())
    a = ograd.grad_mix_maps(m, x, lam, d, o1)
    b = ograd.grad_mix_maps_dense(m, x, lam, d, o1)
    for key in b:
        np.testing.assert_allclose(a[key], b[key], rtol=1e-10, atol=1e-10 * np.abs(b[key]).max())
    dq0, dt0 = ograd.grad_terms_dense(m, x, lam, d, o1, o2)
    dq1, dt1 = ograd.grad_terms(m, x, lam, d, o1, o2)
    np.testing.assert_allclose(dq1, dq0, rtol=1e-10, atol=1e-10 * np.abs(dq0).max())
    np.testing.assert_allclose(dt1, dt0, rtol=1e-10, atol=1e-10 * np.abs(dt0).max())


def test_constant_map_offset_derivative_equals_scalar_derivative():
    """A constant mixing map on a grid that integrates the products exactly (Gauss-Legendre,
    L_mix >= L) is the scalar mixing of the same value: the model's operators agree, and the
    offset derivative of the map is the scalar dq."""
    w, m, d, o1, o2, wgt = _setup_var(const=True)
    _, m0, _, _, _, _ = _setup(5)
    rng = np.random.default_rng(13)
    x = rng.standard_normal(m.nvec())
    lam = rng.standard_normal(m.nvec())
    np.testing.assert_allclose(omodel.apply_A(m, x), omodel.apply_A(m0, x), rtol=1e-11, atol=1e-11)
    dqv, dtv = ograd.grad_terms(m, x, lam, d)
    dqs, dts = ograd.grad_terms(m0, x, lam, d)
    np.testing.assert_allclose(dqv, dqs, rtol=1e-9, atol=1e-12 * np.abs(dqs).max())
    np.testing.assert_allclose(dtv, dts, rtol=1e-12)
