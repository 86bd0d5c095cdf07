"""Pins of oracle.model (no GPU): symmetry/PD of A, closed form, dense agreement, CR covariance."""
import numpy as np
import pytest

from oracle import closed_form, grids, model as om
from tests._models import multires_small, oracle_model, tiny_workload


@pytest.fixture(scope="module")
def small():
    return oracle_model(multires_small(64))


def test_A_symmetric_operator(small):
    m, _ = small
    rng = np.random.default_rng(3)
    x, y = rng.standard_normal((2, m.nvec()))
    a, b = x @ om.apply_A(m, y), y @ om.apply_A(m, x)
    assert abs(a - b) <= 1e-11 * abs(a)


def test_dense_A_matches_operator_and_is_spd(small):
    m, _ = small
    A = om.dense_A(m)
    np.testing.assert_allclose(A, A.T, atol=1e-10 * np.abs(A).max())
    np.linalg.cholesky(A)
    x = np.random.default_rng(4).standard_normal(m.nvec())
    np.testing.assert_allclose(om.apply_A(m, x), A @ x, rtol=1e-10, atol=1e-10 * np.abs(A @ x).max())


def test_flat_noise_matches_closed_form():
    work = tiny_workload(15)
    m, inp = oracle_model(work, flat=True)
    sig = [b.sigma for b in work.bands]
    x = np.random.default_rng(5).standard_normal(m.nvec())
    ref = closed_form.apply_A(m.lmax_comp, m.lmax_band, m.beam, m.cl, m.q, sig, x)
    np.testing.assert_allclose(om.apply_A(m, x), ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


def test_flat_noise_multires_gl_closed_form():
    # different band-limits per band and component, still GL and flat per unit area
    import skygen
    work = skygen.tiny_plain()
    for b, L in zip(work.bands, (9, 14, 20)):
        b.n = b.lmax = L
    work.comps[0].lmax, work.comps[1].lmax = 12, 18
    m, _ = oracle_model(work, flat=True)
    sig = [b.sigma for b in work.bands]
    x = np.random.default_rng(6).standard_normal(m.nvec())
    ref = closed_form.apply_A(m.lmax_comp, m.lmax_band, m.beam, m.cl, m.q, sig, x)
    np.testing.assert_allclose(om.apply_A(m, x), ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


def test_constant_mixing_map_equals_scalar_mixing():
    # Eq. Q with a constant map on a GL grid that resolves max(L_k, L_nu) is exactly q I
    work = tiny_workload(10)
    m, inp = oracle_model(work)
    mg = [[grids.gauss_legendre(10) for _ in range(m.ncomp)] for _ in range(m.nobs)]
    mm = [[np.full(mg[nu][k].npix, m.q[nu, k]) for k in range(m.ncomp)] for nu in range(m.nobs)]
    mv, _ = oracle_model(work, mix_maps=mm, mix_grids=mg)
    x = np.random.default_rng(8).standard_normal(m.nvec())
    np.testing.assert_allclose(om.apply_A(mv, x), om.apply_A(m, x), rtol=1e-11,
                               atol=1e-11 * np.abs(om.apply_A(m, x)).max())


def test_variable_mixing_A_symmetric():
    work = tiny_workload(8)
    m, _ = oracle_model(work)
    mg = [[grids.gauss_legendre(12) for _ in range(m.ncomp)] for _ in range(m.nobs)]
    rng = np.random.default_rng(9)
    mm = [[m.q[nu, k] * (1.0 + 0.5 * rng.random(mg[nu][k].npix)) for k in range(m.ncomp)]
          for nu in range(m.nobs)]
    mv, _ = oracle_model(work, mix_maps=mm, mix_grids=mg)
    A = om.dense_A(mv)
    np.testing.assert_allclose(A, A.T, atol=1e-11 * np.abs(A).max())
    np.linalg.cholesky(A)


def test_cr_rhs_covariance_equals_A():
    # with d = 0, b = P^T N^-1/2 w1 + S^-1/2 w2 is linear in (w1, w2) with Cov(b) = A
    work = tiny_workload(6)
    m, _ = oracle_model(work)
    npix = [g.npix for g in m.grids]
    cols = []
    zeros = [np.zeros(n) for n in npix]
    for nu in range(m.nobs):
        for i in range(npix[nu]):
            w1 = [z.copy() for z in zeros]
            w1[nu][i] = 1.0
            cols.append(om.rhs(m, zeros, omega1=w1))
    for j in range(m.nvec()):
        w2 = np.zeros(m.nvec())
        w2[j] = 1.0
        cols.append(om.rhs(m, zeros, omega1=None, omega2=w2))
    G = np.stack(cols, axis=1)
    A = om.dense_A(m)
    np.testing.assert_allclose(G @ G.T, A, atol=1e-10 * np.abs(A).max())
