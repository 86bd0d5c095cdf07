"""Pins of oracle.precond (no GPU): U^+ U = I, M_PI = A^-1 when T = I, alpha and q minimisers."""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

from oracle import closed_form, model as om, precond
from oracle.cg import pcg
from tests._models import multires_small, oracle_model, tiny_workload


def test_alpha_is_least_squares_minimiser():
    rng = np.random.default_rng(1)
    tau = rng.uniform(0.2, 3.0, 500)
    w = rng.uniform(0.8, 1.2, 500) * 1e-3
    r = tau / w
    res = minimize_scalar(lambda s: np.sum((s * r - 1.0) ** 2), bracket=(1e-6, 1e-2))
    alpha_brute = 1.0 / np.sqrt(res.x)
    assert abs(precond.optimal_alpha(tau, w) - alpha_brute) < 1e-6 * alpha_brute


def test_q_formula_minimises_relative_misfit():
    q = np.random.default_rng(2).uniform(1.0, 3.0, 400)
    res = minimize_scalar(lambda s: np.sum((s * q - 1.0) ** 2), bracket=(0.1, 1.0))
    assert abs(precond.optimal_q(q) - 1.0 / res.x) < 1e-6
    assert abs(precond.optimal_q(np.full(10, 2.5)) - 2.5) < 1e-15


def test_pinv_is_left_inverse():
    m, _ = oracle_model(multires_small(64))
    U = precond.U_blocks(m)
    Up = precond.pinv_blocks(U)
    for l in range(U.shape[0]):
        act = [k for k in range(m.ncomp) if l <= m.lmax_comp[k]]
        P = Up[l] @ U[l]
        np.testing.assert_allclose(P[np.ix_(act, act)], np.eye(len(act)), atol=1e-10)
        absent = [k for k in range(m.ncomp) if k not in act]
        assert np.all(Up[l][absent] == 0.0)


def test_flat_case_precond_is_exact_inverse():
    work = tiny_workload(15)
    m, _ = oracle_model(work, flat=True)
    sig = [b.sigma for b in work.bands]
    r = np.random.default_rng(3).standard_normal(m.nvec())
    z = precond.apply_precond(m, r)
    ref = closed_form.solve(m.lmax_comp, m.lmax_band, m.beam, m.cl, m.q, sig, r)
    np.testing.assert_allclose(z, ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())
    assert np.allclose(precond.alphas(m), 1.0 / np.array(sig), rtol=1e-13)
    # PCG with M_PI converges in one iteration (M_PI A = I)
    x, info = pcg(lambda v: om.apply_A(m, v), r, lambda v: precond.apply_precond(m, v), tol=1e-10)
    assert info["iters"] == 1


def test_precond_symmetric_positive():
    m, _ = oracle_model(multires_small(64))
    rng = np.random.default_rng(4)
    x, y = rng.standard_normal((2, m.nvec()))
    a = x @ precond.apply_precond(m, y)
    b = y @ precond.apply_precond(m, x)
    assert abs(a - b) <= 1e-10 * abs(a)
    assert x @ precond.apply_precond(m, x) > 0


def test_square_U_case_clusters_near_identity():
    # Sec. 3.3: Ncomp = Nobs, no prior, matched band-limits -> M_PI A ~ I
    import skygen
    work = skygen.tiny_plain()
    work.bands = work.bands[:2]
    for b in work.bands:
        b.grid, b.n, b.lmax, b.contrast, b.fwhm = "healpix", 4, 11, 2.0, 200.0
    for c in work.comps:
        c.lmax, c.cl_kind = 11, None
    work.comps[1].beta = 3.0
    m, _ = oracle_model(work)
    n = m.nvec()
    A = om.dense_A(m)
    MA = np.stack([precond.apply_precond(m, A[:, j]) for j in range(n)], axis=1)
    ev = np.linalg.eigvals(MA).real
    assert np.median(np.abs(ev - 1.0)) < 0.2
