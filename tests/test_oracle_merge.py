"""Pins of oracle.merge: observation merging in the preconditioner (App. A.3)."""
import numpy as np
import pytest

from oracle import cg as ocg
from oracle import merge as omerge
from oracle import model as omodel
from oracle import precond as opc
from tests._models import multires_small, oracle_model, split_model, tiny_workload


def test_exact_split_preserves_UtU_and_M_PI():
    """Detector splits with unequal hit fractions (gamma != 1): U'^T U' = U^T U per l (the
    identity of App. A.3), and the merged preconditioner equals M_PI of the split model."""
    m0, _ = oracle_model(tiny_workload(15))
    m, groups = split_model(m0, (0.3, 0.7))
    U = opc.U_blocks(m)
    Um = omerge.merged_U_blocks(m, groups)
    assert Um.shape[1] == len(groups) + m.ncomp
    for l in range(U.shape[0]):
        np.testing.assert_allclose(Um[l].T @ Um[l], U[l].T @ U[l], rtol=1e-12,
                                   atol=1e-12 * np.abs(U[l].T @ U[l]).max())
    r = np.random.default_rng(2).standard_normal(m.nvec())
    z = omerge.apply_merged_precond(m, groups, r)
    zr = opc.apply_precond(m, r)
    assert np.abs(z - zr).max() < 1e-10 * np.abs(zr).max()
    # and the merged model needs one SHT pair per group, i.e. M_PI of the unsplit channel
    np.testing.assert_allclose(z, opc.apply_precond(m0, r), rtol=0,
                               atol=1e-10 * np.abs(zr).max())


def test_exact_split_multires_healpix():
    m0, _ = oracle_model(multires_small(64))
    m, groups = split_model(m0, (0.25, 0.25, 0.5))
    r = np.random.default_rng(3).standard_normal(m.nvec())
    z = omerge.apply_merged_precond(m, groups, r)
    zr = opc.apply_precond(m, r)
    assert np.abs(z - zr).max() < 1e-10 * np.abs(zr).max()


def test_flat_split_merged_is_A_inverse():
    """Flat inverse noise per unit area on GL grids: M_PI = A^-1 (Sec. 3.3); the merged
    preconditioner of a split model too, so PCG converges in one iteration."""
    m0, _ = oracle_model(tiny_workload(11), flat=True)
    m, groups = split_model(m0, (0.4, 0.6))
    b = np.random.default_rng(4).standard_normal(m.nvec())
    x = np.linalg.solve(omodel.dense_A(m), b)
    z = omerge.apply_merged_precond(m, groups, b)
    assert np.abs(z - x).max() < 1e-9 * np.abs(x).max()
    _, res = ocg.pcg(lambda v: omodel.apply_A(m, v), b,
                     lambda v: omerge.apply_merged_precond(m, groups, v), tol=1e-8)
    assert res["iters"] <= 2


def test_rank_one_row_is_leading_singular_pair():
    rng = np.random.default_rng(5)
    for shape in ((2, 3), (4, 3), (3, 1), (5, 8)):
        R = rng.standard_normal(shape)
        u = omerge.rank_one_row(R)
        _, s, Vt = np.linalg.svd(R)
        np.testing.assert_allclose(np.abs(u), s[0] * np.abs(Vt[0]), rtol=1e-12, atol=1e-14)
        # Eckart-Young: no other rank-one fit of R^T R is closer (random trials)
        S = R.T @ R
        best = np.linalg.norm(S - np.outer(u, u))
        for _ in range(50):
            v = u + 0.05 * rng.standard_normal(u.size) * np.abs(u).max()
            assert np.linalg.norm(S - np.outer(v, v)) >= best - 1e-12
    # proportional rows: the exact merge sqrt(1 + gamma^2) U_1
    u1 = np.array([0.3, -1.2, 0.5])
    np.testing.assert_allclose(omerge.rank_one_row(np.stack([u1, 2.5 * u1])),
                               -np.sqrt(1 + 2.5 ** 2) * u1, rtol=1e-14)


def test_printed_merge_factor_breaks_the_identity():
    """The printed (gamma + 1)^1/2 U_1 misses U_1^T U_1 + U_2^T U_2 unless gamma is 0 or 1."""
    u1 = np.array([0.3, -1.2, 0.5])
    for gamma in (0.5, 2.5):
        target = np.outer(u1, u1) * (1 + gamma ** 2)
        printed = np.sqrt(gamma + 1) * u1
        assert np.abs(np.outer(printed, printed) - target).max() > 0.1 * np.abs(target).max()
        derived = omerge.rank_one_row(np.stack([u1, gamma * u1]))
        np.testing.assert_allclose(np.outer(derived, derived), target, rtol=1e-13)


def test_compromise_merge_is_a_valid_preconditioner():
    """Bands that are only similar (different beams, mixing and noise patterns) merged in
    the preconditioner alone: M stays symmetric positive definite and PCG converges."""
    m0, inp = oracle_model(tiny_workload(15))
    m, groups = split_model(m0, (0.5, 0.5))
    rng = np.random.default_rng(6)
    th, _ = m.grids[1].pixel_angles()
    m.tau[1] = m.tau[1] * (1.0 + 0.3 * np.cos(th))
    m.beam[1] = m.beam[1] ** 1.2
    q = np.array(m.q, dtype=np.float64)
    q[1] *= np.array([1.0, 1.15])
    m.q = q
    n = m.nvec()
    M = np.stack([omerge.apply_merged_precond(m, groups, e) for e in np.eye(n)], axis=1)
    assert np.abs(M - M.T).max() < 1e-10 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0
    b = omodel.apply_A(m, rng.standard_normal(n))
    _, r_m = ocg.pcg(lambda v: omodel.apply_A(m, v), b,
                     lambda v: omerge.apply_merged_precond(m, groups, v), tol=1e-8, maxiter=500)
    _, r_u = ocg.pcg(lambda v: omodel.apply_A(m, v), b, lambda v: opc.apply_precond(m, v),
                     tol=1e-8, maxiter=500)
    assert r_m["rel_res"][-1] <= 1e-8 and r_u["rel_res"][-1] <= 1e-8
    assert r_m["iters"] <= 2 * r_u["iters"] + 5, (r_m["iters"], r_u["iters"])


def test_groups_validated():
    m0, _ = oracle_model(tiny_workload(7))
    m, groups = split_model(m0)
    with pytest.raises(ValueError):
        omerge.merged_U_blocks(m, [[0, 1], [2, 3]])          # not a partition
    with pytest.raises(ValueError):
        omerge.merged_U_blocks(m, [[0, 2], [1, 3], [4, 5]])  # bands on different grids
