"""Pins of oracle.sampling: the generator against numpy's Philox4x64-10, the normals against
their distribution, and the CR draws against the posterior they must sample (Sec. 2.3)."""
import numpy as np
import pytest
from scipy import stats

from oracle import model as omodel
from oracle import sampling as osamp
from tests._models import oracle_model, tiny_workload

_M64 = (1 << 64) - 1


def _numpy_block(ctr, key, t=0):
    """Block t of numpy's Philox started at `ctr`; numpy advances the counter before each
    block, so block t is the generator at counter ctr + t + 1."""
    g = np.random.Philox(key=np.array([int(k) for k in key], dtype=np.uint64),
                         counter=np.array([int(c) for c in ctr], dtype=np.uint64))
    return [int(v) for v in g.random_raw(4 * (t + 1))[4 * t:]]


def _add(ctr, n):
    v = sum(int(c) << (64 * i) for i, c in enumerate(ctr)) + n
    return [(v >> (64 * i)) & _M64 for i in range(4)]


@pytest.mark.parametrize("ctr,key", [
    ([0, 0, 0, 0], [0, 0]),
    ([0, 0, 0, 0], [1, 2]),
    ([_M64, 5, 0, 0], [0xDEADBEEF, 0x12345678]),           # carry into the second word
    ([123456789, 987654321, 5555, 77], [_M64, _M64]),
    ([_M64, _M64, _M64, _M64 - 1], [0x243F6A8885A308D3, 0x13198A2E03707344]),
])
def test_philox_matches_numpy(ctr, key):
    for t in range(3):
        assert list(osamp.philox4x64_int(_add(ctr, t + 1), key)) == _numpy_block(ctr, key, t)


def test_vectorised_philox_matches_integer_form():
    rng = np.random.default_rng(11)
    c = rng.integers(0, 2 ** 63, size=(64, 4), dtype=np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, size=(64, 4), dtype=np.uint64)
    for key in ([0, 0], [3, 9], [_M64, 1 << 63]):
        got = np.stack(osamp.philox4x64(c[:, 0], c[:, 1], c[:, 2], c[:, 3], *key), axis=1)
        for i in range(c.shape[0]):
            assert [int(v) for v in got[i]] == list(osamp.philox4x64_int(c[i], key))


def test_variate_indexing_is_offset_invariant():
    full = osamp.words(5, 3, 2, 0, 103)
    for off, n in ((0, 1), (1, 7), (3, 1), (4, 4), (5, 98), (101, 2), (17, 0)):
        assert np.array_equal(osamp.words(5, 3, 2, off, n), full[off:off + n])
        np.testing.assert_array_equal(osamp.normals(5, 3, 2, off, n),
                                      osamp.normals(5, 3, 2, 0, 103)[off:off + n])
    # variate 4 i + t is word t of counter (i, stream, 0, 0) under key (seed, sample)
    assert int(full[9]) == osamp.philox4x64_int([2, 2, 0, 0], [5, 3])[1]
    # distinct streams, samples and seeds give distinct words
    assert not np.array_equal(full[:8], osamp.words(5, 3, 1, 0, 8))
    assert not np.array_equal(full[:8], osamp.words(5, 4, 2, 0, 8))
    assert not np.array_equal(full[:8], osamp.words(6, 3, 2, 0, 8))


def test_uniforms_exact_and_inside_open_interval():
    w = osamp.words(1, 1, 0, 0, 1000)
    u = osamp.uniforms(1, 1, 0, 0, 1000)
    # u = (k + 1/2) / 2^52 with k the top 52 bits of the word, exactly
    from fractions import Fraction
    k = [int(v) >> 12 for v in w]
    assert all(Fraction(float(ui)) == Fraction(2 * ki + 1, 2 ** 53) for ui, ki in zip(u, k))
    assert u.min() > 0.0 and u.max() < 1.0
    # the extreme words stay inside (0, 1)
    for wx in (0, _M64):
        ux = ((np.uint64(wx) >> np.uint64(12)).astype(np.float64) + 0.5) * 2.0 ** -52
        assert 0.0 < ux < 1.0 and Fraction(float(ux)) == Fraction(2 * (wx >> 12) + 1, 2 ** 53)


def test_uniform_and_normal_distributions():
    n = 400_000
    u = osamp.uniforms(2017, 0, 0, 0, n)
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    z = osamp.normals(2017, 0, 1, 0, n)
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert abs(np.mean(z ** 4) - 3.0) < 5 * np.sqrt(96.0 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # the two normals of a pair, and neighbouring pairs, are uncorrelated
    zz = z.reshape(-1, 2)
    assert abs(np.corrcoef(zz[:, 0], zz[:, 1])[0, 1]) < 5 / np.sqrt(n / 2)
    q = z.reshape(-1, 4)
    assert abs(np.corrcoef(q[:, 1], q[:, 2])[0, 1]) < 5 / np.sqrt(n / 4)


def _whitened_draws(rhs_of_sample, N, L=3):
    m, inp = oracle_model(tiny_workload(L))
    d = [a + b for a, b in zip(omodel.project(m, inp["x_true"]), inp["noise"])]
    A = omodel.dense_A(m)
    Lc = np.linalg.cholesky(A)
    mu = np.linalg.solve(A, omodel.rhs(m, d))
    Y = np.empty((N, m.nvec()))
    for s in range(N):
        Y[s] = Lc.T @ (np.linalg.solve(A, rhs_of_sample(m, d, s)) - mu)
    return Y


def _is_standard_normal(Y):
    N, n = Y.shape
    C = Y.T @ Y / N
    ev = np.linalg.eigvalsh(C)
    edge = 2 * np.sqrt(n / N) + 5 / np.sqrt(N)   # Marchenko-Pastur edge plus margin
    return (np.abs(Y.mean(axis=0)).max() < 5 / np.sqrt(N) and ev.min() > 1 - edge
            and ev.max() < 1 + edge and abs(np.trace(C) / n - 1) < 5 * np.sqrt(2.0 / (N * n)))


def test_cr_draws_sample_the_posterior():
    """x = A^-1 b over many draws: mean A^-1 P^T N^-1 d and covariance A^-1 (Sec. 2.3).
    Whitened by A = L L^T, y = L^T (x - mu) must be N(0, I)."""
    Y = _whitened_draws(lambda m, d, s: osamp.cr_rhs(m, d, 1710, s), 4000)
    assert _is_standard_normal(Y)


def test_posterior_pin_rejects_planted_mistakes():
    """The same check fails for the printed S^-1 omega_2 and for a dropped N^-1/2 omega_1."""
    def printed(m, d, s):
        w1, w2 = osamp.cr_omegas(m, 1710, s)
        return omodel.rhs(m, d, w1, None) + omodel.prior_inv_diag(m, 1.0) * w2

    def no_w1(m, d, s):
        _, w2 = osamp.cr_omegas(m, 1710, s)
        return omodel.rhs(m, d, None, w2)

    assert not _is_standard_normal(_whitened_draws(printed, 1000))
    assert not _is_standard_normal(_whitened_draws(no_w1, 1000))


def test_cr_draws_reproducible_and_distinct():
    m, inp = oracle_model(tiny_workload(3))
    d = omodel.project(m, inp["x_true"])
    b0 = osamp.cr_rhs(m, d, 7, 0)
    assert np.array_equal(b0, osamp.cr_rhs(m, d, 7, 0))
    assert not np.allclose(b0, osamp.cr_rhs(m, d, 7, 1))
    w1, w2 = osamp.cr_omegas(m, 7, 0)
    assert [w.size for w in w1] == [t.size for t in m.tau] and w2.size == m.nvec()
    np.testing.assert_array_equal(w1[1], osamp.normals(7, 0, 2, 0, m.tau[1].size))


def test_powerlaw_mixing():
    beta = np.array([-3.0, 0.0, 1.0, 1.6, 2.5])
    np.testing.assert_allclose(osamp.powerlaw_mixing(2.0, beta), [0.125, 1.0, 2.0, 2 ** 1.6,
                                                                  2 ** 2.5], rtol=1e-15)
    mask = np.array([1, 0, 1, 1, 0.0])
    np.testing.assert_array_equal(osamp.powerlaw_mixing(0.3, beta, mask)[[1, 4]], 0.0)
    # log q is linear in beta with slope ln(nu / nu_0)
    q = osamp.powerlaw_mixing(353.0 / 30.0, beta)
    np.testing.assert_allclose(np.diff(np.log(q)) / np.diff(beta), np.log(353.0 / 30.0),
                               rtol=1e-13)
