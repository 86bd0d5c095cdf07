"""Pins of the mask-restricted multigrid preconditioner of the oracle (oracle/maskmg.py)."""
import numpy as np
import pytest

import skygen
from oracle import alm as oalm
from oracle import cg as ocg
from oracle import grids as og
from oracle import maskmg as mg
from oracle import model as omodel
from oracle import precond as oprec
from oracle import sht as osht


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 16, 32])
def test_ang2pix_returns_every_pixel_centre(nside):
    g = og.healpix(nside)
    th, ph = g.pixel_angles()
    np.testing.assert_array_equal(mg.ang2pix_ring(nside, th, ph), np.arange(g.npix))


@pytest.mark.parametrize("nside", [2, 4, 8, 16, 32])
def test_every_coarse_pixel_has_four_nearby_children(nside):
    par = mg.coarse_parent(nside)
    assert np.all(np.bincount(par, minlength=12 * (nside // 2) ** 2) == 4)
    # children lie within one coarse pixel size of their parent's centre
    g, gc = og.healpix(nside), og.healpix(nside // 2)
    th, ph = g.pixel_angles()
    tc, pc = gc.pixel_angles()
    v = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    vc = np.stack([np.sin(tc) * np.cos(pc), np.sin(tc) * np.sin(pc), np.cos(tc)], 1)
    ang = np.arccos(np.clip(np.sum(v * vc[par], 1), -1, 1))
    assert ang.max() < 1.5 * np.sqrt(4 * np.pi / gc.npix)


def _band_mask(nside, zcut=0.35):
    g = og.healpix(nside)
    th, _ = g.pixel_angles()
    return np.abs(np.cos(th)) < zcut


def _cinv(L):
    c = skygen.cl_shape("cmb", L) * 1e3
    return 1.0 / c


def test_bottom_is_a_pseudo_inverse_of_the_dense_G():
    nside, L = 4, 11
    lv = mg.build_levels(nside, L, _band_mask(nside), _cinv(L), max_bottom=10 ** 6)
    assert len(lv) == 1
    b = lv[0]
    Y = osht.dense_Y(b.grid, L)[b.idx]
    G = (Y * b.d[oalm.ell_of_index(L)][None, :]) @ Y.T
    # eigenvalues kept down to 1e-5 of the largest: G G^+ G = G up to the dropped part
    ev = np.linalg.eigvalsh(G)
    dropped = ev[ev <= 1e-5 * ev.max()]
    bound = (np.abs(dropped).max() if dropped.size else 0.0) + 1e-10 * np.abs(G).max()
    assert np.abs(G @ b.Gp @ G - G).max() <= 1.01 * bound
    # the operator form of G agrees with the dense matrix
    x = np.zeros(b.grid.npix)
    x[b.idx] = np.random.default_rng(0).standard_normal(b.idx.size)
    np.testing.assert_allclose(b.G(x)[b.idx], G @ x[b.idx], atol=1e-10 * np.abs(G).max())


def test_vcycle_is_symmetric_and_accelerates_cg():
    nside, L = 16, 47
    mask = _band_mask(nside)
    lv = mg.build_levels(nside, L, mask, _cinv(L), max_bottom=60)
    assert len(lv) >= 3
    h = lv[0]
    idx = np.where(h.mask)[0]
    rng = np.random.default_rng(1)

    def rand():
        v = np.zeros(h.grid.npix)
        v[idx] = rng.standard_normal(idx.size)
        return v

    # the V-cycle is a symmetric operator: u . V v = v . V u
    for _ in range(3):
        u, v = rand(), rand()
        a, b = u @ mg.vcycle(lv, v), v @ mg.vcycle(lv, u)
        assert abs(a - b) <= 1e-10 * max(abs(a), abs(b))
    # the coarse-grid correction removes large-scale error: for smooth fields (l <= 8) one
    # V-cycle leaves < 20 % error, against the same two smoothing sweeps without it
    a = rng.standard_normal((L + 1) ** 2) * (oalm.ell_of_index(L) <= 8)
    x = np.where(h.mask, osht.synthesis(h.grid, L, a), 0.0)
    b = h.G(x)
    e_mg = np.linalg.norm(x - mg.vcycle(lv, b)) / np.linalg.norm(x)
    y = h.smooth * b
    y = y + h.smooth * np.where(h.mask, b - h.G(y), 0.0)
    e_sm = np.linalg.norm(x - y) / np.linalg.norm(x)
    assert e_mg < 0.2 and e_mg < 0.5 * e_sm, (e_mg, e_sm)


def _masked_model(nside=8, L=23, zcut=0.35):
    w = skygen.tiny_plain()
    w.comps = w.comps[:1]                            # CMB only, as in the paper's masked benchmark
    gs = [og.healpix(nside) for _ in w.bands]
    for b in w.bands:
        b.grid, b.n, b.lmax = "healpix", nside, L
    w.comps[0].lmax = L
    coords = [(np.cos(g.pixel_angles()[0]), g.pixel_angles()[1]) for g in gs]
    inp = skygen.make_inputs(w, coords, [g.pixel_weights() for g in gs])
    mask = _band_mask(nside, zcut)
    mgrid = og.healpix(nside)
    mmaps = [[np.where(mask, 0.0, 1.0) * inp["q"][nu, 0]] for nu in range(3)]
    m = omodel.Model(lmax_comp=[L], grids=gs, lmax_band=[L] * 3, beam=inp["beams"], cl=inp["cl"],
                     tau=inp["tau"], q=inp["q"], mix_grid=[[mgrid]] * 3, mix_map=mmaps)
    return m, inp, mask


def test_mask_precond_with_exact_inner_inverse_is_eq_M_mask():
    m, inp, mask = _masked_model(nside=4, L=11)
    mp = mg.MaskPrecond(m, 0, 4, mask, max_bottom=10 ** 6)
    h = mp.levels[0]
    assert h.Gp is not None
    Y = osht.dense_Y(h.grid, mp.L0)[h.idx]
    Z = Y * mp.r0[oalm.ell_of_index(mp.L0)][None, :]
    Sinv = omodel.prior_inv_diag(m)
    M = Z.T @ np.linalg.pinv(Z @ np.diag(Sinv) @ Z.T, rcond=1e-5) @ Z
    rng = np.random.default_rng(2)
    r = rng.standard_normal(m.nvec())
    # both sides are pseudo-inverses of G with the same cut-off (1e-5 of the largest
    # eigen- / singular value), so they agree to eps x 1e5; a wrong factor would be O(1)
    np.testing.assert_allclose(mp.apply(m, r), M @ r, rtol=1e-8, atol=1e-8 * np.abs(M @ r).max())


def test_M_add_speeds_up_the_masked_solve():
    m, inp, mask = _masked_model()
    mp = mg.MaskPrecond(m, 0, 8, mask, max_bottom=60)
    x_true = inp["x_true"]
    b = omodel.apply_A(m, x_true)
    Up = oprec.pinv_blocks(oprec.U_blocks(m))
    _, rep_pi = ocg.pcg(lambda v: omodel.apply_A(m, v), b,
                        apply_M=lambda v: oprec.apply_precond(m, v, Up), tol=1e-6, maxiter=3000)
    x, rep_add = ocg.pcg(lambda v: omodel.apply_A(m, v), b,
                         apply_M=lambda v: mg.apply_M_add(m, [mp], v, Up), tol=1e-6, maxiter=3000)
    assert rep_add["iters"] * 2 < rep_pi["iters"], (rep_add["iters"], rep_pi["iters"])
    assert np.linalg.norm(x - x_true) < 1e-4 * np.linalg.norm(x_true)


def test_optimized_vcycle_with_exact_J_is_the_basic_vcycle():
    """The reorganisation of Fig. code:mg is exact when J = Y^T W P Y is kept."""
    nside, L = 16, 47
    mask = _band_mask(nside)
    lv = mg.build_levels(nside, L, mask, _cinv(L), max_bottom=60)
    assert len(lv) >= 3
    rng = np.random.default_rng(3)
    idx = np.where(lv[0].mask)[0]
    for _ in range(2):
        b = np.zeros(lv[0].grid.npix)
        b[idx] = rng.standard_normal(idx.size)
        xb = mg.vcycle(lv, b)
        xo = mg.vcycle_optimized(lv, b, exact_J=True)
        assert np.abs(xo - xb).max() <= 1e-11 * np.abs(xb).max()
        # J ~ I changes the operator (the mask is not the full sky) ...
        xj = mg.vcycle_optimized(lv, b)
        assert np.abs(xj - xb).max() > 1e-8 * np.abs(xb).max()


def test_optimized_vcycle_is_symmetric_and_reduces_large_scale_error():
    """With J ~ I the restriction and interpolation of the optimized cycle are still each
    other's transposes, so the cycle is symmetric; it still removes large-scale error."""
    nside, L = 16, 47
    mask = _band_mask(nside)
    lv = mg.build_levels(nside, L, mask, _cinv(L), max_bottom=60)
    h = lv[0]
    idx = np.where(h.mask)[0]
    rng = np.random.default_rng(4)
    for _ in range(3):
        u, v = np.zeros(h.grid.npix), np.zeros(h.grid.npix)
        u[idx], v[idx] = rng.standard_normal(idx.size), rng.standard_normal(idx.size)
        a, b = u @ mg.vcycle_optimized(lv, v), v @ mg.vcycle_optimized(lv, u)
        assert abs(a - b) <= 1e-10 * max(abs(a), abs(b))
    a = rng.standard_normal((L + 1) ** 2) * (oalm.ell_of_index(L) <= 8)
    x = np.where(h.mask, osht.synthesis(h.grid, L, a), 0.0)
    b = h.G(x)
    e_opt = np.linalg.norm(x - mg.vcycle_optimized(lv, b)) / np.linalg.norm(x)
    y = h.smooth * b
    y = y + h.smooth * np.where(h.mask, b - h.G(y), 0.0)
    e_sm = np.linalg.norm(x - y) / np.linalg.norm(x)
    # measured: 0.22-0.26 left (basic cycle 0.14, smoothing alone 0.55)
    assert e_opt < 0.5 * e_sm, (e_opt, e_sm)


def test_M_add_with_optimized_vcycle_converges_like_basic():
    """The paper neglects J (Sec. 4.4: 6 SHTs per level); the masked solve still needs about
    the iterations of the basic cycle."""
    m, inp, mask = _masked_model()
    Up = oprec.pinv_blocks(oprec.U_blocks(m))
    b = omodel.apply_A(m, inp["x_true"])
    its = {}
    for cyc in ("basic", "optimized"):
        mp = mg.MaskPrecond(m, 0, 8, mask, max_bottom=60, cycle=cyc)
        x, rep = ocg.pcg(lambda v: omodel.apply_A(m, v), b,
                         apply_M=lambda v: mg.apply_M_add(m, [mp], v, Up), tol=1e-6, maxiter=3000)
        assert np.linalg.norm(x - inp["x_true"]) < 1e-4 * np.linalg.norm(inp["x_true"])
        its[cyc] = rep["iters"]
    assert its["optimized"] <= 1.5 * its["basic"] + 2, its


def _unit_vectors(g):
    th, ph = g.pixel_angles()
    return np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)


@pytest.mark.parametrize("nside", [2, 4, 8, 16, 32])
def test_coarse_mask_keeps_a_pixel_only_when_its_four_children_are_masked(nside):
    """Sec. 4.4: a coarse pixel belongs to the coarse mask only if it is 100 % masked.

    Brute force, independent of ang2pix: the centre of a coarse pixel is the vertex its four
    children share (the subdivision halves the pixel along both face directions), so the
    children are the four fine pixels whose centres lie nearest to it; the fifth nearest
    lies clearly farther out.  A coarse pixel is kept exactly when all four are masked."""
    from scipy.spatial import cKDTree
    f, c = og.healpix(nside), og.healpix(nside // 2)
    dist, near = cKDTree(_unit_vectors(f)).query(_unit_vectors(c), k=5)
    assert np.all(dist[:, 4] > 1.01 * dist[:, 3])
    children = near[:, :4]
    # the oracle's parent map agrees with the brute-force children
    par = mg.coarse_parent(nside)
    np.testing.assert_array_equal(par[children], np.repeat(np.arange(c.npix)[:, None], 4, 1))
    rng = np.random.default_rng(nside)
    kept = dropped = 0
    for frac in (0.3, 0.7, 0.95):
        mask = rng.uniform(size=f.npix) < frac
        mask |= _band_mask(nside, 0.2)            # whole masked blocks as well as random pixels
        want = mask[children].all(axis=1)
        got = mg.coarse_mask(nside, mask)
        np.testing.assert_array_equal(got, want)
        kept += int(want.sum())
        dropped += int((~want & mask[children].any(axis=1)).sum())
    assert kept > 0 and dropped > 0               # both outcomes occur


@pytest.mark.parametrize("L", [2, 7, 40, 191, 1535])
def test_rl_filter_matches_eq_rl(L):
    """Eq. rl: r_l = exp(-beta l^2 (l+1)^2), beta fixed by r^2 = 0.05 at l = L/2.

    beta is recovered from one value, r at lr = ceil(L/2) (where r is well below 1, so its
    logarithm is well conditioned); every other r_l must follow the l^2 (l+1)^2 shape with
    that beta, and the squared filter at L/2 (an integer or a half-integer l) must equal 0.05."""
    r = mg.rl_filter(L, 2 * L)
    assert r[0] == 1.0 and np.all(np.diff(r) < 0)
    lr = max(1, (L + 1) // 2)
    beta = -np.log(r[lr]) / (lr * lr * (lr + 1.0) ** 2)
    l = np.arange(2 * L + 1, dtype=np.float64)
    np.testing.assert_allclose(np.log(r[1:]), -beta * (l * l * (l + 1) ** 2)[1:], rtol=1e-10,
                               atol=1e-15)
    h = 0.5 * L
    assert abs(np.exp(-2.0 * beta * h * h * (h + 1) ** 2) - 0.05) < 1e-13
    if L % 2 == 0:
        assert abs(r[L // 2] ** 2 - 0.05) < 1e-13
