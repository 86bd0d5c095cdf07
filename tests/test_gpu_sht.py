"""GPU parity of the SHT stages (Legendre + ring FFT) against the oracle, through the C ABI."""
import numpy as np
import pytest

import paper_1710_00621_gb300 as cw
from oracle import grids as og, sht as osht
from tests._gpu import rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu

EPS64, EPS48, EPS32 = 2.0 ** -53, 2.0 ** -48, 2.0 ** -24
TC_PRECS = [cw.CMBWS_TF32, cw.CMBWS_3XTF32, cw.CMBWS_BF16, cw.CMBWS_BF16X3]


def tol(prec, lmax, op="synth"):
    """Parity bound relative to the largest output magnitude, for synthesis (op "synth") or
    adjoint synthesis / analysis (op "adj"); each is a few times the error measured on GB300
    over the cases below and the full-size Nside 1024, L = 3071 checks.

    FP64: the recurrence and the quadrature sums lose accuracy in proportion to L (measured
    ~10 (L+1) eps at L = 100 and L = 3071): 40 (L+1) eps64, floor 1e-14.
    FP32X2 (double-float, eps48 = 2^-48): synthesis 16 (L+1) eps48 (measured 3.6e-11 at
    L = 3071: 3.3 (L+1) eps48), the adjoint, which restarts from FP64-accurate checkpoints
    every 4 values of l, 2 (L+1) eps48; floor 1e-13.
    FP32: rounding errors of the recurrence and of the FP32 sums add up like a random walk,
    ~sqrt(L+1) eps32 (measured synthesis 2.3e-6 at L = 191, 1.3e-5 at L = 3071; the adjoint
    restarts every 8 values of l from checkpoints, 0.75e-6 and 1.9e-6): synthesis
    15 sqrt(L+1) eps32, adjoint 6 sqrt(L+1) eps32, floor 1e-6.
    TF32 (synthesis only): both factors rounded to 11 significant bits (relative 2^-11 each),
    so up to 2^-10 per term (measured up to 5.9e-4, for a single term at L = 0): 1.5e-3.
    BF16: 8 significant bits per factor (2^-9 each; measured 1.8e-3 to 5.0e-3): 1.5e-2.
    3XTF32: split TF32 drops only the lo x lo product (2^-22); the recurrence is the FP32 one
    and its accumulation order differs: twice the FP32 bound.  BF16X3: the split keeps about
    16 significant bits per factor (measured 4.4e-6 to 1.2e-5): twice the FP32 bound, at
    least 4e-5.  TF32 and 3XTF32 share the FP32 adjoint; the BF16 and BF16X3 adjoints run on
    the tensor cores (BF16 factors, the FP32 adjoint's checkpointed recurrence) and take the
    synthesis bounds of their mode.
    """
    if op == "adj" and prec in (cw.CMBWS_TF32, cw.CMBWS_3XTF32):
        prec = cw.CMBWS_FP32
    if op == "adj" and prec in (cw.CMBWS_BF16, cw.CMBWS_BF16X3):
        op = "synth"
    n = lmax + 1
    if prec == cw.CMBWS_FP64:
        return max(1e-14, 40 * n * EPS64)
    if prec == cw.CMBWS_FP32X2:
        return max(1e-13, (16 if op == "synth" else 2) * n * EPS48)
    if prec == cw.CMBWS_TF32:
        return 1.5e-3
    if prec == cw.CMBWS_BF16:
        return 1.5e-2
    f32 = max(1e-6, (15 if op == "synth" else 6) * np.sqrt(n) * EPS32)
    if prec == cw.CMBWS_BF16X3:
        return max(4e-5, 2 * f32)
    return 2 * f32 if prec == cw.CMBWS_3XTF32 else f32


# (kind, n, lmax): tiny, ragged, several CTAs of the Legendre kernels, folded spectra
CASES = [
    ("gl", 0, 0), ("gl", 1, 1), ("gl", 63, 63), ("gl", 100, 100), ("gl", 40, 31),
    ("hp", 1, 2), ("hp", 4, 11), ("hp", 8, 40), ("hp", 16, 47), ("hp", 64, 191),
]


def _grids(kind, n, lmax):
    if kind == "gl":
        return cw.cmbws_plan_grid(cw.CMBWS_GRID_GL, n + 1, lmax), og.gauss_legendre(n) if n >= lmax else None
    return cw.cmbws_plan_grid(cw.CMBWS_GRID_HEALPIX, n, lmax), og.healpix(n)


def _oracle_grid(kind, n, lmax, g):
    if kind == "gl":
        # GL ring count n+1 with 2 lmax + 1 pixels per ring
        x, w = np.polynomial.legendre.leggauss(n + 1)
        o = np.argsort(-x)
        nphi = np.full(n + 1, 2 * lmax + 1)
        return og.RingGrid("gl", n + 1, np.arccos(x[o]), np.zeros(n + 1), nphi,
                           w[o] * 2 * np.pi / (2 * lmax + 1), np.concatenate([[0], np.cumsum(nphi)]))
    return og.healpix(n)


@pytest.mark.parametrize("kind,n,lmax", CASES)
def test_grid_geometry_matches_oracle(kind, n, lmax):
    g, _ = _grids(kind, n, lmax)
    o = _oracle_grid(kind, n, lmax, g)
    np.testing.assert_allclose(g.theta, o.theta, rtol=0, atol=2e-14)
    # both Gauss-Legendre weight computations carry ~1e-11 relative error on the tiny
    # polar weights (checked against mpmath at n = 101); elsewhere they agree to 1e-14
    np.testing.assert_allclose(g.weight, o.weight, rtol=5e-11)
    np.testing.assert_allclose(g.phi0, o.phi0, atol=1e-15)
    np.testing.assert_array_equal(g.nphi, o.nphi)
    assert g.npix == o.npix


PRECS = [cw.CMBWS_FP64, cw.CMBWS_FP32, cw.CMBWS_FP32X2, cw.CMBWS_TF32, cw.CMBWS_3XTF32,
         cw.CMBWS_BF16, cw.CMBWS_BF16X3]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kind,n,lmax", CASES)
def test_synthesis_parity(kind, n, lmax, prec):
    g, _ = _grids(kind, n, lmax)
    o = _oracle_grid(kind, n, lmax, g)
    rng = np.random.default_rng(lmax + 7 * n)
    nmaps = 3
    alm = rng.standard_normal((nmaps, (lmax + 1) ** 2))
    out = to_dev(np.zeros((nmaps, g.npix)))
    cw.cmbws_sht_synth(g, prec, to_dev(alm), out, nmaps)
    got = to_host(out)
    for k in range(nmaps):
        ref = osht.synthesis(o, lmax, alm[k])
        assert rel_err(got[k], ref) < tol(prec, lmax), (k, rel_err(got[k], ref))


@pytest.mark.parametrize("weighted", [0, 1])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kind,n,lmax", CASES)
def test_adjoint_parity(kind, n, lmax, prec, weighted):
    g, _ = _grids(kind, n, lmax)
    o = _oracle_grid(kind, n, lmax, g)
    rng = np.random.default_rng(1000 + lmax + 7 * n)
    nmaps = 2
    maps = rng.standard_normal((nmaps, g.npix))
    out = to_dev(np.zeros((nmaps, (lmax + 1) ** 2)))
    cw.cmbws_sht_analysis(g, prec, to_dev(maps), out, nmaps, weighted)
    got = to_host(out)
    for k in range(nmaps):
        ref = osht.adjoint(o, lmax, maps[k], weighted=bool(weighted))
        assert rel_err(got[k], ref) < tol(prec, lmax, "adj"), (k, rel_err(got[k], ref))


@pytest.mark.parametrize("nmaps", [1, 4, 5, 9])
def test_map_batches_of_any_size(nmaps):
    g = cw.cmbws_plan_grid(cw.CMBWS_GRID_HEALPIX, 8, 23)
    o = og.healpix(8)
    alm = np.random.default_rng(nmaps).standard_normal((nmaps, 24 ** 2))
    out = to_dev(np.zeros((nmaps, g.npix)))
    cw.cmbws_sht_synth(g, cw.CMBWS_FP64, to_dev(alm), out, nmaps)
    got = to_host(out)
    back = to_dev(np.zeros((nmaps, 24 ** 2)))
    cw.cmbws_sht_analysis(g, cw.CMBWS_FP64, out, back, nmaps, 0)
    gb = to_host(back)
    for k in range(nmaps):
        assert rel_err(got[k], osht.synthesis(o, 23, alm[k])) < tol(cw.CMBWS_FP64, 23)
        assert rel_err(gb[k], osht.adjoint(o, 23, got[k])) < tol(cw.CMBWS_FP64, 23, "adj")


@pytest.mark.parametrize("prec", TC_PRECS)
@pytest.mark.parametrize("nmaps", [1, 2, 3, 4, 5, 9])
def test_tensor_core_synthesis_map_batches(nmaps, prec):
    # every map-count variant of the tensor-core kernel (1..4 maps per launch, 16 columns)
    g = cw.cmbws_plan_grid(cw.CMBWS_GRID_HEALPIX, 32, 95)
    o = og.healpix(32)
    alm = np.random.default_rng(50 + nmaps).standard_normal((nmaps, 96 ** 2))
    out = to_dev(np.zeros((nmaps, g.npix)))
    cw.cmbws_sht_synth(g, prec, to_dev(alm), out, nmaps)
    got = to_host(out)
    for k in range(nmaps):
        assert rel_err(got[k], osht.synthesis(o, 95, alm[k])) < tol(prec, 95), k


def round_trip_tol(prec, lmax):
    """Bound on the Gauss-Legendre round trip Y^T W Y a - a.  Unlike one transform, it also
    carries the error of the quadrature weights, and the oracle's own FP64 round trip grows
    like L^2 (1.6e-12 at L = 255, 7e-12 at L = 511): FP64 1e-16 (L+1)^2, double-float four
    times that; FP32 the sum of the synthesis and adjoint bounds."""
    n = lmax + 1
    if prec == cw.CMBWS_FP64:
        return max(1e-13, 1e-16 * n * n)
    if prec == cw.CMBWS_FP32X2:
        return max(4e-13, 4e-16 * n * n)
    return tol(prec, lmax) + tol(prec, lmax, "adj")


@pytest.mark.parametrize("lmax", [31, 255, 1023])
def test_gl_round_trip_exact_on_gpu(lmax):
    # the double-float path must match FP64 accuracy
    g0 = cw.cmbws_plan_grid(cw.CMBWS_GRID_GL, lmax + 1, lmax)
    a0 = np.random.default_rng(lmax + 1).standard_normal((lmax + 1) ** 2)
    m0 = to_dev(np.zeros(g0.npix))
    b0 = to_dev(np.zeros((lmax + 1) ** 2))
    cw.cmbws_sht_synth(g0, cw.CMBWS_FP32X2, to_dev(a0), m0, 1)
    cw.cmbws_sht_analysis(g0, cw.CMBWS_FP32X2, m0, b0, 1, 1)
    assert rel_err(to_host(b0), a0) < round_trip_tol(cw.CMBWS_FP32X2, lmax), rel_err(to_host(b0), a0)
    # Sec. 2.1: Y^T W Y = I on the Gauss-Legendre grid
    g = cw.cmbws_plan_grid(cw.CMBWS_GRID_GL, lmax + 1, lmax)
    a = np.random.default_rng(lmax).standard_normal((lmax + 1) ** 2)
    m = to_dev(np.zeros(g.npix))
    back = to_dev(np.zeros((lmax + 1) ** 2))
    cw.cmbws_sht_synth(g, cw.CMBWS_FP64, to_dev(a), m, 1)
    cw.cmbws_sht_analysis(g, cw.CMBWS_FP64, m, back, 1, 1)
    assert rel_err(to_host(back), a) < round_trip_tol(cw.CMBWS_FP64, lmax), rel_err(to_host(back), a)
    cw.cmbws_sht_synth(g, cw.CMBWS_FP32, to_dev(a), m, 1)
    cw.cmbws_sht_analysis(g, cw.CMBWS_FP32, m, back, 1, 1)
    assert rel_err(to_host(back), a) < round_trip_tol(cw.CMBWS_FP32, lmax), rel_err(to_host(back), a)


def test_adjointness_large_healpix():
    # <Y a, f> = <a, Y^T f> at Nside 256, L = 767 (several CTAs per m in both Legendre kernels)
    g = cw.cmbws_plan_grid(cw.CMBWS_GRID_HEALPIX, 256, 767)
    rng = np.random.default_rng(5)
    a = rng.standard_normal(768 ** 2)
    f = rng.standard_normal(g.npix)
    ya = to_dev(np.zeros(g.npix))
    ytf = to_dev(np.zeros(768 ** 2))
    cw.cmbws_sht_synth(g, cw.CMBWS_FP64, to_dev(a), ya, 1)
    cw.cmbws_sht_analysis(g, cw.CMBWS_FP64, to_dev(f), ytf, 1, 0)
    lhs = float(to_host(ya) @ f)
    rhs = float(a @ to_host(ytf))
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


@pytest.mark.parametrize("prec", [cw.CMBWS_FP64, cw.CMBWS_FP32X2, cw.CMBWS_FP32, cw.CMBWS_TF32,
                                  cw.CMBWS_3XTF32, cw.CMBWS_BF16, cw.CMBWS_BF16X3])
def test_full_size_sampled_rings_nside1024(prec):
    """Every precision against the oracle on rings from the pole to the equator.  Near the
    poles the FP32 recurrence runs in its difference form (an almost double characteristic
    root there makes the plain form lose ~l^2 eps); the tensor-core modes are also compared
    with the FP32 CUDA-core path, which shares their recurrence."""
    g = cw.cmbws_plan_grid(cw.CMBWS_GRID_HEALPIX, 1024, 3071)
    o = og.healpix(1024)
    L = 3071
    rng = np.random.default_rng(11)
    ell = np.concatenate([np.arange(L + 1)] + [np.r_[np.arange(m, L + 1), np.arange(m, L + 1)]
                                               for m in range(1, L + 1)])
    a = rng.standard_normal((L + 1) ** 2) / (1.0 + ell)
    out = to_dev(np.zeros(g.npix))
    cw.cmbws_sht_synth(g, prec, to_dev(a), out, 1)
    got = to_host(out)
    rings = np.array([0, 1, 5, 700, 1023, 1500, 2047, 2600, 4094])
    sub = og.RingGrid("healpix", 1024, o.theta[rings], o.phi0[rings], o.nphi[rings], o.weight[rings],
                      np.concatenate([[0], np.cumsum(o.nphi[rings])]))
    ref = osht.synthesis(sub, L, a)
    gsub = np.concatenate([got[o.offset[r]:o.offset[r + 1]] for r in rings])
    assert rel_err(gsub, ref) < tol(prec, L), rel_err(gsub, ref)
    if prec in TC_PRECS:
        f32 = to_dev(np.zeros(g.npix))
        cw.cmbws_sht_synth(g, cw.CMBWS_FP32, to_dev(a), f32, 1)
        g32 = to_host(f32)
        g32 = np.concatenate([g32[o.offset[r]:o.offset[r + 1]] for r in rings])
        # the tensor cores replace only the contraction: TF32 rounding (2^-11 per factor), or
        # split TF32 (2^-22) whose difference from the CUDA-core path is that of two FP32
        # accumulations of L terms in different orders (within the split mode's own bound)
        bound = tol(prec, L)
        assert rel_err(gsub, g32) < bound, rel_err(gsub, g32)


SAMPLED_M = [0, 1, 2, 700, 1535, 3000, 3071]


def full_size_adjoint_tol(prec):
    """The adjoint bound of tol() at L = 3071 (FP64 1.4e-11, FP32X2 2.2e-11, FP32 1.8e-5,
    BF16 1.5e-2, BF16X3 4e-5; measured on GB300: 1.3e-12, 2.5e-12, 1.9e-6)."""
    return tol(prec, 3071, "adj")


@pytest.fixture(scope="module")
def nside1024():
    g = cw.cmbws_plan_grid(cw.CMBWS_GRID_HEALPIX, 1024, 3071)
    return g, og.healpix(1024)


@pytest.mark.parametrize("weighted", [0, 1])
@pytest.mark.parametrize("prec", [cw.CMBWS_FP64, cw.CMBWS_FP32X2, cw.CMBWS_FP32, cw.CMBWS_BF16,
                                  cw.CMBWS_BF16X3])
def test_full_size_adjoint_sampled_orders_nside1024(nside1024, prec, weighted):
    """Adjoint synthesis / analysis of three maps at HEALPix Nside 1024, L = 3071 (the
    bench's largest band grid, three bands per launch as in its solves) against the oracle on
    every l of a sample of orders m, from m = 0 to m = L: the Legendre stage is independent
    per m, so the oracle evaluates those columns exactly."""
    g, o = nside1024
    L, nmaps = 3071, 3
    rng = np.random.default_rng(31 + weighted)
    maps = rng.standard_normal((nmaps, g.npix))
    out = to_dev(np.zeros((nmaps, (L + 1) ** 2)))
    cw.cmbws_sht_analysis(g, prec, to_dev(maps), out, nmaps, weighted)
    got = to_host(out)
    errs = []
    for k in range(nmaps):
        ref = osht.adjoint_m(o, L, maps[k], SAMPLED_M, weighted=bool(weighted))
        gv = np.concatenate([np.concatenate(osht.packed_m(got[k], L, m)) for m in SAMPLED_M])
        rv = np.concatenate([np.concatenate(ref[m]) for m in SAMPLED_M])
        errs.append(rel_err(gv, rv))
    print(f"full-size adjoint prec={prec} weighted={weighted}: max rel err {max(errs):.3e}")
    assert max(errs) < full_size_adjoint_tol(prec), errs


@pytest.mark.parametrize("prec", [cw.CMBWS_BF16, cw.CMBWS_BF16X3])
@pytest.mark.parametrize("nmaps", [1, 2, 3, 4, 5, 9])
def test_tensor_core_adjoint_map_batches(nmaps, prec):
    """Every map-count variant of the tensor-core adjoint (1..4 maps per launch) on a grid
    with several 128-l tiles per m and a ragged last stage of ring pairs (Nside 40: 80 ring
    pairs, 64 per stage), against the oracle and against the FP32 CUDA-core adjoint."""
    g = cw.cmbws_plan_grid(cw.CMBWS_GRID_HEALPIX, 40, 150)
    o = og.healpix(40)
    maps = np.random.default_rng(70 + nmaps).standard_normal((nmaps, g.npix))
    out = to_dev(np.zeros((nmaps, 151 ** 2)))
    ref32 = to_dev(np.zeros((nmaps, 151 ** 2)))
    cw.cmbws_sht_analysis(g, prec, to_dev(maps), out, nmaps, 1)
    cw.cmbws_sht_analysis(g, cw.CMBWS_FP32, to_dev(maps), ref32, nmaps, 1)
    got, g32 = to_host(out), to_host(ref32)
    for k in range(nmaps):
        ref = osht.adjoint(o, 150, maps[k], weighted=True)
        assert rel_err(got[k], ref) < tol(prec, 150, "adj"), (k, rel_err(got[k], ref))
        assert rel_err(got[k], g32[k]) < tol(prec, 150, "adj"), k

