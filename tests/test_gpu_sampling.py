"""GPU parity of the constrained-realization draws (cmbws_draw, cmbws_cr_rhs, cmbws_cr_sample,
cmbws_powerlaw_mixing) against oracle/sampling.py (Sec. 2.3)."""
import ctypes

import numpy as np
import pytest

from oracle import model as omodel
from oracle import sampling as osamp
from tests._gpu import gpu_model, rel_err, to_dev, to_host
from tests._models import multires_small, oracle_model, tiny_workload

pytestmark = pytest.mark.gpu

M64 = (1 << 64) - 1
ERR_ARG = -1   # CMBWS_ERR_ARG
# (seed, sample, stream, offset, n): ragged offsets and lengths, extreme keys and counters
CASES = [(0, 0, 0, 0, 1), (1, 2, 3, 1, 3), (7, 0, 1, 2, 4), (M64, 1 << 63, M64, 3, 5),
         (1710, 5, 2, 4099, 1023), (42, 9, 0, 0, 100003), (5, 5, 5, (1 << 40) + 1, 77)]


def _draw(seed, sample, sid, offset, n, kind):
    import paper_1710_00621_gb300 as cw
    import torch
    out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    cw.cmbws_draw(seed, sample, sid, offset, out, kind=kind)
    return to_host(out)


@pytest.mark.parametrize("case", CASES)
def test_uniforms_bit_exact(case):
    seed, sample, sid, off, n = case
    assert np.array_equal(_draw(seed, sample, sid, off, n, 1),
                          osamp.uniforms(seed, sample, sid, off, n))


@pytest.mark.parametrize("case", CASES)
def test_normals(case):
    seed, sample, sid, off, n = case
    got = _draw(seed, sample, sid, off, n, 0)
    ref = osamp.normals(seed, sample, sid, off, n)
    # the same exact uniforms on both sides; FP64 log / sqrt / cos / sin (|z| < 9): ~1e-15
    assert np.max(np.abs(got - ref)) < 1e-13


def test_draw_full_size_band_sampled():
    """One Nside-1024 band (12.6 M pixels) in one launch: sampled variates against the
    oracle one by one, and the moments of all of them."""
    n = 12 * 1024 ** 2
    seed, sample, sid = 171000621, 3, 9
    got = _draw(seed, sample, sid, 0, n, 0)
    rng = np.random.default_rng(1)
    idx = np.concatenate([[0, 1, 2, 3, 4, n - 5, n - 1], rng.integers(0, n, 1500)])
    ref = np.array([osamp.normals(seed, sample, sid, int(j), 1)[0] for j in idx])
    assert np.max(np.abs(got[idx] - ref)) < 1e-13
    assert abs(got.mean()) < 5 / np.sqrt(n)
    assert abs(got.var() - 1.0) < 5 * np.sqrt(2.0 / n)


def test_draw_errors_and_empty():
    import paper_1710_00621_gb300 as cw
    import torch
    lib = cw.load_library()
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    assert lib.cmbws_draw(1, 1, 0, -1, 4, 0, p, None) == ERR_ARG
    assert lib.cmbws_draw(1, 1, 0, 0, -4, 0, p, None) == ERR_ARG
    assert lib.cmbws_draw(1, 1, 0, 0, 4, 2, p, None) == ERR_ARG
    assert lib.cmbws_draw(1, 1, 0, 0, 4, 0, None, None) == ERR_ARG
    assert lib.cmbws_draw(1, 1, 0, 0, 0, 0, None, None) == 0
    torch.cuda.synchronize()
    assert float(buf.abs().sum()) == 0.0


def _data(m, inp):
    return [a + b for a, b in zip(omodel.project(m, inp["x_true"]), inp["noise"])]


@pytest.mark.parametrize("case", ["gl_tiny", "multires"])
def test_cr_rhs_parity(case):
    import paper_1710_00621_gb300 as cw
    import torch
    w = tiny_workload(15) if case == "gl_tiny" else multires_small(32)
    m, inp = oracle_model(w)
    d = _data(m, inp)
    for prec in (cw.CMBWS_FP64, cw.CMBWS_FP32):
        gm, _ = gpu_model(w, inp, prec)
        b = torch.zeros(m.nvec(), dtype=torch.float64, device="cuda")
        cw.cmbws_cr_rhs(gm, [to_dev(x) for x in d], 1710, 4, b)
        ref = osamp.cr_rhs(m, d, 1710, 4)
        # FP64 transforms, or double-float ones (FP32 models), both FP64-accurate
        assert rel_err(to_host(b), ref) < 1e-10, (prec, rel_err(to_host(b), ref))


def test_cr_sample_matches_oracle_solution_and_warm_start():
    import paper_1710_00621_gb300 as cw
    import torch
    w = tiny_workload(15)
    m, inp = oracle_model(w)
    d = _data(m, inp)
    A = omodel.dense_A(m)
    dd = [to_dev(x) for x in d]
    ref = [np.linalg.solve(A, osamp.cr_rhs(m, d, 77, s)) for s in range(2)]
    for prec, cert, tol, bound in ((cw.CMBWS_FP64, cw.CMBWS_FP64, 1e-11, 1e-8),
                                   (cw.CMBWS_FP32, cw.CMBWS_FP32X2, 1e-9, 1e-6)):
        gm, _ = gpu_model(w, inp, prec)
        x = torch.zeros(m.nvec(), dtype=torch.float64, device="cuda")
        r0 = cw.cmbws_cr_sample(gm, dd, 77, 0, x, tol=tol, maxiter=2000, cert_prec=cert)
        assert r0["rel_res"] <= tol
        assert rel_err(to_host(x), ref[0]) < bound, rel_err(to_host(x), ref[0])
        # the next sample of a chain, started from the previous one
        r1 = cw.cmbws_cr_sample(gm, dd, 77, 1, x, tol=tol, maxiter=2000, cert_prec=cert)
        assert r1["rel_res"] <= tol
        assert rel_err(to_host(x), ref[1]) < bound
        # cold start gives the same sample
        xc = torch.zeros_like(x)
        cw.cmbws_cr_sample(gm, dd, 77, 1, xc, tol=tol, maxiter=2000, cert_prec=cert)
        assert rel_err(to_host(xc), ref[1]) < bound
    assert rel_err(ref[0], ref[1]) > 1e-3        # distinct draws


def test_powerlaw_mixing_parity_and_variable_model():
    """q = mask (nu / nu_0)^beta(n) on a mixing grid, and a model with those maps for the dust
    component against the oracle model with the oracle's maps (Eq. Q)."""
    import paper_1710_00621_gb300 as cw
    import torch
    from oracle import grids as og
    w = tiny_workload(15)
    m0, inp = oracle_model(w)
    Lmix = 20
    g = og.gauss_legendre(Lmix)
    th, ph = g.pixel_angles()
    beta = 1.6 + 0.15 * np.cos(th) + 0.1 * np.sin(th) * np.cos(2 * ph)
    mask = (np.abs(np.cos(th)) >= np.sin(np.radians(15.0))).astype(np.float64)
    k = 1
    dust = w.comps[k]
    maps = [[None] * m0.ncomp for _ in range(m0.nobs)]
    lm = [[None] * m0.ncomp for _ in range(m0.nobs)]
    for nu, b in enumerate(w.bands):
        ratio = b.freq / dust.nu0
        ref = osamp.powerlaw_mixing(ratio, beta, mask)
        q = torch.empty(g.npix, dtype=torch.float64, device="cuda")
        cw.cmbws_powerlaw_mixing(ratio, to_dev(beta), q, mask=to_dev(mask))
        got = to_host(q)
        assert np.array_equal(got == 0, ref == 0)
        assert rel_err(got, ref) < 1e-14
        maps[nu][k] = got
        lm[nu][k] = Lmix
    mg = [[g if maps[nu][kk] is not None else None for kk in range(m0.ncomp)]
          for nu in range(m0.nobs)]
    mo, _ = oracle_model(w, mix_maps=maps, mix_grids=mg)
    gm, _ = gpu_model(w, inp, cw.CMBWS_FP64, mix=(lm, maps))
    x = np.random.default_rng(4).standard_normal(mo.nvec())
    y = torch.zeros(mo.nvec(), dtype=torch.float64, device="cuda")
    cw.cmbws_apply_A(gm, to_dev(x), y)
    assert rel_err(to_host(y), omodel.apply_A(mo, x)) < 1e-10
