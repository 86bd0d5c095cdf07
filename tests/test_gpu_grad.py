"""GPU parity of the solution gradient (cmbws_grad_terms and the autograd wrapper).

* the gradient terms against the oracle's operator form on the same x, lambda, d;
* the full gradient of ||W x||^2 against the oracle (dense Cholesky solves) at L = 31;
* the gradient in spectral indices and amplitudes against central finite differences
  of FP64 GPU solves (step 1e-4), at L = 127 and at the full L = 511 problem, where the
  FP32 model (FP64 scalars, double-float certified residual) is compared as well.
"""
import numpy as np
import pytest

import skygen
from oracle import grad as ograd
from oracle import model as omodel
from tests._gpu import GridCache, gpu_model, rel_err, to_dev, to_host
from tests._models import oracle_model

pytestmark = pytest.mark.gpu


def _inputs(L, cr=False):
    w = skygen.differentiable(lmax=L)
    m, inp = oracle_model(w)
    d = omodel.project(m, inp["x_true"])
    d = [a + n for a, n in zip(d, inp["noise"])]
    rng = np.random.default_rng([L, 3])
    o1 = [rng.standard_normal(t.size) for t in m.tau] if cr else None
    o2 = rng.standard_normal(m.nvec()) if cr else None
    return w, m, inp, d, o1, o2


@pytest.mark.parametrize("L,cr", [(31, False), (31, True), (100, True)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_grad_terms_parity(L, cr, prec):
    import paper_1710_00621_gb300 as cw
    import torch
    w, m, inp, d, o1, o2 = _inputs(L, cr)
    p = cw.CMBWS_FP64 if prec == "fp64" else cw.CMBWS_FP32
    gm, _ = gpu_model(w, inp, p)
    rng = np.random.default_rng(17)
    x = rng.standard_normal(m.nvec())
    lam = rng.standard_normal(m.nvec())
    dq0, dt0 = ograd.grad_terms(m, x, lam, d, o1, o2)
    out = torch.empty(m.nobs * m.ncomp + m.ncomp, dtype=torch.float64, device="cuda")
    cw.cmbws_grad_terms(gm, to_dev(x), to_dev(lam), [to_dev(a) for a in d], out,
                        [to_dev(a) for a in o1] if cr else None, to_dev(o2) if cr else None)
    g = to_host(out)
    # FP64-accurate transforms either way (FP32 models evaluate the terms in double-float)
    tol = max(1e-11, 4e-16 * (L + 1) ** 2)
    assert rel_err(g[:m.nobs * m.ncomp].reshape(m.nobs, m.ncomp), dq0) < tol
    assert rel_err(g[m.nobs * m.ncomp:], dt0) < 1e-13


def _var_inputs(L, Lmix, cr=False):
    """The differentiable workload with the dust pair of every band on a variable mixing map
    (a smooth pattern around the scalar value) on a Gauss-Legendre mixing grid of band-limit
    Lmix, and band maps drawn from that model."""
    from oracle import grids as og
    w, m0, inp, _, o1, o2 = _inputs(L, cr)
    g = og.gauss_legendre(Lmix)
    th, ph = g.pixel_angles()
    k = 2
    lm = [[None] * m0.ncomp for _ in range(m0.nobs)]
    maps = [[None] * m0.ncomp for _ in range(m0.nobs)]
    for nu in range(m0.nobs):
        maps[nu][k] = m0.q[nu, k] * (1.0 + 0.4 * np.cos(th) + 0.2 * np.sin(th) * np.cos(ph + nu))
        lm[nu][k] = Lmix
    grids = [[g if maps[nu][j] is not None else None for j in range(m0.ncomp)] for nu in range(m0.nobs)]
    m = omodel.Model(**{**m0.__dict__, "mix_map": maps, "mix_grid": grids})
    d = [a + n for a, n in zip(omodel.project(m, inp["x_true"]), inp["noise"])]
    return w, m, inp, d, o1, o2, (lm, maps)


@pytest.mark.parametrize("cr", [False, True])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_grad_variable_mixing_parity(prec, cr):
    """cmbws_grad_terms (offset entries of the variable pairs) and cmbws_grad_mix_maps against
    the oracle's operator forms on the same x, lambda, d."""
    import paper_1710_00621_gb300 as cw
    import torch
    w, m, inp, d, o1, o2, mix = _var_inputs(15, 20, cr)
    p = cw.CMBWS_FP64 if prec == "fp64" else cw.CMBWS_FP32
    gm, _ = gpu_model(w, inp, p, mix=mix)
    rng = np.random.default_rng(19)
    x = rng.standard_normal(m.nvec())
    lam = rng.standard_normal(m.nvec())
    dq0, dt0 = ograd.grad_terms(m, x, lam, d, o1, o2)
    maps0 = ograd.grad_mix_maps(m, x, lam, d, o1)
    out = torch.empty(m.nobs * m.ncomp + m.ncomp, dtype=torch.float64, device="cuda")
    dd = [to_dev(a) for a in d]
    w1 = [to_dev(a) for a in o1] if cr else None
    cw.cmbws_grad_terms(gm, to_dev(x), to_dev(lam), dd, out, w1, to_dev(o2) if cr else None)
    g = to_host(out)
    assert rel_err(g[:m.nobs * m.ncomp].reshape(m.nobs, m.ncomp), dq0) < 1e-11
    assert rel_err(g[m.nobs * m.ncomp:], dt0) < 1e-13
    outm = [[None if (nu, k) not in maps0 else torch.zeros(maps0[(nu, k)].size, dtype=torch.float64,
                                                          device="cuda")
             for k in range(m.ncomp)] for nu in range(m.nobs)]
    cw.cmbws_grad_mix_maps(gm, to_dev(x), to_dev(lam), dd, outm, w1)
    for (nu, k), ref in maps0.items():
        assert rel_err(to_host(outm[nu][k]), ref) < 1e-11, (nu, k)
    # the sum of each map is its offset entry
    for (nu, k), ref in maps0.items():
        assert abs(to_host(outm[nu][k]).sum() - g[nu * m.ncomp + k]) <= 1e-12 * np.abs(ref).sum()
    # a model without variable mixing is refused
    gs, _ = gpu_model(w, inp, p)
    with pytest.raises(cw.CmbwsError) as e:
        cw.cmbws_grad_mix_maps(gs, to_dev(x), to_dev(lam), dd, [[None] * m.ncomp for _ in range(m.nobs)])
    assert e.value.code == -1


def test_mixing_map_gradient_l31_dense_oracle_and_central_differences():
    """A variable-map model at L = 31 (mixing grid L = 40): the GPU solves x and lambda for the
    loss ||W x||^2 in FP64; the mixing-map gradient equals the oracle's dense form on those
    vectors, and central differences of the GPU loss in single map pixels (pole, equator, mid
    latitudes; two bands, the model rebuilt each time) match it."""
    import paper_1710_00621_gb300 as cw
    import torch
    w, m, inp, d, _, _, (lm, maps) = _var_inputs(31, 40)
    wgt = skygen.harmonic_weight(m.lmax_comp)
    dd = [to_dev(a) for a in d]
    cache = GridCache()

    def solve(mp):
        gm, _ = gpu_model(w, inp, cw.CMBWS_FP64, cache=cache, mix=(lm, mp))
        b = torch.zeros(m.nvec(), dtype=torch.float64, device="cuda")
        cw.cmbws_rhs(gm, dd, b)
        x = torch.zeros_like(b)
        rep = cw.cmbws_cg_solve(gm, b, x, tol=1e-13, maxiter=5000)
        assert rep["rel_res"] <= 1e-13
        xh = to_host(x)
        return gm, xh, float(np.sum((wgt * xh) ** 2))

    gm, x, L0 = solve(maps)
    gl = to_dev(2.0 * wgt * wgt * x)
    lam = torch.zeros_like(gl)
    cw.cmbws_cg_solve(gm, gl, lam, tol=1e-13, maxiter=5000)
    lam = to_host(lam)
    outm = [[None if maps[nu][k] is None else torch.zeros(maps[nu][k].size, dtype=torch.float64,
                                                         device="cuda")
             for k in range(m.ncomp)] for nu in range(m.nobs)]
    cw.cmbws_grad_mix_maps(gm, to_dev(x), to_dev(lam), dd, outm)
    ref = ograd.grad_mix_maps_dense(m, x, lam, d)
    for (nu, k), r in ref.items():
        assert rel_err(to_host(outm[nu][k]), r) < 1e-10, (nu, k, rel_err(to_host(outm[nu][k]), r))
    npix = maps[0][2].size
    for nu in (0, 3):
        gmap = to_host(outm[nu][2])
        for p in (0, npix // 2, npix // 3 + 7, npix - 1):
            h = 1e-4 * abs(maps[nu][2][p])
            vals = []
            for sgn in (+1, -1):
                mp = [[None if q is None else q.copy() for q in row] for row in maps]
                mp[nu][2][p] += sgn * h
                vals.append(solve(mp)[2])
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - gmap[p]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(gmap).max()), (nu, p, fd, gmap[p])


def test_spectral_index_map_autograd_central_differences():
    """A spectral-index map beta(p) of the dust on its mixing grid, q_{nu,dust}(p) =
    (nu / nu_0)^beta(p) in torch, through wiener_solution_maps: d||W x||^2 / dbeta(p) by
    autograd against central differences of the same FP64 solves in single pixels."""
    import paper_1710_00621_gb300 as cw
    import torch
    from paper_1710_00621_gb300.autodiff import WienerProblem, wiener_solution_maps
    from oracle import grids as og
    w, m, inp, d, _, _, (lm, maps) = _var_inputs(15, 20)
    cache = GridCache()
    g = og.gauss_legendre(20)
    th, _ = g.pixel_angles()
    mgrid = cw.cmbws_plan_grid(cw.CMBWS_GRID_GL, 21, 20)
    k = 2
    mix_grids = [[mgrid if j == k else None for j in range(m.ncomp)] for _ in range(m.nobs)]
    prob = WienerProblem([c.lmax for c in w.comps], [cache.get(b) for b in w.bands], inp["beams"],
                         inp["cl"], [to_dev(t) for t in inp["tau"]], [to_dev(a) for a in d],
                         prec=cw.CMBWS_FP64, tol=1e-13, maxiter=5000, mix_grids=mix_grids)
    freqs = torch.tensor([b.freq for b in w.bands], dtype=torch.float64, device="cuda")
    nu0 = w.comps[k].nu0
    beta0 = torch.as_tensor(w.comps[k].beta + 0.1 * np.cos(th), device="cuda")
    wgt = to_dev(skygen.harmonic_weight(m.lmax_comp))
    q = torch.as_tensor(m.q, device="cuda")
    t = torch.zeros(m.ncomp, dtype=torch.float64, device="cuda")

    def loss_of(beta):
        mp = [[(freqs[nu] / nu0) ** beta if j == k else None for j in range(m.ncomp)]
              for nu in range(m.nobs)]
        x = wiener_solution_maps(q, t, mp, prob)
        return ((wgt * x) ** 2).sum()

    beta = beta0.clone().requires_grad_(True)
    loss = loss_of(beta)
    loss.backward()
    gb = beta.grad.cpu().numpy()
    h = 1e-5
    with torch.no_grad():
        for p in (0, th.size // 2, th.size // 3 + 4, th.size - 1):
            vals = []
            for sgn in (+1, -1):
                bb = beta0.clone()
                bb[p] += sgn * h
                vals.append(float(loss_of(bb)))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - gb[p]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(gb).max()), (p, fd, gb[p])


def _problem(w, inp, d, prec, tol, cache):
    import paper_1710_00621_gb300 as cw
    from paper_1710_00621_gb300.autodiff import WienerProblem
    grids = [cache.get(b) for b in w.bands]
    return WienerProblem([c.lmax for c in w.comps], grids, inp["beams"], inp["cl"],
                         [to_dev(t) for t in inp["tau"]], [to_dev(a) for a in d], prec=prec,
                         tol=tol, maxiter=5000)


def _params(w):
    import torch
    betas = torch.tensor([0.0 if c.beta is None else c.beta for c in w.comps], dtype=torch.float64,
                         requires_grad=True)
    logamp = torch.zeros(len(w.comps), dtype=torch.float64, requires_grad=True)
    return betas, logamp


def _loss(w, prob, betas, logamp, wgt):
    from paper_1710_00621_gb300.autodiff import power_law_q, wiener_solution
    q = power_law_q([b.freq for b in w.bands], [c.nu0 for c in w.comps], betas,
                    [c.beta is None for c in w.comps])
    x = wiener_solution(q, logamp, prob)
    return ((wgt * x) ** 2).sum()


def test_gradient_matches_oracle_dense_l31():
    import paper_1710_00621_gb300 as cw
    w, m, inp, d, _, _ = _inputs(31)
    wgt_h = skygen.harmonic_weight(m.lmax_comp)
    b = omodel.rhs(m, d)
    x = ograd.solve_dense(m, b)
    L0, g = ograd.weighted_loss(x, wgt_h)
    lam = ograd.solve_dense(m, g)
    dq, dt = ograd.grad_terms(m, x, lam, d)
    freqs = np.array([bd.freq for bd in w.bands])
    dbeta = np.array([0.0 if c.beta is None else np.sum(dq[:, k] * m.q[:, k] * np.log(freqs / c.nu0))
                      for k, c in enumerate(w.comps)])
    prob = _problem(w, inp, d, cw.CMBWS_FP64, 1e-12, GridCache())
    betas, logamp = _params(w)
    loss = _loss(w, prob, betas, logamp, to_dev(wgt_h))
    loss.backward()
    assert abs(loss.item() - L0) < 1e-9 * L0
    gb = betas.grad.numpy()
    ga = logamp.grad.numpy()
    for k, c in enumerate(w.comps):
        if c.beta is not None:
            assert abs(gb[k] - dbeta[k]) < 1e-7 * abs(dbeta[k]), (k, gb[k], dbeta[k])
    np.testing.assert_allclose(ga, dt, rtol=1e-7)


def _fd_check(L, h=1e-4):
    import paper_1710_00621_gb300 as cw
    import torch
    w, m, inp, d, _, _ = _inputs(L)
    cache = GridCache()
    wgt = to_dev(skygen.harmonic_weight(m.lmax_comp))
    prob = _problem(w, inp, d, cw.CMBWS_FP64, 1e-12, cache)
    betas, logamp = _params(w)
    loss = _loss(w, prob, betas, logamp, wgt)
    loss.backward()
    grad = np.concatenate([betas.grad.numpy(), logamp.grad.numpy()])
    fd = np.zeros_like(grad)
    base = np.concatenate([betas.detach().numpy(), logamp.detach().numpy()])
    nc = len(w.comps)
    with torch.no_grad():
        for i in range(2 * nc):
            if i < nc and w.comps[i].beta is None:
                continue
            vals = []
            for s in (+1, -1):
                p = base.copy()
                p[i] += s * h
                vals.append(float(_loss(w, prob, torch.tensor(p[:nc]), torch.tensor(p[nc:]), wgt)))
            fd[i] = (vals[0] - vals[1]) / (2 * h)
    for i in range(2 * nc):
        if i < nc and w.comps[i].beta is None:
            continue
        assert abs(fd[i] - grad[i]) <= 2e-6 * max(abs(fd[i]), 1e-6 * loss.item()), (i, fd[i], grad[i])
    return w, inp, d, cache, wgt, grad


def test_gradient_central_differences_l127():
    _fd_check(127)


def test_gradient_full_size_l511_fp64_fd_and_fp32():
    import paper_1710_00621_gb300 as cw
    w, inp, d, cache, wgt, g64 = _fd_check(511)
    prob = _problem(w, inp, d, cw.CMBWS_FP32, 1e-10, cache)
    betas, logamp = _params(w)
    loss = _loss(w, prob, betas, logamp, wgt)
    loss.backward()
    g32 = np.concatenate([betas.grad.numpy(), logamp.grad.numpy()])
    nc = len(w.comps)
    for i in range(2 * nc):
        if i < nc and w.comps[i].beta is None:
            continue
        assert abs(g32[i] - g64[i]) <= 1e-7 * abs(g64[i]), (i, g32[i], g64[i])


@pytest.mark.parametrize("kind", ["gl", "healpix"])
def test_sht_autograd_pair_gradients(kind):
    """The synthesis / adjoint-synthesis autograd pair: gradients of a quadratic loss through
    Y and through Y^T against the explicit transposes (the oracle's dense Y at L = 15) and
    against central finite differences of the library's own transforms."""
    import torch
    import paper_1710_00621_gb300 as cw
    from paper_1710_00621_gb300.autodiff import sht_adjoint, sht_synth
    from oracle import grids as og, sht as osht
    L = 15
    if kind == "gl":
        g = cw.cmbws_plan_grid(cw.CMBWS_GRID_GL, L + 1, L)
        o = og.gauss_legendre(L)
    else:
        g = cw.cmbws_plan_grid(cw.CMBWS_GRID_HEALPIX, 8, L)
        o = og.healpix(8)
    Y = osht.dense_Y(o, L)
    rng = np.random.default_rng(41)
    a0 = rng.standard_normal((2, (L + 1) ** 2))
    wm = rng.standard_normal((2, g.npix))
    # L(a) = sum w * (Y a)^2  ->  dL/da = 2 Y^T (w * Y a)
    a = torch.tensor(a0, device="cuda", requires_grad=True)
    loss = (to_dev(wm) * sht_synth(a, g) ** 2).sum()
    loss.backward()
    ref = np.stack([2 * Y.T @ (wm[k] * (Y @ a0[k])) for k in range(2)])
    assert rel_err(a.grad.cpu().numpy(), ref) < 1e-12
    # L(f) = sum v * (Y^T f)^2  ->  dL/df = 2 Y (v * Y^T f)
    f0 = rng.standard_normal((2, g.npix))
    va = rng.standard_normal((2, (L + 1) ** 2))
    f = torch.tensor(f0, device="cuda", requires_grad=True)
    loss2 = (to_dev(va) * sht_adjoint(f, g) ** 2).sum()
    loss2.backward()
    ref2 = np.stack([2 * Y @ (va[k] * (Y.T @ f0[k])) for k in range(2)])
    assert rel_err(f.grad.cpu().numpy(), ref2) < 1e-12
    # central differences of the library's transforms along a random direction
    dirn = rng.standard_normal((2, (L + 1) ** 2))
    h = 1e-4

    def lossf(av):
        with torch.no_grad():
            return float((to_dev(wm) * sht_synth(to_dev(av), g) ** 2).sum())
    fd = (lossf(a0 + h * dirn) - lossf(a0 - h * dirn)) / (2 * h)
    assert abs(fd - float((a.grad.cpu().numpy() * dirn).sum())) <= 1e-7 * abs(fd)
