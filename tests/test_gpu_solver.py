"""GPU parity of A, M_PI, the RHS and the PCG solve against the oracle, through the C ABI."""
import numpy as np
import pytest

import paper_1710_00621_gb300 as cw
import skygen
from oracle import closed_form, model as om, precond as opc
from oracle.cg import pcg
from tests._gpu import GridCache, gpu_model, rel_err, to_dev, to_host
from tests._models import multires_small, oracle_model, tiny_workload

pytestmark = pytest.mark.gpu

TOL = {cw.CMBWS_FP64: 1e-10, cw.CMBWS_FP32: 1e-4, cw.CMBWS_FP32X2: 1e-10}
PRECS = [cw.CMBWS_FP64, cw.CMBWS_FP32, cw.CMBWS_FP32X2]


def _setups():
    out = {}
    out["tiny15"] = tiny_workload(15)
    out["multires64"] = multires_small(64)
    out["multires16"] = multires_small(16)     # Nside 16/32/64, L_nu up to 191, comps 125/31/187
    return out


SETUPS = _setups()


@pytest.fixture(scope="module")
def models():
    cache = {}
    for name, work in SETUPS.items():
        om_, inp = oracle_model(work)
        cache[name] = (work, om_, inp)
    return cache


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", list(SETUPS))
def test_apply_A_parity(models, name, prec):
    work, m, inp = models[name]
    g, _ = gpu_model(work, inp, prec)
    x = np.random.default_rng(1).standard_normal(m.nvec())
    y = to_dev(np.zeros(m.nvec()))
    cw.cmbws_apply_A(g, to_dev(x), y)
    assert rel_err(to_host(y), om.apply_A(m, x)) < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", list(SETUPS))
def test_apply_precond_parity(models, name, prec):
    work, m, inp = models[name]
    g, _ = gpu_model(work, inp, prec)
    r = np.random.default_rng(2).standard_normal(m.nvec())
    z = to_dev(np.zeros(m.nvec()))
    cw.cmbws_apply_precond(g, to_dev(r), z)
    assert rel_err(to_host(z), opc.apply_precond(m, r)) < TOL[prec]


def test_model_counts_shts_like_the_paper(models):
    # Sec. 3.3: A costs 2 (2 Nmix + Nobs) SHTs, M_PI costs 2 Nobs; scalar mixing has Nmix = 0
    work, m, inp = models["multires64"]
    g, _ = gpu_model(work, inp)
    assert g.nsht_A == 2 * 9 and g.nsht_M == 2 * 9
    assert g.nvec == m.nvec()


@pytest.mark.parametrize("prec", [cw.CMBWS_FP64, cw.CMBWS_FP32])
@pytest.mark.parametrize("name", ["tiny15", "multires64"])
def test_rhs_parity(models, name, prec):
    # the RHS is FP64-accurate for every model (double-float transforms for FP32 models)
    work, m, inp = models[name]
    g, grids = gpu_model(work, inp, prec)
    d = [mp + n for mp, n in zip(om.project(m, inp["x_true"]), inp["noise"])]
    rng = np.random.default_rng(3)
    w1 = [rng.standard_normal(x.size) for x in d]
    w2 = rng.standard_normal(m.nvec())
    b = to_dev(np.zeros(m.nvec()))
    cw.cmbws_rhs(g, [to_dev(x) for x in d], b)
    assert rel_err(to_host(b), om.rhs(m, d)) < 1e-10
    cw.cmbws_rhs(g, [to_dev(x) for x in d], b, omega1=[to_dev(x) for x in w1], omega2=to_dev(w2))
    assert rel_err(to_host(b), om.rhs(m, d, w1, w2)) < 1e-10


def test_flat_noise_solve_is_closed_form_in_one_iteration():
    work = tiny_workload(31)
    m, inp = oracle_model(work, flat=True)
    g, _ = gpu_model(work, inp)
    sig = [b.sigma for b in work.bands]
    b = np.random.default_rng(4).standard_normal(m.nvec())
    ref = closed_form.solve(m.lmax_comp, m.lmax_band, m.beam, m.cl, m.q, sig, b)
    x = to_dev(np.zeros(m.nvec()))
    rep = cw.cmbws_cg_solve(g, to_dev(b), x, tol=1e-10, maxiter=50)
    assert rep["iters"] == 1
    assert rel_err(to_host(x), ref) < 1e-10


def test_tiny_plain_workload_solve_matches_oracle():
    # Ncomp 2, Nobs 3, GL L = 63 (64 x 127 px), tol 1e-8, b = A x_true (Sec. 2.3 error tracking)
    work = skygen.tiny_plain()
    m, inp = oracle_model(work)
    g, _ = gpu_model(work, inp)
    b = om.apply_A(m, inp["x_true"])
    x = to_dev(np.zeros(m.nvec()))
    rep = cw.cmbws_cg_solve(g, to_dev(b), x, tol=1e-8, maxiter=500)
    assert rep["rel_res"] <= 1e-8
    xo, info = pcg(lambda v: om.apply_A(m, v), b, lambda v: opc.apply_precond(m, v), tol=1e-12)
    assert rel_err(to_host(x), xo) < 1e-6
    assert abs(rep["iters"] - info["iters"]) <= 3 or rep["iters"] <= info["iters"]


@pytest.mark.parametrize("name", ["multires64"])
def test_wiener_solve_fp64_and_fp32_refined(models, name):
    work, m, inp = models[name]
    d = [mp + n for mp, n in zip(om.project(m, inp["x_true"]), inp["noise"])]
    b = om.rhs(m, d)
    xo, _ = pcg(lambda v: om.apply_A(m, v), b, lambda v: opc.apply_precond(m, v), tol=1e-12,
                maxiter=2000)
    for prec, cert in ((cw.CMBWS_FP64, cw.CMBWS_FP64), (cw.CMBWS_FP32, cw.CMBWS_FP64),
                       (cw.CMBWS_FP32, cw.CMBWS_FP32X2), (cw.CMBWS_FP32X2, cw.CMBWS_FP32X2)):
        g, _ = gpu_model(work, inp, prec)
        x = to_dev(np.zeros(m.nvec()))
        rep = cw.cmbws_cg_solve(g, to_dev(b), x, tol=1e-6, maxiter=2000, inner_tol=1e-3,
                                cert_prec=cert)
        assert rep["rel_res"] <= 1e-6
        # the certified residual is the true one: recompute it with the oracle
        r = b - om.apply_A(m, to_host(x))
        assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.01e-6
        # relative error vs the FP64 oracle solution, bounded by cond * tol
        assert rel_err(to_host(x), xo) < 1e-4, (prec, rep)


@pytest.mark.parametrize("pc", [cw.CMBWS_BF16, cw.CMBWS_TF32, cw.CMBWS_FP64])
def test_solve_with_preconditioner_in_another_precision(models, pc):
    """The transforms of M_PI may run in their own arithmetic (here BF16 / TF32 tensor cores,
    or FP64) inside the solve of an FP32 model: the preconditioner only shapes the Krylov space,
    so the certified residual and the solution still reach the tolerance; cmbws_apply_precond
    keeps the model's own precision."""
    work, m, inp = models["multires64"]
    d = [mp + n for mp, n in zip(om.project(m, inp["x_true"]), inp["noise"])]
    b = om.rhs(m, d)
    xo, _ = pcg(lambda v: om.apply_A(m, v), b, lambda v: opc.apply_precond(m, v), tol=1e-12,
                maxiter=2000)
    g, _ = gpu_model(work, inp, cw.CMBWS_FP32)
    v = to_dev(np.random.default_rng(5).standard_normal(m.nvec()))
    z0, z1 = to_dev(np.zeros(m.nvec())), to_dev(np.zeros(m.nvec()))
    cw.cmbws_apply_precond(g, v, z0)
    cw.cmbws_model_set_precond_prec(g, pc)
    cw.cmbws_apply_precond(g, v, z1)
    assert np.array_equal(to_host(z0), to_host(z1))
    x = to_dev(np.zeros(m.nvec()))
    rep = cw.cmbws_cg_solve(g, to_dev(b), x, tol=1e-6, maxiter=2000, inner_tol=1e-3,
                            cert_prec=cw.CMBWS_FP64)
    assert rep["code"] == 0 and rep["rel_res"] <= 1e-6, rep
    r = b - om.apply_A(m, to_host(x))
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.01e-6
    assert rel_err(to_host(x), xo) < 1e-4, rep
    with pytest.raises(cw.CmbwsError) as e:
        cw.cmbws_model_set_precond_prec(g, 99)
    assert e.value.code == -1
    cw.cmbws_model_set_precond_prec(g, -1)


def test_multires_fp64_solve_matches_oracle_solution_to_1e6(models):
    """FP64 mode: the multi-resolution model at 1/16 of the benchmark's resolution (HEALPix
    Nside 16/32/64 bands, L_nu up to 191, three components) solved to a residual of 1e-10 lies
    within 1e-6 of the oracle's own solution (its FP64 PCG run to 1e-12)."""
    work, m, inp = models["multires16"]
    d = [mp + n for mp, n in zip(om.project(m, inp["x_true"]), inp["noise"])]
    b = om.rhs(m, d)
    xo, _ = pcg(lambda v: om.apply_A(m, v), b, lambda v: opc.apply_precond(m, v), tol=1e-12,
                maxiter=2000)
    g, _ = gpu_model(work, inp, cw.CMBWS_FP64)
    x = to_dev(np.zeros(m.nvec()))
    rep = cw.cmbws_cg_solve(g, to_dev(b), x, tol=1e-10, maxiter=2000)
    assert rep["rel_res"] <= 1e-10
    err = float(np.linalg.norm(to_host(x) - xo) / np.linalg.norm(xo))
    print(f"multires FP64 solve: {rep['iters']} iterations, |x - x_oracle| / |x_oracle| = {err:.2e}")
    assert err <= 1e-6
    assert rel_err(to_host(x), xo) <= 1e-6


def test_invalid_calls_return_error_codes(models):
    work, m, inp = models["tiny15"]
    g, grids = gpu_model(work, inp)
    x = to_dev(np.zeros(m.nvec()))
    with pytest.raises(cw.CmbwsError) as e:
        cw.cmbws_apply_A(g, x, x)
    assert e.value.code == -1
    with pytest.raises(cw.CmbwsError):
        cw.cmbws_plan_grid(cw.CMBWS_GRID_GL, 3, 10)       # fewer rings than lmax + 1
    # a component with neither prior nor data at some l is rejected (zero column of U)
    inp2 = dict(inp)
    inp2["cl"] = [None, None]
    inp2["beams"] = [np.where(np.arange(b.size) > 10, 0.0, b) for b in inp["beams"]]
    with pytest.raises(cw.CmbwsError) as e:
        gpu_model(work, inp2)
    assert e.value.code == -4
    # iteration cap -> NOT_CONVERGED with the report filled
    b = to_dev(np.random.default_rng(9).standard_normal(m.nvec()))
    rep = cw.cmbws_cg_solve(g, b, x, tol=1e-14, maxiter=2, check=False)
    assert rep["code"] == -6 and rep["iters"] == 2


def _variable_mixing_setup(L=15, Lmix=20, masked=True):
    """Tiny model whose dust pairs carry spatially variable mixing maps (max/min ~2) on GL
    mixing grids, with a galactic-band mask folded into the maps (Sec. 2.2, Sec. 4.1)."""
    from oracle import grids as og
    work = tiny_workload(L)
    m0, inp = oracle_model(work)
    g = og.gauss_legendre(Lmix)
    th, ph = g.pixel_angles()
    rng = np.random.default_rng(77)
    lm = [[None] * m0.ncomp for _ in range(m0.nobs)]
    maps = [[None] * m0.ncomp for _ in range(m0.nobs)]
    for nu in range(m0.nobs):
        k = 1  # dust
        s = 0.5 * (1 + np.cos(th) * rng.uniform(0.5, 1.0)) + 0.3 * np.sin(th) * np.cos(ph + nu)
        q = m0.q[nu, k] * (1.0 + s)
        if masked:
            q = np.where(np.abs(np.cos(th)) < np.sin(np.radians(20.0)), 0.0, q)
        lm[nu][k] = Lmix
        maps[nu][k] = q
    mg = [[g if maps[nu][k] is not None else None for k in range(m0.ncomp)] for nu in range(m0.nobs)]
    mo, _ = oracle_model(work, mix_maps=maps, mix_grids=mg)
    return work, mo, inp, (lm, maps)


@pytest.mark.parametrize("prec", PRECS)
def test_variable_mixing_operators_parity(prec):
    work, m, inp, mix = _variable_mixing_setup()
    g, _ = gpu_model(work, inp, prec, mix=mix)
    assert g.nsht_A == 2 * (2 * 3 + 3) and g.nsht_M == 2 * 3     # Nmix = 3, Nobs = 3
    rng = np.random.default_rng(5)
    x = rng.standard_normal(m.nvec())
    y = to_dev(np.zeros(m.nvec()))
    cw.cmbws_apply_A(g, to_dev(x), y)
    assert rel_err(to_host(y), om.apply_A(m, x)) < TOL[prec]
    z = to_dev(np.zeros(m.nvec()))
    cw.cmbws_apply_precond(g, to_dev(x), z)
    assert rel_err(to_host(z), opc.apply_precond(m, x)) < TOL[prec]
    d = [to_dev(np.zeros(gr.npix)) for gr in m.grids]
    cw.cmbws_project(g, to_dev(x), d)
    ref = om.project(m, x)
    for nu in range(m.nobs):
        assert rel_err(to_host(d[nu]), ref[nu]) < TOL[prec]


def test_variable_mixing_rhs_and_solve():
    work, m, inp, mix = _variable_mixing_setup()
    g, _ = gpu_model(work, inp, cw.CMBWS_FP32, mix=mix)
    d = [mp + n for mp, n in zip(om.project(m, inp["x_true"]), inp["noise"])]
    b = to_dev(np.zeros(m.nvec()))
    cw.cmbws_rhs(g, [to_dev(x) for x in d], b)
    bref = om.rhs(m, d)
    assert rel_err(to_host(b), bref) < 1e-10
    x = to_dev(np.zeros(m.nvec()))
    rep = cw.cmbws_cg_solve(g, to_dev(bref), x, tol=1e-8, maxiter=500, cert_prec=cw.CMBWS_FP32X2)
    assert rep["rel_res"] <= 1e-8
    r = bref - om.apply_A(m, to_host(x))
    assert np.linalg.norm(r) / np.linalg.norm(bref) <= 1.01e-8


def test_batched_solve_equals_sequential_solves():
    # independent uneven problems (GL L 12..40, galactic-band masks through the mixing maps),
    # solved concurrently and one by one: identical results (all reductions are deterministic)
    import skygen
    from oracle import grids as og
    probs = skygen.batched_uneven(nprob=6, lmin=12, lmax=40)
    models, bs, ms_o = [], [], []
    for work, f in probs:
        m, inp = oracle_model(work)
        L = work.bands[0].lmax
        g = og.gauss_legendre(L)
        z = np.cos(g.pixel_angles()[0])
        mask = skygen.galactic_mask(z, f)
        maps = [[m.q[nu, k] * mask for k in range(m.ncomp)] for nu in range(m.nobs)]
        lm = [[L] * m.ncomp for _ in range(m.nobs)]
        gm, _ = gpu_model(work, inp, cw.CMBWS_FP32, mix=(lm, maps))
        b = om.rhs(m, [mp + n for mp, n in zip(om.project(m, inp["x_true"]), inp["noise"])])
        models.append(gm)
        bs.append(to_dev(b))
        ms_o.append((m, b))
    xs = [to_dev(np.zeros(g.nvec)) for g in models]
    reps = cw.cmbws_cg_solve_batched(models, bs, xs, tol=1e-6, maxiter=3000,
                                     cert_prec=cw.CMBWS_FP32X2, nworkers=4)
    assert all(r["status"] == 0 and r["rel_res"] <= 1e-6 for r in reps)
    for i, g in enumerate(models):
        xi = to_dev(np.zeros(g.nvec))
        r1 = cw.cmbws_cg_solve(g, bs[i], xi, tol=1e-6, maxiter=3000, cert_prec=cw.CMBWS_FP32X2)
        np.testing.assert_array_equal(to_host(xi), to_host(xs[i]))
        assert r1["iters"] == reps[i]["iters"]
    # the first problem's certified residual, recomputed by the oracle
    m, b = ms_o[0]
    mg = [[og.gauss_legendre(m.lmax_band[0])] * m.ncomp for _ in range(m.nobs)]
    z = np.cos(mg[0][0].pixel_angles()[0])
    mask = skygen.galactic_mask(z, probs[0][1])
    mo, _ = oracle_model(probs[0][0], mix_maps=[[m.q[nu, k] * mask for k in range(m.ncomp)]
                                                 for nu in range(m.nobs)], mix_grids=mg)
    r = b - om.apply_A(mo, to_host(xs[0]))
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.01e-6
