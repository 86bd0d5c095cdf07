"""GPU parity of the mask-restricted multigrid preconditioner (cmbws_model_add_mask_precond,
cmbws_apply_M_add, precond = 2) against the oracle (oracle/maskmg.py)."""
import numpy as np
import pytest

from oracle import cg as ocg
from oracle import maskmg as omg
from oracle import model as omodel
from oracle import precond as oprec
from tests._gpu import rel_err, to_dev, to_host
from tests.test_oracle_maskmg import _masked_model

pytestmark = pytest.mark.gpu


def _gpu_masked(m, inp, mask, prec, nside=8, L=23, max_bottom=60):
    import paper_1710_00621_gb300 as cw
    grids = [cw.cmbws_plan_grid(cw.CMBWS_GRID_HEALPIX, nside, L) for _ in range(3)]
    mg = cw.cmbws_plan_grid(cw.CMBWS_GRID_HEALPIX, nside, L)
    maps = [[to_dev(m.mix_map[nu][0])] for nu in range(3)]
    gm = cw.cmbws_model_create([L], grids, inp["beams"], inp["cl"], [to_dev(t) for t in m.tau],
                               inp["q"], prec, mix_grids=[[mg]] * 3, mix_maps=maps)
    cw.cmbws_model_add_mask_precond(gm, 0, nside, to_dev(mask.astype(np.float64)), max_bottom)
    return gm, (grids, mg, maps)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_M_mask_parity(prec):
    import paper_1710_00621_gb300 as cw
    import torch
    m, inp, mask = _masked_model()
    mp = omg.MaskPrecond(m, 0, 8, mask, max_bottom=60)
    p = cw.CMBWS_FP64 if prec == "fp64" else cw.CMBWS_FP32
    gm, keep = _gpu_masked(m, inp, mask, p)
    rng = np.random.default_rng(4)
    r = rng.standard_normal(m.nvec())
    zadd = torch.empty(m.nvec(), dtype=torch.float64, device="cuda")
    zpi = torch.empty_like(zadd)
    cw.cmbws_apply_M_add(gm, to_dev(r), zadd)
    cw.cmbws_apply_precond(gm, to_dev(r), zpi)
    got = to_host(zadd - zpi)
    ref = mp.apply(m, r)
    # the bottom pseudo-inverses (Jacobi SVD here, eigen-decomposition in the oracle, both cut
    # at 1e-5) agree to eps x 1e5; FP32 transforms add ~1e-5 per level, amplified by <= 1e5
    # only in the weakest kept directions
    assert rel_err(got, ref) < (1e-9 if prec == "fp64" else 2e-3), rel_err(got, ref)


def test_masked_solve_with_M_add():
    import paper_1710_00621_gb300 as cw
    import torch
    m, inp, mask = _masked_model()
    gm, keep = _gpu_masked(m, inp, mask, cw.CMBWS_FP64)
    b = omodel.apply_A(m, inp["x_true"])
    x_ref = np.linalg.solve(omodel.dense_A(m), b)
    its = {}
    for pc in (1, 2):
        x = torch.zeros(m.nvec(), dtype=torch.float64, device="cuda")
        rep = cw.cmbws_cg_solve(gm, to_dev(b), x, tol=1e-8, maxiter=3000, precond=pc)
        its[pc] = rep["iters"]
        assert rep["rel_res"] <= 1e-8
        assert rel_err(to_host(x), x_ref) < 1e-6
    mp = omg.MaskPrecond(m, 0, 8, mask, max_bottom=60)
    Up = oprec.pinv_blocks(oprec.U_blocks(m))
    _, rep_o = ocg.pcg(lambda v: omodel.apply_A(m, v), b,
                       apply_M=lambda v: omg.apply_M_add(m, [mp], v, Up), tol=1e-8, maxiter=3000)
    assert its[2] <= rep_o["iters"] + 2, (its, rep_o["iters"])
    assert its[2] * 2 <= its[1], its


def test_masked_solve_fp32_certified():
    import paper_1710_00621_gb300 as cw
    import torch
    m, inp, mask = _masked_model()
    gm, keep = _gpu_masked(m, inp, mask, cw.CMBWS_FP32)
    b = omodel.apply_A(m, inp["x_true"])
    x = torch.zeros(m.nvec(), dtype=torch.float64, device="cuda")
    rep = cw.cmbws_cg_solve(gm, to_dev(b), x, tol=1e-6, maxiter=3000, precond=2,
                            cert_prec=cw.CMBWS_FP32X2)
    assert rep["status"] == 0 and rep["rel_res"] <= 1e-6
    assert rel_err(to_host(x), inp["x_true"]) < 1e-4


def test_mask_precond_needs_a_prior():
    import paper_1710_00621_gb300 as cw
    m, inp, mask = _masked_model(nside=4, L=11)
    grids = [cw.cmbws_plan_grid(cw.CMBWS_GRID_HEALPIX, 4, 11) for _ in range(3)]
    gm = cw.cmbws_model_create([11], grids, inp["beams"], [None], [to_dev(t) for t in m.tau],
                               inp["q"], cw.CMBWS_FP64)
    with pytest.raises(cw.CmbwsError):
        cw.cmbws_model_add_mask_precond(gm, 0, 4, to_dev(mask.astype(np.float64)), 60)


def test_masked_constrained_realization_fp32_matches_fp64():
    """The masked CR workload (4 components, 9 bands, band + disks mask in all 36 mixing maps,
    omega_1 / omega_2 right-hand side) at reduced size: the FP32-refined solution with M_add
    agrees with the FP64 one, both certified, and M_PI alone needs more iterations."""
    import bench
    out = bench.masked_cr_measure(tol=1e-8, scale=8, max_bottom=100)
    assert out["fp32"]["certified"] and out["fp64"]["certified"], out
    # two solutions certified to 1e-8 in residual differ by at most ~cond x 1e-8
    assert out["fp32_vs_fp64_rel_diff"] < 1e-5, out
    assert out["M_PI_alone_fp32"]["iters"] > out["fp32"]["iters"], out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_M_mask_parity_optimized_vcycle(prec):
    """The optimized V-cycle (J ~ I, 6 SHTs per level) against the oracle's."""
    import paper_1710_00621_gb300 as cw
    import torch
    m, inp, mask = _masked_model()
    mp = omg.MaskPrecond(m, 0, 8, mask, max_bottom=60, cycle="optimized")
    p = cw.CMBWS_FP64 if prec == "fp64" else cw.CMBWS_FP32
    gm, keep = _gpu_masked(m, inp, mask, p)
    cw.cmbws_model_set_vcycle(gm, cw.CMBWS_VCYCLE_OPTIMIZED)
    r = np.random.default_rng(5).standard_normal(m.nvec())
    zadd = torch.empty(m.nvec(), dtype=torch.float64, device="cuda")
    zpi = torch.empty_like(zadd)
    cw.cmbws_apply_M_add(gm, to_dev(r), zadd)
    cw.cmbws_apply_precond(gm, to_dev(r), zpi)
    got = to_host(zadd - zpi)
    assert rel_err(got, mp.apply(m, r)) < (1e-9 if prec == "fp64" else 2e-3), rel_err(got, mp.apply(m, r))
    # and it is a different operator from the basic cycle
    basic = omg.MaskPrecond(m, 0, 8, mask, max_bottom=60).apply(m, r)
    assert rel_err(got, basic) > 1e-6


def test_masked_solve_optimized_vcycle_fewer_shts():
    import paper_1710_00621_gb300 as cw
    import torch
    m, inp, mask = _masked_model()
    gm, keep = _gpu_masked(m, inp, mask, cw.CMBWS_FP64)
    b = to_dev(omodel.apply_A(m, inp["x_true"]))
    reps = {}
    for kind in (cw.CMBWS_VCYCLE_BASIC, cw.CMBWS_VCYCLE_OPTIMIZED):
        cw.cmbws_model_set_vcycle(gm, kind)
        x = torch.zeros_like(b)
        rep = cw.cmbws_cg_solve(gm, b, x, tol=1e-8, maxiter=3000, precond=2)
        assert rep["rel_res"] <= 1e-8
        assert rel_err(to_host(x), inp["x_true"]) < 1e-5
        reps[kind] = rep
    ib, io = reps[0]["iters"], reps[1]["iters"]
    assert io <= 1.5 * ib + 2, (ib, io)
    assert reps[1]["n_sht"] / io < reps[0]["n_sht"] / ib
    with pytest.raises(cw.CmbwsError):
        cw.cmbws_model_set_vcycle(gm, 2)
