"""GPU parity of observation merging in the preconditioner (cmbws_model_merge_precond,
App. A.3) against oracle/merge.py."""
import numpy as np
import pytest

from oracle import merge as omerge
from oracle import precond as opc
from tests._gpu import GridCache, rel_err, to_dev, to_host
from tests._models import multires_small, oracle_model, split_model, tiny_workload

pytestmark = pytest.mark.gpu


def _gpu_split(work, m, nb, prec):
    """Library model of an oracle split model: band nu is a subset of work band nu // nb and
    uses that band's grid handle."""
    import paper_1710_00621_gb300 as cw
    cache = GridCache()
    grids = [cache.get(work.bands[nu // nb]) for nu in range(m.nobs)]
    gm = cw.cmbws_model_create(list(m.lmax_comp), grids, m.beam, m.cl,
                               [to_dev(t) for t in m.tau], np.asarray(m.q), prec)
    return gm, grids


def _apply(gm, r):
    import paper_1710_00621_gb300 as cw
    import torch
    z = torch.zeros(len(r), dtype=torch.float64, device="cuda")
    cw.cmbws_apply_precond(gm, to_dev(r), z)
    return to_host(z)


def _compromise(m):
    """Subsets that are only similar: another noise pattern, beam and mixing for band 1."""
    th, _ = m.grids[1].pixel_angles()
    m.tau[1] = m.tau[1] * (1.0 + 0.3 * np.cos(th))
    m.beam[1] = m.beam[1] ** 1.2
    q = np.array(m.q, dtype=np.float64)
    q[1] *= np.array([1.0, 1.15])
    m.q = q
    return m


@pytest.mark.parametrize("case", ["tiny_exact", "tiny_compromise", "multires_exact"])
def test_merged_precond_parity(case):
    import paper_1710_00621_gb300 as cw
    work = multires_small(64) if case == "multires_exact" else tiny_workload(15)
    m0, _ = oracle_model(work)
    fr = (0.25, 0.25, 0.5) if case == "multires_exact" else (0.3, 0.7)
    m, groups = split_model(m0, fr)
    if case == "tiny_compromise":
        m = _compromise(m)
    group = [g for g, G in enumerate(groups) for _ in G]
    r = np.random.default_rng(7).standard_normal(m.nvec())
    ref = omerge.apply_merged_precond(m, groups, r)
    for prec, tol in ((cw.CMBWS_FP64, 1e-10), (cw.CMBWS_FP32, 1e-4)):
        gm, _ = _gpu_split(work, m, len(fr), prec)
        unmerged = _apply(gm, r)
        assert gm.nsht_M == 2 * m.nobs
        cw.cmbws_model_merge_precond(gm, group)
        assert gm.nsht_M == 2 * len(groups)
        got = _apply(gm, r)
        assert rel_err(got, ref) < tol, (prec, rel_err(got, ref))
        if case.endswith("exact"):
            # exact splits: the merged preconditioner is M_PI itself
            assert rel_err(got, unmerged) < tol
            assert rel_err(unmerged, opc.apply_precond(m, r)) < tol
        cw.cmbws_model_merge_precond(gm, None)
        assert gm.nsht_M == 2 * m.nobs
        assert np.array_equal(_apply(gm, r), unmerged)


def test_merged_solve_same_iterations_fewer_shts():
    import paper_1710_00621_gb300 as cw
    import torch
    from oracle import model as omodel
    work = multires_small(32)
    m0, inp = oracle_model(work)
    m, groups = split_model(m0, (0.5, 0.5))
    gm, _ = _gpu_split(work, m, 2, cw.CMBWS_FP64)
    b = to_dev(omodel.apply_A(m, inp["x_true"]))
    res = {}
    for name, group in (("per_band", None), ("merged", [nu // 2 for nu in range(m.nobs)])):
        cw.cmbws_model_merge_precond(gm, group)
        x = torch.zeros_like(b)
        rep = cw.cmbws_cg_solve(gm, b, x, tol=1e-8, maxiter=2000, precond=1)
        assert rep["rel_res"] <= 1e-8
        assert rel_err(to_host(x), inp["x_true"]) < 1e-5
        res[name] = rep
    assert abs(res["merged"]["iters"] - res["per_band"]["iters"]) <= 1, res
    assert res["merged"]["n_sht"] < res["per_band"]["n_sht"]


def test_merge_errors():
    import paper_1710_00621_gb300 as cw
    work = multires_small(64)
    m0, _ = oracle_model(work)
    m, groups = split_model(m0, (0.5, 0.5))
    gm, _ = _gpu_split(work, m, 2, cw.CMBWS_FP64)
    n = m.nobs
    ok = [nu // 2 for nu in range(n)]
    bad_range = list(ok)
    bad_range[0] = n
    unused = [g + 1 for g in ok]                       # id 0 unused
    mixed = list(ok)
    mixed[0], mixed[-1] = mixed[-1], mixed[0]          # Nside 64 and Nside 16 bands in one row
    for group in (bad_range, unused, mixed, [-1] + ok[1:]):
        with pytest.raises(cw.CmbwsError):
            cw.cmbws_model_merge_precond(gm, group)
    assert gm.nsht_M == 2 * n                          # a failed call leaves the model as it was
    cw.cmbws_model_merge_precond(gm, ok)
    assert gm.nsht_M == n
