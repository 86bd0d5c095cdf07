"""Band-sharded operators and solve (GPU): two processes on one GPU, each with the same model
description and half of the bands (one of them the prior), summing their partial outputs with
a gloo all-reduce of host copies.  The processes meet only on the host (their kernels never
wait on each other).  The summed partial A x, M_PI r and b equal the one-process results, and
the sharded PCG reaches the unsharded solution."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import datetime

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    try:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(0)
        dist.init_process_group("gloo", rank=rank, world_size=world,
                                timeout=datetime.timedelta(seconds=60))
        import paper_1710_00621_gb300 as cw
        from paper_1710_00621_gb300 import sharding
        from oracle import model as om
        from tests._gpu import gpu_model, to_dev, to_host
        from tests._models import multires_small, oracle_model

        work = multires_small(64)
        m, inp = oracle_model(work)
        g, grids = gpu_model(work, inp, cw.CMBWS_FP64)
        n, nobs = m.nvec(), m.nobs
        keys = [(b.grid, b.n, b.lmax) for b in work.bands]
        costs = [(2 * b.n) * (b.lmax + 1) ** 2 for b in work.bands]
        owned = sharding.assign_bands(keys, costs, world)[rank]
        rng = np.random.default_rng(5)
        x = rng.standard_normal(n)
        d = [mp_ + e for mp_, e in zip(om.project(m, inp["x_true"]), inp["noise"])]
        dd = [to_dev(v) for v in d]

        def summed(fn):
            out = to_dev(np.zeros(n))
            fn(out)
            h = out.cpu()
            dist.all_reduce(h)
            return h.numpy()

        full_A = to_dev(np.zeros(n))
        cw.cmbws_apply_A(g, to_dev(x), full_A)
        full_M = to_dev(np.zeros(n))
        cw.cmbws_apply_precond(g, to_dev(x), full_M)
        full_b = to_dev(np.zeros(n))
        cw.cmbws_rhs(g, dd, full_b)
        sharding.set_shard(g, owned, nobs, prior=1 if rank == 0 else 0)
        sA = summed(lambda o: cw.cmbws_apply_A(g, to_dev(x), o))
        sM = summed(lambda o: cw.cmbws_apply_precond(g, to_dev(x), o))
        sb = summed(lambda o: cw.cmbws_rhs(g, dd, o))

        def rel(a, b):
            return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))

        errs = {"A": rel(sA, to_host(full_A)), "M": rel(sM, to_host(full_M)),
                "b": rel(sb, to_host(full_b))}
        # a plain solve refuses the sharded model
        try:
            cw.cmbws_cg_solve(g, full_b, to_dev(np.zeros(n)), tol=1e-8)
            errs["refused"] = False
        except cw.CmbwsError as e:
            errs["refused"] = e.code == -1
        # the sharded PCG against the one-process solution
        xs = to_dev(np.zeros(n))
        rep = sharding.cg_solve_sharded(g, full_b, xs, tol=1e-10, maxiter=500)
        sharding.set_shard(g, None, nobs, prior=1)
        x1 = to_dev(np.zeros(n))
        rep1 = cw.cmbws_cg_solve(g, full_b, x1, tol=1e-10, maxiter=500)
        errs["x"] = rel(to_host(xs), to_host(x1))
        errs["iters"] = (rep["iters"], rep1["iters"])
        errs["rel_res"] = rep["rel_res"]
        q.put((rank, "ok", errs))
        dist.destroy_process_group()
    except Exception as e:  # noqa: BLE001 - reported to the parent
        q.put((rank, "err", repr(e)[:500]))


def test_two_shards_sum_to_the_full_operators_and_solve():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = {}
    for _ in range(2):
        r, status, v = q.get(timeout=600)
        out[r] = (status, v)
    for p in ps:
        p.join(timeout=120)
        if p.is_alive():
            p.kill()
    for r in range(2):
        status, e = out[r]
        assert status == "ok", e
        # partial sums in another order than the one-process kernels: rounding level
        assert e["A"] < 1e-12 and e["M"] < 1e-12 and e["b"] < 1e-12, e
        assert e["refused"], e
        assert e["rel_res"] <= 1e-10 and e["x"] < 1e-8, e
        assert abs(e["iters"][0] - e["iters"][1]) <= 2, e
    # both shards hold the same solution path
    assert out[0][1]["x"] == out[1][1]["x"] and out[0][1]["iters"] == out[1][1]["iters"]
