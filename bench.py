"""Benchmark: Wiener-filter solve time to a certified 1e-6 residual on GB300.

Workload (default): the multi-resolution full-sky model -- Ncomp = 3 (CMB L 2000,
synchrotron beta -3.0 L 500, dust beta 1.6 L 3000), Nobs = 9 HEALPix bands at Nside
256/512/1024 (L_nu = 3 Nside - 1), Gaussian beams 33' -> 5', noise rms varying x3 over
the sky -- with seeded synthetic inputs (skygen).  One step is one Wiener filter from the
band maps d: b = P^T N^-1 d (cmbws_rhs), then PCG with M_PI (cmbws_cg_solve) until
||b - A x|| / ||b|| <= 1e-6, certified by an FP64 apply of A.  The default arithmetic is
FP32 transforms with FP64 vectors, scalars and iterative refinement; --prec fp64 runs the
plain FP64 solver.  One plain FP64 solve is also timed once and reported as fp64_plain.

Timing: W untimed warm-up steps, then K steps bracketed by a barrier and a device
synchronise on both sides, CUDA events on the launching stream, max over ranks.  Inputs
(band maps 0.4 GB, vectors 0.1 GB each, tables) exceed the 129 MB L2, so no flush is done.
The library's kernel-timing records (CUDA events on the launching stream) give the per-stage
time and the roofline of the dominant kernel.  --gpus N runs N independent replicas (one
per rank) and reports the max time over ranks; there is no data-path collective.

--impl reference times the FP64 NumPy oracle on every host core on a bounded sample (one
SHT pair of the Nside-192 grid per core) and scales it to the same solve, with the
oracle's own PCG iteration count (measured on the model at 1/16 resolution).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import skygen  # noqa: E402

SEED_CR = skygen.SEED_BASE + 3
SEED_SPLIT = skygen.SEED_BASE + 5
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # FP32 FMA lanes x 2 flops x max SM clock
FP64_PEAK_TFLOPS = 1.25                               # GB300 FP64 (profiling recipe, nominal)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--scale", type=int, default=1, help="divide Nside and band-limits (debug)")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--no-fp64-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--precond-prec", choices=["model", "bf16", "tf32", "fp32"], default="bf16",
                    help="arithmetic of the M_PI transforms of the FP32 solve (model: the model's own)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the tiny-problem and differentiable-solve measurements")
    ap.add_argument("--no-masked-cr", action="store_true",
                    help="skip the masked constrained-realization solve (FP32 vs FP64, M_add)")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the per-precision synthesis time / error report")
    ap.add_argument("--inner-tol", type=float, default=1e-3,
                    help="relative residual reduction per refinement pass (FP32 solves)")
    ap.add_argument("--with-batched", type=int, default=64, metavar="NPROB",
                    help="also time NPROB independent uneven masked problems (GL L 128..1024), "
                         "batched vs sequential, reported under 'batched'")
    ap.add_argument("--autotune", type=int, default=2, choices=[0, 1, 2],
                    help="synthesis tiles: 0 default, 1 heuristic, 2 measured on first use")
    ap.add_argument("--cert", default="fp32x2", choices=["fp32x2", "fp64"],
                    help="arithmetic of the FP64-accurate residual applies of the mixed solve")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def workload(scale):
    return skygen.multires_fullsky(scale=scale)


def dist_init(n):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    """Maximum of a per-rank value over all ranks (NCCL on GPUs, gloo on the host)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def build_problem(work, prec, seed_offset=0):
    """Library grids, seeded inputs, model and band maps d = P x_true + n on the device."""
    import torch
    import paper_1710_00621_gb300 as cw
    grids = {}
    band_grids = []
    for b in work.bands:
        key = (b.grid, b.n, b.lmax)
        if key not in grids:
            kind = cw.CMBWS_GRID_GL if b.grid == "gl" else cw.CMBWS_GRID_HEALPIX
            grids[key] = cw.cmbws_plan_grid(kind, b.n + 1 if b.grid == "gl" else b.n, b.lmax)
        band_grids.append(grids[key])
    coords = [g.pixel_coords() for g in band_grids]
    weights = [g.pixel_weights() for g in band_grids]
    work.seed += seed_offset
    inp = skygen.make_inputs(work, coords, weights)
    dev = torch.device("cuda")
    ninv = [torch.as_tensor(t, device=dev) for t in inp["tau"]]
    lk = [c.lmax for c in work.comps]
    m64 = cw.cmbws_model_create(lk, band_grids, inp["beams"], inp["cl"], ninv, inp["q"], cw.CMBWS_FP64)
    m_run = m64 if prec == "fp64" else cw.cmbws_model_create(lk, band_grids, inp["beams"], inp["cl"],
                                                              ninv, inp["q"], cw.CMBWS_FP32)
    x_true = torch.as_tensor(inp["x_true"], device=dev)
    d = [torch.empty(g.npix, dtype=torch.float64, device=dev) for g in band_grids]
    cw.cmbws_project(m64, x_true, d)
    for nu in range(len(d)):
        d[nu] += torch.as_tensor(inp["noise"][nu], device=dev)
    torch.cuda.synchronize()
    return dict(grids=band_grids, inp=inp, m64=m64, model=m_run, d=d, x_true=x_true, ninv=ninv)


INNER_TOL = [1e-3]


def solve_step(P, model, tol, x, b, cert="fp32x2"):
    import paper_1710_00621_gb300 as cw
    cw.cmbws_rhs(model, P["d"], b)
    x.zero_()
    cp = cw.CMBWS_FP32X2 if cert == "fp32x2" else cw.CMBWS_FP64
    return cw.cmbws_cg_solve(model, b, x, tol=tol, maxiter=3000, precond=1,
                             inner_tol=INNER_TOL[0], max_outer=30, cert_prec=cp)


def cr_chain_measure(model, P, xmean, tol, inner_tol, cert, nsamp=3):
    """A chain of constrained realizations (Sec. 2.3) on the bench model: omega_1, omega_2
    drawn on the device (cmbws_cr_sample), each solve started from zero, from the previous
    sample, or from the Wiener-filter mean xmean."""
    import torch
    import paper_1710_00621_gb300 as cw
    cp = cw.CMBWS_FP32X2 if cert == "fp32x2" else cw.CMBWS_FP64
    kw = dict(tol=tol, maxiter=3000, precond=1, inner_tol=inner_tol, max_outer=20,
              cert_prec=cp, timeout_s=120.0, check=False)
    xs = torch.zeros_like(xmean)
    res = {}
    for start in ("zero", "previous", "mean"):
        its, secs, ok = [], [], []
        xs.zero_()
        for s in range(nsamp):
            if start == "zero":
                xs.zero_()
            elif start == "mean":
                xs.copy_(xmean)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = cw.cmbws_cr_sample(model, P["d"], SEED_CR, s, xs, **kw)
            torch.cuda.synchronize()
            secs.append(round(time.perf_counter() - t0, 3))
            its.append(r["iters"])
            ok.append(r["status"] == 0)
        res[start] = {"s": secs, "iters": its, "certified": all(ok)}
    b2 = torch.empty_like(xmean)
    cw.cmbws_cr_rhs(model, P["d"], SEED_CR, nsamp, b2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cw.cmbws_cr_rhs(model, P["d"], SEED_CR, nsamp + 1, b2)
    torch.cuda.synchronize()
    t_rhs = time.perf_counter() - t0
    return {"samples": nsamp, "start": res, "draw_and_rhs_s": round(t_rhs, 4),
            "note": ("constrained realizations with on-device Philox4x64-10 / Box-Muller "
                     "variates; 'previous' starts each solve from the chain's last sample "
                     "(the first from zero)")}


def split_measure(P, xref, tol, inner_tol, cert):
    """Detector splits (App. A.3): every band of the bench model as two half-hit subsets,
    inverse noise tau / 2 each and data d + e, d - e with e ~ N(0, 1 / tau), so each half has
    noise variance 2 / tau, the halves are independent and their mean is d.  The 18-band
    system has the same A and b as the 9-band one; it is solved with one preconditioner row
    per band (36 SHTs per apply of M_PI) and with the halves merged (18)."""
    import torch
    import paper_1710_00621_gb300 as cw
    inp, grids = P["inp"], P["grids"]
    dev = torch.device("cuda")
    gen = torch.Generator(device=dev)
    gen.manual_seed(SEED_SPLIT)
    ninv, d2, grids2, beams2 = [], [], [], []
    for nu, t in enumerate(inp["tau"]):
        tau = torch.as_tensor(t, device=dev)
        e = torch.randn(tau.shape, generator=gen, device=dev, dtype=torch.float64) / torch.sqrt(tau)
        for sgn in (1.0, -1.0):
            ninv.append(0.5 * tau)
            d2.append(P["d"][nu] + sgn * e)
            grids2.append(grids[nu])
            beams2.append(inp["beams"][nu])
    q2 = np.repeat(np.asarray(inp["q"], dtype=np.float64), 2, axis=0)
    lk = list(P["model"].lmax_comp)
    model = cw.cmbws_model_create(lk, grids2, beams2, inp["cl"], ninv, q2, cw.CMBWS_FP32)
    cp = cw.CMBWS_FP32X2 if cert == "fp32x2" else cw.CMBWS_FP64
    kw = dict(tol=tol, maxiter=3000, precond=1, inner_tol=inner_tol, max_outer=20,
              cert_prec=cp, timeout_s=120.0, check=False)
    b = torch.zeros_like(xref)
    x = torch.zeros_like(xref)
    out = {"bands": len(d2)}
    try:
        for name, group in (("per_band", None), ("merged", [nu // 2 for nu in range(len(d2))])):
            cw.cmbws_model_merge_precond(model, group)
            cw.cmbws_rhs(model, d2, b)
            for _ in range(2):          # the first solve allocates the model's workspaces
                x.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = cw.cmbws_cg_solve(model, b, x, **kw)
                torch.cuda.synchronize()
                ts = time.perf_counter() - t0
            diff = float(torch.linalg.vector_norm(x - xref) / torch.linalg.vector_norm(xref))
            out[name] = {"s": round(ts, 3), "iters": r["iters"], "outer": r["outer"],
                         "certified": r["status"] == 0, "n_sht": r["n_sht"],
                         "nsht_M": model.nsht_M, "rel_diff_vs_9_band_solution": diff}
    finally:
        model.close()
    out["note"] = ("each band split into two half-hit detector subsets; merged = App. A.3 "
                   "row merge in the preconditioner")
    return out


def batched_measure(nprob, tol, fmax=0.3, max_bottom=200):
    """Independent uneven problems (Ncomp 2, Nobs 3, GL bands L_p ~ U{128..1024}) with a
    galactic-band mask of sky fraction U[0, fmax] carried by the mixing maps on a HEALPix
    mixing grid (Nside_p: the smallest power of two with 3 Nside_p - 1 >= L_p), solved with
    M_add = M_PI + the mask-restricted multigrid preconditioner of each component: one
    cmbws_cg_solve_batched call vs the same solves one after the other.  Every solve has a
    wall-clock budget; progress goes to stderr."""
    import torch
    import paper_1710_00621_gb300 as cw
    dev = torch.device("cuda")
    models, bs, masked = [], [], []
    keep = []
    t_setup = time.perf_counter()
    for work, f in skygen.batched_uneven(nprob=nprob, fmax=fmax):
        L = work.bands[0].lmax
        g = cw.cmbws_plan_grid(cw.CMBWS_GRID_GL, L + 1, L)
        z, ph = g.pixel_coords()
        w = g.pixel_weights()
        inp = skygen.make_inputs(work, [(z, ph)] * 3, [w] * 3)
        q = inp["q"]
        ninv = [torch.as_tensor(t, device=dev) for t in inp["tau"]]
        mg = maps = mask = None
        nside = 1
        while 3 * nside - 1 < L:
            nside *= 2
        if f > 0:
            hg = cw.cmbws_plan_grid(cw.CMBWS_GRID_HEALPIX, nside, L)
            hz, _ = hg.pixel_coords()
            inside = 1.0 - skygen.galactic_mask(hz, f)          # 1 inside the band |b| < b0
            mask = torch.as_tensor(inside, device=dev)
            keepmap = torch.as_tensor(1.0 - inside, device=dev)
            maps = [[float(q[nu, k]) * keepmap for k in range(2)] for nu in range(3)]
            mg = [[hg, hg]] * 3
        m = cw.cmbws_model_create([c.lmax for c in work.comps], [g] * 3, inp["beams"], inp["cl"],
                                  ninv, q, cw.CMBWS_FP32, mix_grids=mg, mix_maps=maps)
        npx = float(mask.sum()) if mask is not None else 0.0
        if npx > 0:
            for k in range(2):
                cw.cmbws_model_add_mask_precond(m, k, nside, mask, max_bottom)
        x_true = torch.as_tensor(inp["x_true"], device=dev)
        d = [torch.empty(g.npix, dtype=torch.float64, device=dev) for _ in range(3)]
        cw.cmbws_project(m, x_true, d)
        for nu in range(3):
            d[nu] += torch.as_tensor(inp["noise"][nu], device=dev)
        b = torch.empty(m.nvec, dtype=torch.float64, device=dev)
        cw.cmbws_rhs(m, d, b)
        models.append(m)
        bs.append(b)
        masked.append(npx)
        keep.append((g, maps, ninv, mask, mg))
        print(f"[batched] setup L={L} f={f:.3f} nside={nside}", file=sys.stderr, flush=True)
    t_setup = time.perf_counter() - t_setup
    xs = [torch.zeros(m.nvec, dtype=torch.float64, device=dev) for m in models]
    kw = dict(tol=tol, maxiter=3000, cert_prec=cw.CMBWS_FP32X2, inner_tol=1e-3, max_outer=10,
              precond=2, timeout_s=60.0)
    cw.cmbws_cg_solve_batched(models, bs, xs, check=False, **kw)   # warm-up (workspaces)
    torch.cuda.synchronize()
    print("[batched] warm-up done", file=sys.stderr, flush=True)
    for x in xs:
        x.zero_()
    t0 = time.perf_counter()
    reps = cw.cmbws_cg_solve_batched(models, bs, xs, check=False, **kw)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    t0 = time.perf_counter()
    for i, m in enumerate(models):
        xs[i].zero_()
        cw.cmbws_cg_solve(m, bs[i], xs[i], check=False, **kw)
    torch.cuda.synchronize()
    tseq = time.perf_counter() - t0
    print("[batched] timed solves done", file=sys.stderr, flush=True)
    # the batched solves again with every operator apply replayed from a CUDA graph
    x_eager = [x.clone() for x in xs]
    for m in models:
        cw.cmbws_model_set_graphs(m, True)
    for x in xs:
        x.zero_()
    cw.cmbws_cg_solve_batched(models, bs, xs, check=False, **kw)   # captures the graphs
    torch.cuda.synchronize()
    for x in xs:
        x.zero_()
    t0 = time.perf_counter()
    reps_g = cw.cmbws_cg_solve_batched(models, bs, xs, check=False, **kw)
    torch.cuda.synchronize()
    tbg = time.perf_counter() - t0
    same = all(bool(torch.equal(a, c)) for a, c in zip(xs, x_eager))
    for m in models:
        cw.cmbws_model_set_graphs(m, False)
    print("[batched] graph-replayed solves done", file=sys.stderr, flush=True)
    # the same masked problems with M_PI alone, on the three largest masks (budget-bounded)
    big = sorted(range(len(models)), key=lambda i: -masked[i])[:3]
    cmp = []
    for i in big:
        x = torch.zeros_like(xs[i])
        r1 = cw.cmbws_cg_solve(models[i], bs[i], x, check=False,
                               **{**kw, "precond": 1, "maxiter": 1000, "timeout_s": 20.0})
        cmp.append({"L": int(models[i].lmax_comp[0]), "iters_M_PI": r1["iters"],
                    "M_PI_certified": r1["status"] == 0, "iters_M_add": reps[i]["iters"]})
    its = [r["iters"] for r in reps]
    return {"nprob": nprob, "batched_s": round(tb, 3), "sequential_s": round(tseq, 3),
            "speedup": round(tseq / tb, 2),
            "batched_graphs_s": round(tbg, 3), "speedup_graphs_vs_sequential": round(tseq / tbg, 2),
            "graphs_bitwise_equal_to_eager": same,
            "graphs_all_certified": all(r["status"] == 0 and r["rel_res"] <= tol for r in reps_g),
            "iters_min_median_max": [min(its), int(np.median(its)), max(its)],
            "all_certified": all(r["status"] == 0 and r["rel_res"] <= tol for r in reps),
            "n_certified": sum(r["status"] == 0 and r["rel_res"] <= tol for r in reps),
            "setup_s": round(t_setup, 1), "M_PI_vs_M_add_largest_masks": cmp,
            "workload": (f"GL L 128..1024 with resolution-matched beams, Ncomp 2, Nobs 3, galactic-"
                         f"band masks of sky fraction U[0, {fmax}] in HEALPix mixing maps, M_add = "
                         "M_PI + multigrid M_mask, FP32 transforms + FP32X2 certification, "
                         "8 worker streams")}


def variable_dust_measure(P, tol, inner_tol, cert, pc, iters_const):
    """The benchmark model's variant with spatially variable dust mixing (Eq. Q): the dust pair
    of every band (Nmix = 9) carries q(p) = q (1 + f(p)), f a seeded band-limited (l <= 8)
    field rescaled to [0, 1] (max / min = 2), on the Nside-1024 band grid (L 3071 >= L_dust)
    as the mixing grid.  Band maps d = P_var x_true + n; the step's solve (RHS, FP32 PCG with
    the same preconditioner arithmetic, certified refinement)."""
    import torch
    import paper_1710_00621_gb300 as cw
    dev = torch.device("cuda")
    inp, grids = P["inp"], P["grids"]
    lk = list(P["model"].lmax_comp)
    nb, nc = len(grids), len(lk)
    k = max(range(nc), key=lambda j: lk[j])      # the dust component (largest band-limit)
    mg = max(grids, key=lambda g: g.lmax)        # the Nside-1024 band grid
    z, ph = mg.pixel_coords()
    f = skygen.smooth_field(z, ph, np.random.default_rng(skygen.SEED_BASE + 7))
    q = np.asarray(inp["q"], dtype=np.float64)
    maps = [[torch.as_tensor(q[nu, k] * (1.0 + f), device=dev) if j == k else None
             for j in range(nc)] for nu in range(nb)]
    mgs = [[mg if j == k else None for j in range(nc)] for _ in range(nb)]
    m = cw.cmbws_model_create(lk, grids, inp["beams"], inp["cl"], P["ninv"], q, cw.CMBWS_FP32,
                              mix_grids=mgs, mix_maps=maps)
    try:
        cw.cmbws_model_set_precond_prec(m, pc)
        d = [torch.empty(g.npix, dtype=torch.float64, device=dev) for g in grids]
        cw.cmbws_project(m, P["x_true"], d)
        for nu in range(nb):
            d[nu] += torch.as_tensor(inp["noise"][nu], device=dev)
        b = torch.empty(m.nvec, dtype=torch.float64, device=dev)
        x = torch.zeros(m.nvec, dtype=torch.float64, device=dev)
        cp = cw.CMBWS_FP32X2 if cert == "fp32x2" else cw.CMBWS_FP64
        res = {}
        # M_PI, then the block-diagonal M_diag (the paper's comparison with variable dust maps)
        for name, pcm in (("M_PI", 1), ("M_diag", 3)):
            for _ in range(2):                      # the first solve allocates the workspaces
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                cw.cmbws_rhs(m, d, b)
                x.zero_()
                r = cw.cmbws_cg_solve(m, b, x, tol=tol, maxiter=3000, precond=pcm,
                                      inner_tol=inner_tol, max_outer=30, cert_prec=cp, check=False,
                                      timeout_s=120.0)
                torch.cuda.synchronize()
                ts = time.perf_counter() - t0
            res[name] = {"s": round(ts, 4), "iters": r["iters"], "outer": r["outer"],
                         "certified": r["status"] == 0 and r["rel_res"] <= tol,
                         "rel_res": r["rel_res"], "n_sht": r["n_sht"]}
        return {**res, "nsht_A": m.nsht_A, "nsht_M": m.nsht_M,
                "iters_M_diag_over_M_PI": round(res["M_diag"]["iters"] / max(res["M_PI"]["iters"], 1), 2),
                "time_M_diag_over_M_PI": round(res["M_diag"]["s"] / res["M_PI"]["s"], 2),
                "iters_constant_mixing_M_PI": iters_const,
                "workload": ("multires_fullsky_nside256-1024 with the dust pair of all 9 bands on "
                             "q (1 + f), f a seeded l <= 8 field in [0, 1] (max/min 2, Nmix 9), "
                             "mixing grid HEALPix Nside 1024 (L 3071); RHS + solve")}
    finally:
        m.close()


def masked_cr_measure(tol=1e-6, scale=1, max_bottom=200):
    """Planck-shaped masked constrained realization at reduced resolution (skygen.masked_cr:
    4 components, 9 HEALPix bands at Nside 128/256, galactic band |b| < 20 deg and 200 disks
    carried by every mixing map on a HEALPix Nside 256 mixing grid, CR right-hand side with
    omega_1, omega_2): FP32 transforms with double-float certification against the FP64
    solver, both with M_add; M_PI alone within a budget for contrast."""
    import torch
    import paper_1710_00621_gb300 as cw
    dev = torch.device("cuda")
    work = skygen.masked_cr(scale)
    grids = {}
    for bnd in work.bands:
        if bnd.n not in grids:
            grids[bnd.n] = cw.cmbws_plan_grid(cw.CMBWS_GRID_HEALPIX, bnd.n, bnd.lmax)
    bg = [grids[bnd.n] for bnd in work.bands]
    nmix = max(bnd.n for bnd in work.bands)
    Lmix = max(3 * nmix - 1, max(c.lmax for c in work.comps))
    mgrid = cw.cmbws_plan_grid(cw.CMBWS_GRID_HEALPIX, nmix, Lmix)
    inp = skygen.make_inputs(work, [g.pixel_coords() for g in bg], [g.pixel_weights() for g in bg])
    mz, mph = mgrid.pixel_coords()
    inside = skygen.planck_like_mask(mz, mph)
    mask = torch.as_tensor(inside, device=dev)
    keepmap = torch.as_tensor(1.0 - inside, device=dev)
    q = inp["q"]
    nb, nc = len(work.bands), len(work.comps)
    maps = [[float(q[nu, k]) * keepmap for k in range(nc)] for nu in range(nb)]
    mgs = [[mgrid] * nc for _ in range(nb)]
    ninv = [torch.as_tensor(t, device=dev) for t in inp["tau"]]
    models = {}
    for name, p in (("fp32", cw.CMBWS_FP32), ("fp64", cw.CMBWS_FP64)):
        m = cw.cmbws_model_create([c.lmax for c in work.comps], bg, inp["beams"], inp["cl"], ninv, q, p,
                                  mix_grids=mgs, mix_maps=maps)
        for k in range(nc):
            cw.cmbws_model_add_mask_precond(m, k, nmix, mask, max_bottom)
        models[name] = m
    m64 = models["fp64"]
    x_true = torch.as_tensor(inp["x_true"], device=dev)
    d = [torch.empty(g.npix, dtype=torch.float64, device=dev) for g in bg]
    cw.cmbws_project(m64, x_true, d)
    gen = torch.Generator(device=dev).manual_seed(SEED_CR)
    for nu in range(nb):
        d[nu] += torch.as_tensor(inp["noise"][nu], device=dev)
    w1 = [torch.randn(g.npix, dtype=torch.float64, device=dev, generator=gen) for g in bg]
    w2 = torch.randn(m64.nvec, dtype=torch.float64, device=dev, generator=gen)
    b = torch.empty(m64.nvec, dtype=torch.float64, device=dev)
    cw.cmbws_rhs(m64, d, b, omega1=w1, omega2=w2)
    out = {}
    xs = {}
    for name, cert in (("fp32", cw.CMBWS_FP32X2), ("fp64", cw.CMBWS_FP64)):
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = cw.cmbws_cg_solve(models[name], b, x, tol=tol, maxiter=3000, precond=2, inner_tol=1e-3,
                              max_outer=10, cert_prec=cert, timeout_s=240.0, check=False)
        torch.cuda.synchronize()
        out[name] = {"s": round(time.perf_counter() - t0, 3), "iters": r["iters"], "outer": r["outer"],
                     "rel_res": r["rel_res"], "certified": r["status"] == 0, "n_sht": r["n_sht"]}
        xs[name] = x
        print(f"[masked_cr] {name} done", file=sys.stderr, flush=True)
    # the optimized V-cycle (Sec. 4.4: J ~ I, 6 SHTs per level) in the FP32 solve
    cw.cmbws_model_set_vcycle(models["fp32"], cw.CMBWS_VCYCLE_OPTIMIZED)
    x = torch.zeros_like(b)
    cw.cmbws_apply_M_add(models["fp32"], b, x)          # plans the optimized cycle's grids
    x.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = cw.cmbws_cg_solve(models["fp32"], b, x, tol=tol, maxiter=3000, precond=2, inner_tol=1e-3,
                          max_outer=10, cert_prec=cw.CMBWS_FP32X2, timeout_s=240.0, check=False)
    torch.cuda.synchronize()
    out["fp32_optimized_vcycle"] = {"s": round(time.perf_counter() - t0, 3), "iters": r["iters"],
                                    "outer": r["outer"], "rel_res": r["rel_res"],
                                    "certified": r["status"] == 0, "n_sht": r["n_sht"],
                                    "rel_diff_vs_basic": float(torch.linalg.vector_norm(x - xs["fp32"])
                                                               / torch.linalg.vector_norm(xs["fp32"]))}
    cw.cmbws_model_set_vcycle(models["fp32"], cw.CMBWS_VCYCLE_BASIC)
    print("[masked_cr] fp32 optimized V-cycle done", file=sys.stderr, flush=True)
    out["fp32_vs_fp64_rel_diff"] = float(torch.linalg.vector_norm(xs["fp32"] - xs["fp64"])
                                         / torch.linalg.vector_norm(xs["fp64"]))
    x = torch.zeros_like(b)
    r = cw.cmbws_cg_solve(models["fp32"], b, x, tol=tol, maxiter=600, precond=1, inner_tol=1e-3,
                          max_outer=4, cert_prec=cw.CMBWS_FP32X2, timeout_s=30.0, check=False)
    out["M_PI_alone_fp32"] = {"iters": r["iters"], "certified": r["status"] == 0, "rel_res": r["rel_res"]}
    nsht_A = models["fp32"].nsht_A
    out["workload"] = (f"{work.name}: Ncomp {nc}, Nobs {nb} (Nside 128/256), L_k {work.comps[0].lmax}, "
                       f"mask {inside.mean():.1%} of the sky (|b| < 20 deg + 200 disks) in all "
                       f"{nb * nc} mixing maps on HEALPix Nside {nmix}, {nsht_A} SHTs per apply of A, "
                       "CR right-hand side, M_add = M_PI + one multigrid M_mask per component")
    return out


def _gl_problem(work, prec=None):
    """Library model + synthetic data for a workload whose bands share one GL grid."""
    import torch
    import paper_1710_00621_gb300 as cw
    dev = torch.device("cuda")
    L = work.bands[0].lmax
    g = cw.cmbws_plan_grid(cw.CMBWS_GRID_GL, L + 1, L)
    z, ph = g.pixel_coords()
    w = g.pixel_weights()
    nb = len(work.bands)
    inp = skygen.make_inputs(work, [(z, ph)] * nb, [w] * nb)
    ninv = [torch.as_tensor(t, device=dev) for t in inp["tau"]]
    m64 = cw.cmbws_model_create([c.lmax for c in work.comps], [g] * nb, inp["beams"], inp["cl"], ninv,
                                inp["q"], cw.CMBWS_FP64)
    d = [torch.empty(g.npix, dtype=torch.float64, device=dev) for _ in range(nb)]
    cw.cmbws_project(m64, torch.as_tensor(inp["x_true"], device=dev), d)
    for nu in range(nb):
        d[nu] += torch.as_tensor(inp["noise"][nu], device=dev)
    return g, inp, ninv, m64, d


def tiny_measure(reps=5):
    """The tiny two-component GL problem (L = 63, 3 bands): FP64 solve to 1e-8, launch-bound."""
    import torch
    import paper_1710_00621_gb300 as cw
    work = skygen.tiny_plain()
    g, inp, ninv, m64, d = _gl_problem(work)
    b = torch.empty(m64.nvec, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    cw.cmbws_rhs(m64, d, b)
    cw.cmbws_cg_solve(m64, b, x, tol=1e-8, maxiter=1000)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        x.zero_()
        r = cw.cmbws_cg_solve(m64, b, x, tol=1e-8, maxiter=1000)
    torch.cuda.synchronize()
    t_eager = (time.perf_counter() - t0) / reps
    x_eager = x.clone()
    cw.cmbws_model_set_graphs(m64, True)
    x.zero_()
    cw.cmbws_cg_solve(m64, b, x, tol=1e-8, maxiter=1000)   # captures the graphs
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        x.zero_()
        rg = cw.cmbws_cg_solve(m64, b, x, tol=1e-8, maxiter=1000)
    torch.cuda.synchronize()
    t_graph = (time.perf_counter() - t0) / reps
    cw.cmbws_model_set_graphs(m64, False)
    return {"s": round(t_eager, 5), "s_graphs": round(t_graph, 5), "iters": r["iters"],
            "iters_graphs": rg["iters"], "graphs_bitwise_equal": bool(torch.equal(x, x_eager)),
            "rel_res": r["rel_res"], "workload": work.name + ", FP64, M_PI, tol 1e-8"}


def differentiable_measure(L=511):
    """Gradient of ||W x||^2 of the Wiener solution with respect to the two spectral indices and
    the three prior log-amplitudes (autodiff.WienerSolution: forward solve, adjoint solve and
    cmbws_grad_terms), FP32 transforms with FP64 scalars against FP64, wall time of one
    forward + backward."""
    import torch
    import paper_1710_00621_gb300 as cw
    from paper_1710_00621_gb300.autodiff import WienerProblem, power_law_q, wiener_solution
    work = skygen.differentiable(lmax=L)
    g, inp, ninv, m64, d = _gl_problem(work)
    wgt = torch.as_tensor(skygen.harmonic_weight([c.lmax for c in work.comps]), device="cuda")
    out = {}
    grads = {}
    for name, prec, tol in (("fp32", cw.CMBWS_FP32, 1e-10), ("fp64", cw.CMBWS_FP64, 1e-10)):
        prob = WienerProblem([c.lmax for c in work.comps], [g] * len(work.bands), inp["beams"],
                             inp["cl"], ninv, d, prec=prec, tol=tol, maxiter=5000)
        ts = []
        for _ in range(2):  # the first pass builds the double-float tables
            betas = torch.tensor([0.0 if c.beta is None else c.beta for c in work.comps],
                                 dtype=torch.float64, requires_grad=True)
            logamp = torch.zeros(len(work.comps), dtype=torch.float64, requires_grad=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            q = power_law_q([bd.freq for bd in work.bands], [c.nu0 for c in work.comps], betas,
                            [c.beta is None for c in work.comps])
            loss = ((wgt * wiener_solution(q, logamp, prob)) ** 2).sum()
            loss.backward()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        gv = np.concatenate([betas.grad.numpy()[[c.beta is not None for c in work.comps]],
                             logamp.grad.numpy()])
        grads[name] = gv
        out[name] = {"forward_backward_s": round(ts[-1], 3)}
    out["max_rel_grad_diff_fp32_vs_fp64"] = float(np.max(np.abs(grads["fp32"] - grads["fp64"])
                                                         / np.abs(grads["fp64"])))
    out["workload"] = (f"{work.name}: loss ||W x||^2, gradients w.r.t. beta_synch, beta_dust and "
                       "3 prior log-amplitudes; solves certified to 1e-10")
    return out


def precision_report(nside=1024, nmaps=3, reps=3):
    """Synthesis of one full-size band grid (HEALPix Nside 1024, L = 3071, three maps) in every
    transform precision: time per call (CUDA events) and the max-relative difference from the
    FP64 synthesis of the same coefficients (a 1/(l+1) spectrum)."""
    import torch
    import paper_1710_00621_gb300 as cw
    L = 3 * nside - 1
    g = cw.cmbws_plan_grid(cw.CMBWS_GRID_HEALPIX, nside, L)
    ell = skygen.ell_of_index(L)
    rng = np.random.default_rng(11)
    a = torch.as_tensor(rng.standard_normal((nmaps, ell.size)) / (1.0 + ell), device="cuda")
    out = {}
    ref = None
    precs = [("fp64", cw.CMBWS_FP64), ("fp32x2", cw.CMBWS_FP32X2), ("fp32", cw.CMBWS_FP32),
             ("3xtf32", cw.CMBWS_3XTF32), ("tf32", cw.CMBWS_TF32), ("bf16x3", cw.CMBWS_BF16X3),
             ("bf16", cw.CMBWS_BF16)]
    for name, p in precs:
        m = torch.empty((nmaps, g.npix), dtype=torch.float64, device="cuda")
        cw.cmbws_sht_synth(g, p, a, m, nmaps)  # warm-up (lazy tables)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            cw.cmbws_sht_synth(g, p, a, m, nmaps)
        e1.record()
        torch.cuda.synchronize()
        if ref is None:
            ref = m.clone()
        err = float((m - ref).abs().max() / ref.abs().max())
        out[name] = {"ms": round(e0.elapsed_time(e1) / reps, 3), "max_rel_err_vs_fp64": err}
    out["case"] = f"synthesis, HEALPix Nside {nside}, L = {L}, {nmaps} maps, 1/(l+1) spectrum"
    out["note"] = ("tf32 / 3xtf32 / bf16 / bf16x3: Legendre contraction on the tcgen05 tensor cores "
                   "(the recurrence on the CUDA cores in FP32, as for fp32); fp32x2: double-float on "
                   "the FP32 pipe")
    return out


# Implementation flops on the FP32 pipe per (l, m, ring pair) element, as a + b * maps: FP32
# kernels 2 FMA for the recurrence + 2 per map for the contraction (the SHT flop count
# itself); double-float kernels: a double-float recurrence step costs 39 FP32 flops
# (product 10, difference 11, fused multiply-subtract 18) and one compensated Dot2 update 15
# (FMUL + 3 FFMA + 8 FADD), two per map; the synthesis steps the recurrence at every l, the
# adjoint at half of them (the other half restart from the double-float checkpoints).
IMPL_FLOPS = {("legendre_synth", "fp32"): (4.0, 4.0), ("legendre_adjoint", "fp32"): (4.0, 4.0),
              ("legendre_synth", "fp32x2"): (39.0, 30.0),
              ("legendre_adjoint", "fp32x2"): (19.5, 30.0)}


# DRAM bytes (read + write) per element from one ncu capture of the kernel as it stands (a
# smaller case of the same kernel, scaled by the elements of a full-size launch: the
# checkpoint table dominates, so the traffic grows with the elements).  Emptied whenever the
# kernel changes until it is captured again.
DRAM_BYTES_PER_ELEM = {("legendre_adjoint", "fp32x2"): 3.45}   # 4.175 GB / 1.209e9 at Nside 512


def measured_peaks():
    """HBM copy bandwidth (GB/s) from MEASURED_PEAKS.json, else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "of measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "of fallback"


def roofline(prof):
    """Dominant kernel (by summed time) among the Legendre stages, with its achieved rate.

    `achieved` is the method's own work (the SHT flop count: 4 flops per (l, m, ring pair)
    for the recurrence plus 4 per map, over the full (l, m) triangle) per second; every
    Legendre kernel of the step runs on the FP32 pipe (the FP64-accurate ones in double-float
    arithmetic), so the peak is the derived FP32 rate.  `impl_achieved` counts the FP32 flops
    the kernel's algorithm executes (IMPL_FLOPS), which for double-float is several times the
    method's."""
    best = None
    for (stage, prec), v in prof.items():
        ms, n = v[0], v[1]
        if stage not in ("legendre_synth", "legendre_adjoint") or n == 0:
            continue
        if best is None or ms > best[2]:
            best = (stage, prec, ms, n, v)
    if best is None:
        return None
    stage, prec, ms, n, v = best
    fl, elems, melems = v[2], v[3], v[4]
    achieved = fl / (ms * 1e-3) / 1e12
    out = {"bound": "alu", "kernel": f"{stage}_{prec}", "achieved": round(achieved, 3),
           "peak": round(FP32_PEAK_TFLOPS, 2), "unit": "TFLOP/s",
           "frac": round(achieved / FP32_PEAK_TFLOPS, 4), "traffic": None, "launches": n,
           "avg_launch_ms": round(ms / n, 4),
           "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz (of derived)",
           "work": "method flops: 4 (1 + maps) per (l, m, ring pair), full triangle",
           "elements_per_launch": round(elems / n)}
    ab = IMPL_FLOPS.get((stage, prec))
    if ab is not None:
        impl = (ab[0] * elems + ab[1] * melems) / (ms * 1e-3) / 1e12
        out["impl_achieved"] = round(impl, 3)
        out["impl_frac"] = round(impl / FP32_PEAK_TFLOPS, 4)
        out["impl_flops_per_element"] = round((ab[0] * elems + ab[1] * melems) / elems, 2)
    bpe = DRAM_BYTES_PER_ELEM.get((stage, prec))
    if bpe:
        out["traffic"] = round(bpe * elems / n)
    if prec == "fp32x2":
        out["note"] = ("double-float kernel (FP64-accurate on the FP32 pipe): the method's flops "
                       "cost impl_flops_per_element FP32 flops here; GB300's FP64 pipe peaks at "
                       f"{FP64_PEAK_TFLOPS} TFLOP/s")
    return out


def fft_roofline(prof):
    """The ring FFT stage with the largest summed time, as an HBM stream: algorithmic bytes
    (ring spectra read and written once, pixel factors or maps once) per second."""
    best = None
    for (stage, prec), v in prof.items():
        if stage != "ring_fft" or v[1] == 0 or v[5] <= 0:
            continue
        if best is None or v[0] > best[2]:
            best = (stage, prec, v[0], v[1], v[5])
    if best is None:
        return None
    stage, prec, ms, n, byts = best
    peak, src = measured_peaks()
    achieved = byts / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": f"{stage}_{prec}", "achieved": round(achieved, 1),
            "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
            "launches": n, "avg_launch_ms": round(ms / n, 4),
            "bytes_per_launch": round(byts / n), "peak_source": f"HBM copy bandwidth ({src})"}


def _oracle_sht_pair(args):
    """One synthesis + adjoint-synthesis pair of the FP64 oracle on a HEALPix grid (a worker of
    the CPU baseline); returns its wall time in seconds."""
    nside, seed = args
    from oracle import grids as og, sht as osht
    L = 3 * nside - 1
    g = og.healpix(nside)
    a = np.random.default_rng(seed).standard_normal((L + 1) ** 2)
    t0 = time.perf_counter()
    f = osht.synthesis(g, L, a)
    osht.adjoint(g, L, f)
    return time.perf_counter() - t0


def _oracle_warm(_):
    from oracle import grids, sht  # noqa: F401
    return os.getpid()


def cpu_baseline(work, iters_fp64, sample_nside=192):
    """The FP64 oracle on every host core: one SHT pair of the Nside-192 grid (L = 575) per core,
    run concurrently in spawned processes (single-threaded NumPy / BLAS each), scaled by ring
    pairs x (l, m) pairs to the 9 bands and by the iteration count (+ RHS + certification)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_warm, range(cores))                      # start-up outside the timing
        t0 = time.perf_counter()
        secs = pool.map(_oracle_sht_pair, [(sample_nside, i) for i in range(cores)], chunksize=1)
        wall = time.perf_counter() - t0
    L = 3 * sample_nside - 1
    unit_sample = (2 * sample_nside) * (L + 1) * (L + 2) / 2       # ring pairs x (l, m) pairs
    t_pair = wall / cores                                         # throughput of all cores
    # one PCG iteration = A + M_PI = 2 SHT pairs per band
    per_iter = 0.0
    for b in work.bands:
        per_iter += 2 * (2 * b.n) * (b.lmax + 1) * (b.lmax + 2) / 2
    iters = max(int(iters_fp64), 1) + 2                            # + RHS and certification
    est = t_pair * per_iter * iters / unit_sample
    return {"value": round(est, 1), "unit": "s", "cores": cores, "kind": "oracle",
            "threads_per_process": {"OMP_NUM_THREADS": 1, "OPENBLAS_NUM_THREADS": 1},
            "sample": (f"{cores} synthesis + adjoint-synthesis pairs of the FP64 NumPy oracle on "
                       f"the HEALPix Nside {sample_nside} grid (L = {L}), one per core in spawned "
                       f"processes, took {wall:.2f} s wall (per pair {min(secs):.2f}-{max(secs):.2f} s); "
                       f"scaled by ring pairs x (l, m) pairs to the {len(work.bands)} bands and to "
                       f"{iters} iterations ({int(iters_fp64)} PCG iterations to 1e-6 + RHS + "
                       "certification); an extrapolation")}


def oracle_iterations(tol=1e-6, scale=16):
    """PCG iterations of the oracle (M_PI, FP64) to `tol` on the benchmark model at 1/scale of
    its resolution (the pseudo-inverse preconditioner's count hardly depends on resolution)."""
    from oracle import grids as og, model as om, precond as opc
    from oracle.cg import pcg
    w = workload(scale)
    gs = [og.healpix(b.n) for b in w.bands]
    coords = [(np.cos(g.pixel_angles()[0]), g.pixel_angles()[1]) for g in gs]
    inp = skygen.make_inputs(w, coords, [g.pixel_weights() for g in gs])
    m = om.Model(lmax_comp=[c.lmax for c in w.comps], grids=gs, lmax_band=[b.lmax for b in w.bands],
                 beam=inp["beams"], cl=inp["cl"], tau=inp["tau"], q=inp["q"])
    d = [mp_ + n for mp_, n in zip(om.project(m, inp["x_true"]), inp["noise"])]
    b = om.rhs(m, d)
    _, info = pcg(lambda v: om.apply_A(m, v), b, lambda v: opc.apply_precond(m, v), tol=tol,
                  maxiter=500)
    return info["iters"]


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    work = workload(args.scale)
    iters = oracle_iterations(args.tol)
    times = []
    for _ in range(args.warmup + args.steps):
        cb = cpu_baseline(work, iters)
        times.append(cb["value"])
    v = float(np.median(times[args.warmup:])) if args.steps else times[-1]
    cb = dict(cb, value=v)
    line = {"impl": "reference", "metric": "Wiener solve time to 1e-6 residual", "value": v,
            "unit": "s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": work.name,
                       "solve": (f"oracle PCG with M_PI, {iters} iterations to {args.tol} (the "
                                 "oracle's own count on the model at 1/16 resolution), "
                                 "extrapolated from per-core SHT-pair timings")},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0,
                                         "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import paper_1710_00621_gb300 as cw
    INNER_TOL[0] = args.inner_tol
    cw.cmbws_set_autotune(args.autotune)
    rank, world, local = dist_init(args.gpus)
    work = workload(args.scale)
    P = build_problem(work, args.prec, seed_offset=rank)
    model = P["model"]
    n = model.nvec
    PREC_CODES = {"model": -1, "bf16": cw.CMBWS_BF16, "tf32": cw.CMBWS_TF32, "fp32": cw.CMBWS_FP32}
    pc_main = PREC_CODES[args.precond_prec] if args.prec == "fp32" else -1
    cw.cmbws_model_set_precond_prec(model, pc_main)
    dev = torch.device("cuda")
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    b = torch.zeros(n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    cert = args.cert if args.prec == "fp32" else "fp64"
    for _ in range(args.warmup):
        solve_step(P, model, args.tol, x, b, cert)
    torch.cuda.synchronize()

    # timed region
    clocks = ClockSampler(local)
    clocks.start()
    cw.cmbws_profile_read(reset=True)
    cw.cmbws_profile_enable(True)
    barrier(world)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    reps = []
    for _ in range(args.steps):
        reps.append(solve_step(P, model, args.tol, x, b, cert))
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    cw.cmbws_profile_enable(False)
    prof = cw.cmbws_profile_read(reset=True)
    clk = clocks.stop()
    t_step = ev0.elapsed_time(ev1) / 1e3 / max(args.steps, 1)
    t_step = max_over_ranks(t_step, world)
    launches = int(sum(v[1] for v in prof.values()))

    # accuracy of the solution against the FP64 plain solve and x_true
    rep = reps[-1]
    out = {"iters": rep["iters"], "outer": rep["outer"], "rel_res_fp64": rep["rel_res"],
           "n_sht": rep["n_sht"]}

    # end to end through the public API from pinned host memory
    e2e = None
    if not args.no_e2e:
        d_host = [t.cpu().pin_memory() for t in P["d"]]
        x_host = torch.empty(n, dtype=torch.float64).pin_memory()
        d_dev = [torch.empty_like(t) for t in P["d"]]
        Pe = dict(P)
        Pe["d"] = d_dev
        torch.cuda.synchronize()
        barrier(world)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            for dd, hh in zip(d_dev, d_host):
                dd.copy_(hh, non_blocking=True)
            solve_step(Pe, model, args.tol, x, b, cert)
            x_host.copy_(x, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        te = max_over_ranks(e0.elapsed_time(e1) / 1e3 / max(args.steps, 1), world)
        e2e = {"value": round(te, 4), "unit": "s",
               "h2d_bytes_per_step": int(sum(t.numel() * 8 for t in P["d"])),
               "d2h_bytes_per_step": int(n * 8)}

    fp64 = None
    if not args.no_fp64_plain and args.prec == "fp32":
        m64 = P["m64"]
        x64 = torch.zeros(n, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r64 = solve_step(P, m64, args.tol, x64, b, cert="fp64")
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
        diff = float(torch.linalg.vector_norm(x - x64) / torch.linalg.vector_norm(x64))
        fp64 = {"s": round(t64, 3), "iters": r64["iters"], "rel_res_fp64": r64["rel_res"],
                "mixed_vs_fp64_rel_diff": diff}
        out["iters_fp64_plain"] = r64["iters"]

    # the FP64-accurate solver on the FP32 pipe: every transform in double-float (48-bit
    # significands), the fair plain-precision comparator on a GPU whose FP64 pipe runs at a
    # 61st of the FP32 rate
    fp32x2 = None
    if not args.no_fp64_plain and args.prec == "fp32":
        try:
            inp = P["inp"]
            mdf = cw.cmbws_model_create([c.lmax for c in work.comps], P["grids"], inp["beams"],
                                        inp["cl"], P["ninv"], inp["q"], cw.CMBWS_FP32X2)
            xdf = torch.zeros(n, dtype=torch.float64, device=dev)
            for _ in range(2):                      # the first solve allocates the workspaces
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rdf = solve_step(P, mdf, args.tol, xdf, b, cert="fp32x2")
                torch.cuda.synchronize()
                tdf = time.perf_counter() - t0
            fp32x2 = {"s": round(tdf, 3), "iters": rdf["iters"], "rel_res_fp64": rdf["rel_res"],
                      "mixed_vs_fp32x2_rel_diff": float(torch.linalg.vector_norm(x - xdf)
                                                        / torch.linalg.vector_norm(xdf)),
                      "note": ("plain PCG with every transform in double-float (FP64-accurate on "
                               "the FP32 pipe), certified the same way")}
            mdf.close()
        except Exception as e:  # noqa: BLE001
            fp32x2 = {"error": f"{type(e).__name__}: {e}"[:300]}

    # the step's solve with the Legendre synthesis on the tensor cores (TF32 / BF16, single or
    # split), refined and certified like the FP32 solve
    tc_solves = None
    if not args.no_extras and args.prec == "fp32":
        tc_solves = {}
        inp = P["inp"]
        for name, pc in (("tf32", cw.CMBWS_TF32), ("3xtf32", cw.CMBWS_3XTF32),
                         ("bf16x3", cw.CMBWS_BF16X3), ("bf16", cw.CMBWS_BF16)):
            try:
                mt = cw.cmbws_model_create([c.lmax for c in work.comps], P["grids"], inp["beams"],
                                           inp["cl"], P["ninv"], inp["q"], pc)
                xt = torch.zeros(n, dtype=torch.float64, device=dev)
                for _ in range(2):                  # the first solve allocates the workspaces
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    rt = solve_step(P, mt, args.tol, xt, b, cert)
                    torch.cuda.synchronize()
                    tt = time.perf_counter() - t0
                tc_solves[name] = {"s": round(tt, 4), "iters": rt["iters"], "outer": rt["outer"],
                                   "certified": rt["status"] == 0 and rt["rel_res"] <= args.tol,
                                   "rel_diff_vs_fp32_solution": float(torch.linalg.vector_norm(xt - x)
                                                                      / torch.linalg.vector_norm(x))}
                mt.close()
            except Exception as e:  # noqa: BLE001
                tc_solves[name] = {"error": f"{type(e).__name__}: {e}"[:300]}
        # FP32 A with the preconditioner's transforms in FP32, on the tensor cores in TF32
        # (synthesis only) or in BF16 (synthesis and adjoint)
        for name, pc in (("fp32_A_fp32_precond", -1), ("fp32_A_tf32_precond", cw.CMBWS_TF32),
                         ("fp32_A_bf16_precond", cw.CMBWS_BF16)):
            try:
                cw.cmbws_model_set_precond_prec(model, pc)
                xt = torch.zeros(n, dtype=torch.float64, device=dev)
                for _ in range(2):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    rt = solve_step(P, model, args.tol, xt, b, cert)
                    torch.cuda.synchronize()
                    tt = time.perf_counter() - t0
                tc_solves[name] = {"s": round(tt, 4), "iters": rt["iters"], "outer": rt["outer"],
                                   "certified": rt["status"] == 0 and rt["rel_res"] <= args.tol,
                                   "rel_diff_vs_fp32_solution": float(torch.linalg.vector_norm(xt - x)
                                                                      / torch.linalg.vector_norm(x))}
            except Exception as e:  # noqa: BLE001
                tc_solves[name] = {"error": f"{type(e).__name__}: {e}"[:300]}
            finally:
                cw.cmbws_model_set_precond_prec(model, pc_main)

    # the paper's comparison (Sec. 5): the same solve with the block-diagonal preconditioner
    mdiag = None
    if not args.no_extras:
        try:
            xd = torch.zeros(n, dtype=torch.float64, device=dev)
            cwd = cw.CMBWS_FP32X2 if cert == "fp32x2" else cw.CMBWS_FP64
            kwd = dict(tol=args.tol, maxiter=3000, precond=3, inner_tol=args.inner_tol,
                       max_outer=20, cert_prec=cwd, timeout_s=120.0, check=False)
            cw.cmbws_cg_solve(model, b, xd, **kwd)  # builds M_diag
            res = {}
            for name, pc in (("M_PI", 1), ("M_diag", 3)):
                xd.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rd = cw.cmbws_cg_solve(model, b, xd, **{**kwd, "precond": pc})
                torch.cuda.synchronize()
                res[name] = {"s": round(time.perf_counter() - t0, 3), "iters": rd["iters"],
                             "outer": rd["outer"], "certified": rd["status"] == 0}
            mdiag = {**res, "time_ratio_M_diag_over_M_PI": round(res["M_diag"]["s"] / res["M_PI"]["s"], 2),
                     "note": ("the step's solve (right-hand side given) with M_PI and with the "
                              "block-diagonal M_diag = (U^T diag(T) U)^-1, same certification")}
        except Exception as e:  # noqa: BLE001
            mdiag = {"error": f"{type(e).__name__}: {e}"[:300]}

    crchain = None
    if not args.no_extras:
        try:
            crchain = cr_chain_measure(model, P, x, args.tol, args.inner_tol, cert)
        except Exception as e:  # noqa: BLE001
            crchain = {"error": f"{type(e).__name__}: {e}"[:300]}

    split = None
    if not args.no_extras:
        try:
            split = split_measure(P, x, args.tol, args.inner_tol, cert)
        except Exception as e:  # noqa: BLE001
            split = {"error": f"{type(e).__name__}: {e}"[:300]}

    batched = None
    if args.with_batched and args.scale == 1:
        try:
            batched = batched_measure(args.with_batched, args.tol)
        except Exception as e:  # noqa: BLE001 - reported in the line instead of losing it
            batched = {"error": f"{type(e).__name__}: {e}"[:300]}
    precision = precision_report() if (not args.no_precision and args.scale == 1) else None
    extras = {}
    if not args.no_extras and args.scale == 1:
        for key, fn in (("tiny", tiny_measure), ("differentiable", differentiable_measure)):
            try:
                extras[key] = fn()
            except Exception as e:  # noqa: BLE001
                extras[key] = {"error": f"{type(e).__name__}: {e}"[:300]}
    variable = None
    if not args.no_extras and args.prec == "fp32" and args.scale == 1:
        try:
            variable = variable_dust_measure(P, args.tol, args.inner_tol, cert, pc_main, out["iters"])
        except Exception as e:  # noqa: BLE001 - reported in the line instead of losing it
            variable = {"error": f"{type(e).__name__}: {e}"[:300]}
    masked_cr = None
    if not args.no_masked_cr and args.scale == 1:
        try:
            masked_cr = masked_cr_measure(args.tol)
        except Exception as e:  # noqa: BLE001 - reported in the line instead of losing it
            masked_cr = {"error": f"{type(e).__name__}: {e}"[:300]}

    if rank != 0:
        return
    rl = roofline(prof)
    frl = fft_roofline(prof)
    cb = cpu_baseline(work, out.get("iters_fp64_plain", out["iters"])) if world == 1 else None
    stages = {f"{k[0]}_{k[1]}": {"ms": round(v[0], 3), "launches": v[1]} for k, v in prof.items() if v[1]}
    line = {"metric": "Wiener solve time to 1e-6 residual", "value": round(t_step, 4), "unit": "s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(t_step * 1e3, 2), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None,
            "dtype": ("f32+bf16+f64" if args.precond_prec == "bf16" else "f32+f64")
                     if args.prec == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": work.name, "ncomp": len(work.comps), "nobs": len(work.bands),
                       "band_nside": [b.n for b in work.bands], "lmax_comp": [c.lmax for c in work.comps],
                       "tol": args.tol, "inner_tol": args.inner_tol, "precond": "M_PI",
                       "precond_arith": ({"model": "fp32", "bf16": "bf16 (tcgen05 synthesis and adjoint)",
                                          "tf32": "tf32 synthesis (tcgen05), fp32 adjoint",
                                          "fp32": "fp32"}[args.precond_prec]
                                         if args.prec == "fp32" else "fp64"),
                       "arithmetic": ("FP32 transforms, FP64 vectors/scalars, iterative refinement "
                                      f"certified by FP64-accurate ({cert}) applies"
                                      if args.prec == "fp32" else "FP64"),
                       "l2": "inputs larger than L2, no flush",
                       "synthesis_tiles": ["default", "heuristic", "autotuned"][args.autotune],
                       "parallelism": f"replicas x{world}"},
            "solve": out, "fp64_plain": fp64, "fp32x2_plain": fp32x2,
            "tensor_core_solves": tc_solves, "batched": batched,
            "masked_cr": masked_cr, "variable_dust": variable,
            "tiny": extras.get("tiny"), "differentiable": extras.get("differentiable"),
            "M_diag_comparison": mdiag,
            "cr_chain": crchain,
            "detector_splits": split,
            "precision": precision,
            "roofline": rl, "roofline_ring_fft": frl, "cpu_baseline": cb, "e2e": e2e,
            "gpu_launches": launches, "stages": stages, "clocks": clk}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
