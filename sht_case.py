"""Run and time one transform case of the library (used for kernel profiling).

    python sht_case.py --grid healpix --n 1024 --lmax 3071 \
        --nmaps 3 --prec fp32 --op both --reps 3

Plans the grid, fills random band-limited coefficients / maps on the device, runs the
requested transforms `reps` times and prints the per-call time from CUDA events and the
library's per-stage kernel timing.
"""
import argparse
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


def main():
    import torch

    import paper_1710_00621_gb300 as cw
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", default="healpix", choices=["healpix", "gl"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--lmax", type=int, default=3071)
    ap.add_argument("--nmaps", type=int, default=3)
    ap.add_argument("--prec", default="fp32",
                    choices=["fp32", "fp64", "fp32x2", "tf32", "3xtf32", "bf16", "bf16x3"])
    ap.add_argument("--op", default="both", choices=["synth", "analysis", "both", "apply"],
                    help="apply: y = A x of a one-component model with nmaps bands on the grid "
                         "(synthesis, fused ring FFT with the N^-1 multiply, adjoint)")
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args()
    kind = cw.CMBWS_GRID_HEALPIX if a.grid == "healpix" else cw.CMBWS_GRID_GL
    g = cw.cmbws_plan_grid(kind, a.n if a.grid == "healpix" else a.n + 1, a.lmax)
    prec = {"fp32": cw.CMBWS_FP32, "fp64": cw.CMBWS_FP64, "fp32x2": cw.CMBWS_FP32X2,
            "tf32": cw.CMBWS_TF32, "3xtf32": cw.CMBWS_3XTF32, "bf16": cw.CMBWS_BF16,
            "bf16x3": cw.CMBWS_BF16X3}[a.prec]
    nalm = (a.lmax + 1) ** 2
    dev = torch.device("cuda")
    gen = torch.Generator(device=dev).manual_seed(0)
    alm = torch.randn(a.nmaps * nalm, dtype=torch.float64, device=dev, generator=gen)
    maps = torch.empty(a.nmaps * g.npix, dtype=torch.float64, device=dev)
    back = torch.empty_like(alm)
    cw.cmbws_sht_synth(g, prec, alm, maps, a.nmaps)
    model = None
    if a.op == "apply":
        ninv = [1.0 + torch.rand(g.npix, dtype=torch.float64, device=dev, generator=gen)
                for _ in range(a.nmaps)]
        beams = [np.ones(a.lmax + 1)] * a.nmaps
        model = cw.cmbws_model_create([a.lmax], [g] * a.nmaps, beams, [np.ones(a.lmax + 1)], ninv,
                                      np.ones((a.nmaps, 1)), prec)
        x = torch.randn(nalm, dtype=torch.float64, device=dev, generator=gen)
        y = torch.empty_like(x)
        cw.cmbws_apply_A(model, x, y)
    torch.cuda.synchronize()
    cw.cmbws_profile_read(reset=True)
    cw.cmbws_profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        if a.op == "apply":
            cw.cmbws_apply_A(model, x, y)
        if a.op in ("synth", "both"):
            cw.cmbws_sht_synth(g, prec, alm, maps, a.nmaps)
        if a.op in ("analysis", "both"):
            cw.cmbws_sht_analysis(g, prec, maps, back, a.nmaps, 1)
    e1.record()
    torch.cuda.synchronize()
    cw.cmbws_profile_enable(False)
    prof = cw.cmbws_profile_read(reset=True)
    out = {"case": vars(a), "ms_per_rep": e0.elapsed_time(e1) / a.reps,
           "stages": {f"{k[0]}_{k[1]}": {"ms": round(v[0], 3), "launches": v[1],
                                          "tflops": round(v[2] / (v[0] * 1e-3) / 1e12, 3) if v[0] else 0,
                                          "gbs": round(v[5] / (v[0] * 1e-3) / 1e9, 1) if v[0] else 0}
                      for k, v in prof.items() if v[1]}}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
