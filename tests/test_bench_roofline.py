"""Host logic of bench.py's roofline object (no GPU): the dominant Legendre stage, the
achieved rate from the algorithmic flops per element, the scaled DRAM traffic."""
import math

import bench


def _prof(entries):
    """entries: {(stage, prec): (ms, launches, profiler_flops)}"""
    return dict(entries)


def test_dominant_stage_and_achieved_rate():
    elems = 9.7e9                                  # (l, m, ring pair) elements per launch
    fl = 16.0 * elems                              # the profiler counts 4 (NM + 1) flops, NM = 3
    prof = _prof({("legendre_adjoint", "fp32x2"): (30.0, 3, 3 * fl),
                  ("legendre_adjoint", "fp32"): (20.0, 6, 6 * fl),
                  ("ring_fft", "fp32"): (100.0, 6, 0.0)})      # not a Legendre stage
    r = bench.roofline(prof)
    assert r["kernel"] == "legendre_adjoint_fp32x2" and r["launches"] == 3
    per = bench.FP32_FLOPS_PER_ELEM[("legendre_adjoint", "fp32x2")]
    assert math.isclose(r["achieved"], 3 * elems * per / 30e-3 / 1e12, rel_tol=1e-3)
    assert math.isclose(r["frac"], r["achieved"] / bench.FP32_PEAK_TFLOPS, rel_tol=1e-3)
    assert math.isclose(r["avg_launch_ms"], 10.0)
    # traffic: bytes per element from the capture x elements of one launch
    bpe = bench.DRAM_BYTES_PER_ELEM.get(("legendre_adjoint", "fp32x2"))
    if bpe is None:
        assert r["traffic"] is None
    else:
        assert math.isclose(r["traffic"], bpe * elems, rel_tol=1e-6)


def test_fp32_stage_has_no_traffic_figure_and_peak_is_derived():
    fl = 16.0 * 1e9
    r = bench.roofline(_prof({("legendre_synth", "fp32"): (5.0, 2, 2 * fl)}))
    assert r["kernel"] == "legendre_synth_fp32" and r["traffic"] is None
    assert math.isclose(bench.FP32_PEAK_TFLOPS, 152 * 128 * 2 * 2.070e9 / 1e12)
    assert math.isclose(r["achieved"], 2e9 * 16.0 / 5e-3 / 1e12, rel_tol=1e-3)


def test_no_legendre_stage_gives_none():
    assert bench.roofline(_prof({("ring_fft", "fp32"): (1.0, 1, 0.0)})) is None
