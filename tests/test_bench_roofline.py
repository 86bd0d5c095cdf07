"""Host logic of bench.py's roofline objects (no GPU): the dominant Legendre stage and its
method-flop rate, the implementation-flop rate with mixed map counts, the scaled DRAM
traffic, and the ring FFT as an HBM stream."""
import math

import bench


def _rec(ms, n, launches_maps):
    """A profiler record (ms, launches, flops, elements, elements x maps, bytes) for launches
    given as [(elements, maps), ...]."""
    el = sum(e for e, _ in launches_maps)
    me = sum(e * k for e, k in launches_maps)
    return (ms, n, 4.0 * (el + me), el, me, 0.0)


def test_dominant_stage_method_rate_and_mixed_map_counts():
    # three launches of 3 maps and one of 1 map: the method flops and the implementation
    # flops are linear in the maps, so both follow from the summed counts
    lm = [(9.7e9, 3), (9.7e9, 3), (9.7e9, 3), (1.2e9, 1)]
    prof = {("legendre_adjoint", "fp32x2"): _rec(30.0, 4, lm),
            ("legendre_adjoint", "fp32"): _rec(20.0, 6, [(9.7e9, 3)] * 6),
            ("ring_fft", "fp32"): (100.0, 6, 0.0, 0.0, 0.0, 6e9)}      # not a Legendre stage
    r = bench.roofline(prof)
    assert r["kernel"] == "legendre_adjoint_fp32x2" and r["launches"] == 4
    method = sum(4.0 * e * (1 + k) for e, k in lm)
    assert math.isclose(r["achieved"], method / 30e-3 / 1e12, rel_tol=1e-3)
    assert math.isclose(r["frac"], r["achieved"] / bench.FP32_PEAK_TFLOPS, rel_tol=1e-3)
    a, b = bench.IMPL_FLOPS[("legendre_adjoint", "fp32x2")]
    impl = sum(e * (a + b * k) for e, k in lm)
    assert math.isclose(r["impl_achieved"], impl / 30e-3 / 1e12, rel_tol=1e-3)
    assert math.isclose(r["avg_launch_ms"], 7.5)
    bpe = bench.DRAM_BYTES_PER_ELEM.get(("legendre_adjoint", "fp32x2"))
    if bpe is None:
        assert r["traffic"] is None
    else:
        assert math.isclose(r["traffic"], bpe * sum(e for e, _ in lm) / 4, rel_tol=1e-6)


def test_fp32_stage_rate_equals_its_method_rate():
    r = bench.roofline({("legendre_synth", "fp32"): _rec(5.0, 2, [(1e9, 3), (1e9, 3)])})
    assert r["kernel"] == "legendre_synth_fp32" and r["traffic"] is None
    assert math.isclose(bench.FP32_PEAK_TFLOPS, 152 * 128 * 2 * 2.070e9 / 1e12)
    assert math.isclose(r["achieved"], 2e9 * 16.0 / 5e-3 / 1e12, rel_tol=1e-3)
    assert math.isclose(r["achieved"], r["impl_achieved"], rel_tol=1e-6)


def test_ring_fft_is_reported_against_hbm():
    prof = {("ring_fft", "fp32"): (40.0, 10, 0.0, 0.0, 0.0, 2e10),
            ("ring_fft", "fp32x2"): (10.0, 2, 0.0, 0.0, 0.0, 1e10)}
    r = bench.fft_roofline(prof)
    peak, _ = bench.measured_peaks()
    assert r["kernel"] == "ring_fft_fp32" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert math.isclose(r["achieved"], 2e10 / 40e-3 / 1e9, rel_tol=1e-3)
    assert math.isclose(r["frac"], r["achieved"] / peak, rel_tol=1e-3)
    assert r["bytes_per_launch"] == 2e9


def test_no_legendre_stage_gives_none():
    assert bench.roofline({("ring_fft", "fp32"): (1.0, 1, 0.0, 0.0, 0.0, 1.0)}) is None
    assert bench.fft_roofline({("legendre_synth", "fp32"): _rec(1.0, 1, [(1e6, 1)])}) is None
