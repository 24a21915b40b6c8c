"""Throughput microbenchmarks that give the compression's roofline its
denominators (run with -m gpu): measured FP32 FMA, special-function and
FP64 FMA rates, checked for plausibility against the SM count and a clock
range (no vendor figure is assumed beyond the order of magnitude)."""
import pytest

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_plausible():
    import torch
    import paper_2505_00715_gb300 as td
    ctx = td.Context(0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    f32, sfu, f64 = ctx.measure_peak("fma32"), ctx.measure_peak("sfu"), ctx.measure_peak("fma64")
    p64 = ctx.measure_peak("pair64")
    print("per SM and clock at 2 GHz: FP32 FMA %.1f, SFU %.2f, FP64 FMA %.2f; totals %.3e / %.3e / %.3e per s; "
          "FP64 point pairs %.3e per s" % (f32 / sms / 2e9, sfu / sms / 2e9, f64 / sms / 2e9, f32, sfu, f64, p64))
    # between a quarter of and twice one warp-wide FMA issue per SM sub-partition and clock at 1-2.5 GHz
    assert 32 * sms * 1e9 < f32 < 256 * sms * 2.5e9
    assert 1 * sms * 1e9 < sfu < f32
    assert 0 < f64 < f32 / 4
    # an FP64 point pair (square root, exponential, sine, cosine, division) costs many FP64 FMAs
    assert f64 / 500 < p64 < f64 / 5
    with pytest.raises(KeyError):
        ctx.measure_peak("tensor")
