"""symba_measure_rates, the probe whose figures the benchmark's rooflines divide by (needs a
GB300).  The figures must be plausible for the part -- they are measurements, so the test bounds
them loosely: a whole-device FP64 FMA rate within a factor of two of the GB300's 1.2 TFLOP/s, one
warp's FP64 issue interval between 8 and 256 cycles with independent chains no faster than a
dependent one by more than rounding (the per-warp limit the recursion's roofline rests on), and
a positive named-barrier round trip."""
import pytest

pytestmark = pytest.mark.gpu


def test_measured_rates_are_plausible():
    import paper_2304_07325_gb300 as sy
    from paper_2304_07325_gb300 import build
    build.build()
    r = sy.measure_rates()
    assert 0.6e12 < r["fp64_flops"] < 2.5e12, r
    assert 8.0 < r["warp_dfma_dep_cycles"] < 256.0, r
    assert r["warp_dfma_4chain_cycles"] > 0.5 * r["warp_dfma_dep_cycles"], r
    assert 0.0 < r["named_barrier_round_trip_cycles"] < 10000.0, r
    assert r["sms"] >= 1
    # a NULL output array is refused without touching the device
    assert sy.lib().symba_measure_rates(None) == sy.SYMBA_E_INVAL
