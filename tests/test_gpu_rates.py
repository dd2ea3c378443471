"""The rate probe behind the FP64/FP32 roofline denominators."""
import pytest

pytestmark = pytest.mark.gpu


def test_measured_rates_are_consistent():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2506_09743_gb300 import _lib

    r = _lib.measure_rates()
    assert all(v > 0 for v in r.values()), r
    # FP32 FMA issue is tens of times the FP64 FMA rate on this part, and each
    # FP64 special function costs at least one FMA
    assert r["fp32_fma_per_s"] > 10 * r["fp64_fma_per_s"], r
    for k in ("fp64_exp_per_s", "fp64_sqrt_per_s", "fp64_recip_per_s"):
        assert r[k] < r["fp64_fma_per_s"], (k, r)
    print(r)
