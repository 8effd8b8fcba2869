"""Host arithmetic of bench.py's roofline lines, on CPU: the per-call-site
tensor-core fractions count three BF16 products per algorithmic product against
the given peak, and kernels that are not tensor-core call sites are left out."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_tc_site_fracs():
    # (launches, ms, algorithmic flop) over 2 steps
    stats = {"tc_gemm_kernel:pair": (10, 4.0, 2.0e12),
             "tc_gemm_kernel:build": (6, 2.0, 0.5e12),
             "contra3_kernel": (3, 1.0, 0.0)}
    got = bench.tc_site_fracs(stats, 2, 1500.0)
    assert set(got) == {"pair", "build"}
    assert got["pair"]["ms"] == 2.0
    # 3 * 2e12 flop in 4 ms = 1500 TFLOP/s of BF16 products: the whole peak
    assert abs(got["pair"]["frac"] - 1.0) < 1e-12
    assert abs(got["build"]["frac"] - 0.5) < 1e-12


def test_tc_site_fracs_zero_time():
    got = bench.tc_site_fracs({"tc_gemm_kernel:xt": (1, 0.0, 1.0e9)}, 1, 1700.0)
    assert got["xt"]["frac"] is None


def test_clock_summary_counts_samples_inside_the_timed_region():
    c = bench.ClockSampler(0)
    row = lambda mhz, cap: [str(mhz), "2070", "900.0", "0x0", "Not Active", "Not Active",
                            "Not Active", "Active" if cap else "Not Active"]
    # one row before the region (sampler start), three inside
    c.rows = [row(1200, False), row(2070, True), row(2055, False), row(2070, False)]
    c.first = 1
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and "note" not in s
    # a region shorter than the sampling interval: the last earlier row, flagged
    c.first = 4
    s = c.summary()
    assert s["samples"] == 0 and s["sm_mhz"] == 2070.0 and "note" in s
