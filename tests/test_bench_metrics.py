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


def test_whole_step_call_sequence():
    """The default step's calls on a recording context: one integral build and
    one Omega, the valence vectors' rho and sigma with the skip rule off, then
    the core state's with it on, densities and f for every state, and the byte
    tally of what crosses the boundary."""
    import numpy as np
    torch = __import__("pytest").importorskip("torch")
    calls = []

    class Rec:
        def __getattr__(self, name):
            def f(*a):
                calls.append((name, a))
                return 0.5 if name == "oscillator_strength" else None
            return f
    NO, NV, no, nv, NJ = 4, 9, 3, 4, 6
    x, omega = bench.device_system(NO, NV, no, nv, NJ, 3, 1, torch.device("cpu"), True, cvs_last=1)
    assert omega[2] == 10.2 and float(x["R1"][2][:, 1:].abs().max()) == 0.0
    prob = bench.WholeProblem(x, omega, 2, 1)
    o = bench.WholeProblem.outputs(x, 2, torch.zeros_like)
    tally = {"in": 0, "out": 0}

    def count(kind, *arrs):
        tally[kind] += sum(a.numel() * a.element_size() for a in arrs)
    fs = prob.step(Rec(), x, o, tally=count)
    names = [c[0] for c in calls]
    assert names.count("build_integrals") == 1 and names.count("triples_omega") == 1
    assert names.count("jacobian_right") == 2 and names.count("transition_densities") == 2
    td = [c[1] for c in calls if c[0] == "transition_densities"]
    assert len(td[0][0]) == 2 and list(td[1][0]) == [10.2]
    assert fs == [0.5, 0.5, 0.5]
    cvs = [c[1][1] for c in calls if c[0] == "set_param"]
    assert cvs == [0, 1, 1]
    jr = [c[1] for c in calls if c[0] == "jacobian_right"]
    assert len(jr[0][0]) == 2 and list(jr[1][0]) == [10.2]
    assert tally["in"] > x["chol"].numel() * 8 and tally["out"] > 0


def test_site_totals_merge_chunks():
    stats = {"bstc_gemv_kernel:o#1g0:y3d": (4, 2.0, 0.0), "bstc_gemv_kernel:o#1g1:y3d": (4, 4.0, 0.0),
             "tc_gemm_kernel:build": (6, 10.0, 1e12), "contra3_kernel": (2, 0.5, 0.0)}
    got = bench.site_totals(stats, 2)
    assert got == {"tc_gemm_kernel:build": 5.0, "bstc_gemv_kernel:y3d": 3.0}
