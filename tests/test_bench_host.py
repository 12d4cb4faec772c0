"""Host-side pieces of bench.py (no GPU): the algorithmic flop count behind
roofline.achieved, the forms table, the clock-sample summary and the
workload description."""
import bench


def test_forms_table():
    assert bench.FORMS["fp64"] == (0, 0, 0)
    assert bench.FORMS["fp32_newton_gated"] == (1, 1, 1)
    assert set(bench.FORMS) == {"fp32", "fp64", "fp32_newton", "fp64_newton",
                                "fp64_newton_gated", "fp32_newton_gated"}


def test_flops_bisection_counts_every_term():
    n, pairs = 1001, 1000
    # all-FP64 bisection, 50 steps each, double-double b, vectors
    f = bench.eig_kernel_flops(n, pairs, 50 * pairs, 0)
    terms = n - 2
    expect = terms * (3.0 * 50 * pairs + 3.0 * pairs + 20.0 * pairs) + 6.0 * (n - 1) * pairs
    assert f == expect
    # remedy steps are not k_eig's
    assert bench.eig_kernel_flops(n, pairs, 50 * pairs + 7, 7) == expect


def test_flops_gate_derivatives_and_midpoint():
    n, pairs = 101, 100
    base = dict(n=n, ncomp=pairs, total_iter=120, fix_iter=20)
    g = bench.eig_kernel_flops(**base, n_ddb=5)
    dd = bench.eig_kernel_flops(**base)
    # a standard b costs 3 a term instead of 20; the gate's double-double
    # recomputations run after their standard pass (3 + 20)
    assert dd - g == (n - 2) * (20.0 * pairs - (3.0 * pairs + 20.0 * 5))
    # each derivative adds 3 a term
    assert bench.eig_kernel_flops(**base, total_deriv=10) - dd == (n - 2) * 30.0
    # midpoint tests settled in FP32 are not FP64 flops
    assert dd - bench.eig_kernel_flops(**base, n_mid=4) == (n - 2) * 3.0 * (pairs - 4)


def test_form_flops_uses_the_forms_counters():
    info = {"n_reduced": 100, "total_iter": 150, "fix_iter": 30, "n_ddb": 7,
            "total_deriv": 11, "n_mid64": 3}
    n = 101
    assert bench.form_flops(n, info, "fp64_newton") == bench.eig_kernel_flops(
        n, 100, 150, 30, None, 11, n_mid=None)
    assert bench.form_flops(n, info, "fp32_newton_gated") == bench.eig_kernel_flops(
        n, 100, 150, 30, 7, 11, n_mid=3)


def test_clock_summary():
    c = bench.Clocks(0)
    c.rows = [["0", "2070", "2070", "900.1", "0x0", "Not Active", "Not Active", "Not Active",
               "Active"],
              ["0", "2055", "2070", "950.0", "0x0", "Not Active", "Not Active", "Not Active",
               "Not Active"],
              ["0", "2070", "2070", "990.0", "0x0", "Not Active", "Not Active", "Not Active",
               "Not Active"]]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3
    assert bench.Clocks(0).summary()["reasons"] == ["unsampled"]


def test_workload_config():
    c = bench.workload_config(16384, "fp32_newton_gated", 2)
    assert c["n"] == 16384 and c["form"] == "fp32_newton_gated"
    assert c["parallelism"] == "2 independent instances"
    assert "16384" in c["workload"]
