"""Host-side pieces of bench.py (no GPU): the algorithmic flop count behind
roofline.achieved, the forms table, the clock-sample summary and the
workload description."""
import numpy as np

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


def test_fp64_instruction_model():
    info = {"n_reduced": 100, "total_iter": 130, "fix_iter": 10, "n_ddb": 7,
            "total_deriv": 20, "n_mid64": 3}
    n = 101
    c = bench.INSTR_PER_TERM
    got = bench.fp64_instructions(n, info, "fp32_newton_gated")
    per_terms = (c["mid"] * 3 + c["b_std"] * 100 + c["b_dd"] * 7 + c["eval"] * 120 +
                 c["deriv"] * 20)
    assert got == (n - 2) * per_terms + c["vector"] * 100 * (n - 1)
    # without the gate every b is double-double; in FP64 every midpoint test runs
    got = bench.fp64_instructions(n, info, "fp64_newton")
    per_terms = c["mid"] * 100 + c["b_dd"] * 100 + c["eval"] * 120 + c["deriv"] * 20
    assert got == (n - 2) * per_terms + c["vector"] * 100 * (n - 1)


def test_remedy_work():
    info = {"n_dpr1shift": 3, "n_nearzero": 1, "n_otherpole": 2, "fix_iter": 9}
    c = bench.INSTR_PER_TERM
    fl, ins = bench.remedy_work(info, 50.0)
    assert fl == 50.0 * (20.0 * 4 + 3.0 * 2 + 3.0 * 9) + 6.0 * 51.0 * 6
    assert ins == 50.0 * (c["b_dd"] * 4 + c["b_std"] * 2 + c["eval"] * 9) + c["vector"] * 51.0 * 6
    none = {"n_dpr1shift": 0, "n_nearzero": 0, "n_otherpole": 0, "fix_iter": 0}
    assert bench.remedy_work(none, 50.0) == (0.0, 0.0)


def test_fp32_flops_and_roofline_numbers():
    info = {"n_f32_passes": 10, "n_df_passes": 4}
    f = bench.FP32_FLOPS_PER_TERM
    assert bench.fp32_flops(52, info) == 50 * (f["f32"] * 10 + f["df"] * 4)
    peaks = {"fp64_tflops": 1.0, "fp32_tflops": 64.0}
    r = bench.roofline_numbers(0.5e12, 0.25e12, 16e12, 1.0, peaks)
    assert r["achieved"] == 0.5 and r["frac"] == 0.5
    # 0.25e12 FMA lane-instructions at 0.5e12 a second: half the pipe's time
    assert r["fp64_pipe_busy_implied"] == 0.5
    # FP32 needs 0.25 s, FP64 0.5 s: the FP64 pipe bounds
    assert r["mixed"]["frac"] == 0.5 and r["mixed"]["t_fp32_ms"] == 250.0


def test_batch_terms_weights_by_eigenpairs():
    assert bench.batch_terms([10]) == 8.0
    # 10 eigenpairs of 8 terms and 30 of 28 terms
    assert bench.batch_terms([10, 30]) == (10 * 8 + 30 * 28) / 40


def test_reference_arm_keeps_every_core_busy():
    for t in (1, 8, 16):
        assert bench.reference_per_step(t) >= 4 * t


def test_error_summary_and_parity_flag():
    n = 100
    res = {"lam": np.array([1.0, -2.0, 0.0]), "abserr": np.array([0.0, 0.0, 1e-30]),
           "V": np.eye(3)}
    e = bench.max_err_neps(np.array([1.0, -2.0 * (1 + 5 * n * bench.EPS64), 0.0]),
                           np.eye(3), res, n)
    assert abs(e["lambda"] - 5.0) < 1e-9 and e["vectors"] == 0.0
    # the exact zero is compared against the oracle's bound (counted as widened)
    assert e["widened"] == 1 and e["pairs"] == 3
    assert bench.err_ok(e) and bench.err_ok(None)
    e["vectors"] = 10.5
    assert not bench.err_ok(e)


def test_sample_positions():
    ks = bench.sample_ks(1000, 64)
    assert ks[0] == 0 and ks[-1] == 999 and 500 in ks and np.all(np.diff(ks) > 0)
